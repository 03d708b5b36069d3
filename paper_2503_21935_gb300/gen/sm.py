"""Standard-Model content used by the process compiler.

Each particle: spin kind ('F' Dirac fermion, 'V' vector), colour (1, 3, -3, 8),
electric charge Q and weak isospin T3 of the particle (not the antiparticle).
The electroweak couplings follow from {alpha(mZ), G_F, mZ}:
  mW^2 = mZ^2/2 + sqrt(mZ^4/4 - pi alpha mZ^2 / (sqrt2 G_F)),  sw^2 = 1 - mW^2/mZ^2,
  photon vertex -i e Q gamma^mu,  Z vertex -i gamma^mu (gL P_L + gR P_R),
  gL = e (T3 - Q sw^2)/(sw cw),  gR = -e Q sw^2/(sw cw).
"""
import math

# name: (kind, colour, charge, t3, antiparticle, is_antiparticle, mass parameter, width parameter)
_TABLE = {}


def _pair(p, ap, colour, q, t3, mass="", width=""):
    _TABLE[p] = ("F", colour, q, t3, ap, False, mass, width)
    _TABLE[ap] = ("F", -colour if colour == 3 else colour, q, t3, p, True, mass, width)


_pair("e-", "e+", 1, -1.0, -0.5)
_pair("mu-", "mu+", 1, -1.0, -0.5)
_pair("ta-", "ta+", 1, -1.0, -0.5, "mta")
_pair("u", "u~", 3, 2.0 / 3.0, 0.5)
_pair("t", "t~", 3, 2.0 / 3.0, 0.5, "mt", "wt")
_TABLE["g"] = ("V", 8, 0.0, 0.0, "g", False, "", "")
_TABLE["a"] = ("V", 1, 0.0, 0.0, "a", False, "", "")
_TABLE["z"] = ("V", 1, 0.0, 0.0, "z", False, "mz", "wz")


def kind(p):
    return _TABLE[p][0]


def colour(p):
    return _TABLE[p][1]


def anti(p):
    return _TABLE[p][4]


def is_anti(p):
    return _TABLE[p][5]


def mass_param(p):
    return _TABLE[p][6]


def width_param(p):
    return _TABLE[p][7]


def charge(p):
    """Charge of the particle species of the line (fermion, not antifermion)."""
    return _TABLE[p][2]


def t3(p):
    return _TABLE[p][3]


def known(p):
    return p in _TABLE


def ew_couplings(alpha_em, gf, mz):
    """(e, sw2, sw, cw) in the {alpha, G_F, mZ} scheme."""
    e = math.sqrt(4.0 * math.pi * alpha_em)
    mz2 = mz * mz
    mw2 = 0.5 * mz2 + math.sqrt(0.25 * mz2 * mz2 - math.pi * alpha_em * mz2 / (math.sqrt(2.0) * gf))
    sw2 = 1.0 - mw2 / mz2
    return e, sw2, math.sqrt(sw2), math.sqrt(1.0 - sw2)
