"""Closed-form tree-level results used to pin the oracle.

* e+e- -> mu+mu- through photon and Z, massless fermions, per helicity:
  with A_ij = e^2 Qe Qmu / s + g_i(e) g_j(mu) / (s - mZ^2 + i mZ GammaZ), i, j in {L, R},
  gL = e (T3 - Q sw^2)/(sw cw), gR = -e Q sw^2/(sw cw):
    |M|^2 = s^2 |A_ij|^2 (1 + cos th)^2  for i = j,   s^2 |A_ij|^2 (1 - cos th)^2 for i != j,
  th the angle between e- and mu-; every other helicity configuration vanishes.
* g g -> Q Qbar (Combridge 1979; Ellis-Stirling-Webber, "QCD and collider
  physics", Eq. 10.12), spin- and colour-averaged, with tau1 = 2 p1.p3/s,
  tau2 = 2 p2.p3/s, rho = 4 m^2/s:
    g^4 (1/(6 tau1 tau2) - 3/8) (tau1^2 + tau2^2 + rho - rho^2/(4 tau1 tau2)).
* g g -> g g, averaged: (9/2) g^4 (3 - t u/s^2 - s u/t^2 - s t/u^2).
"""
import math
import numpy as np

from .model import Params, PARTICLES


def _dot(a, b):
    return a[..., 0] * b[..., 0] - (a[..., 1:] * b[..., 1:]).sum(-1)


def eemumu_helicity(p, params=None):
    """|M|^2 for the 16 helicities of e+ e- > mu+ mu- (order e+, e-, mu+, mu-): [nevt, 16]."""
    prm = params or Params()
    s = 2.0 * _dot(p[:, 0], p[:, 1])
    pem = p[:, 1, 1:]
    pmu = p[:, 3, 1:]
    cth = (pem * pmu).sum(-1) / np.sqrt((pem ** 2).sum(-1) * (pmu ** 2).sum(-1))
    e = prm.ee
    ge = prm.z_couplings(PARTICLES["e-"])
    gm = prm.z_couplings(PARTICLES["mu-"])
    prop = 1.0 / (s - prm.mz ** 2 + 1j * prm.mz * prm.wz)
    out = np.zeros((p.shape[0], 16))
    for i in range(2):          # e- chirality: 0 = L (helicity -1), 1 = R (+1)
        for j in range(2):      # mu- chirality
            A = e * e * 1.0 / s + ge[i] * gm[j] * prop
            ang = (1.0 + cth) ** 2 if i == j else (1.0 - cth) ** 2
            val = s * s * np.abs(A) ** 2 * ang
            # massless: e+ has helicity opposite to e-, mu+ opposite to mu-
            he_m, hm_m = i, j
            he_p, hm_p = 1 - i, 1 - j
            h = (he_p << 3) | (he_m << 2) | (hm_p << 1) | hm_m
            out[:, h] = val
    return out


def eemumu_qed_average(p, params=None):
    prm = params or Params()
    pem, pmu = p[:, 1, 1:], p[:, 3, 1:]
    cth = (pem * pmu).sum(-1) / np.sqrt((pem ** 2).sum(-1) * (pmu ** 2).sum(-1))
    return prm.ee ** 4 * (1.0 + cth ** 2)


def ggQQ_average(p, alpha_s, mass):
    s = 2.0 * _dot(p[:, 0], p[:, 1])
    t1 = 2.0 * _dot(p[:, 0], p[:, 2]) / s
    t2 = 2.0 * _dot(p[:, 1], p[:, 2]) / s
    rho = 4.0 * mass * mass / s
    g4 = (4.0 * math.pi * np.asarray(alpha_s)) ** 2
    return g4 * (1.0 / (6.0 * t1 * t2) - 3.0 / 8.0) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4.0 * t1 * t2))


def gggg_average(p, alpha_s):
    s = 2.0 * _dot(p[:, 0], p[:, 1])
    t = -2.0 * _dot(p[:, 0], p[:, 2])
    u = -2.0 * _dot(p[:, 0], p[:, 3])
    g4 = (4.0 * math.pi * np.asarray(alpha_s)) ** 2
    return 4.5 * g4 * (3.0 - t * u / s ** 2 - s * u / t ** 2 - s * t / u ** 2)
