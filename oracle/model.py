"""Standard-Model particle content and parameters for the oracle.

Electroweak input scheme {alpha(mZ), G_F, mZ} (the scheme of MadGraph's default
SM model; the paper gives no EW scheme):
  mW^2 = mZ^2/2 + sqrt(mZ^4/4 - pi*alpha*mZ^2/(sqrt(2) G_F)),  sw^2 = 1 - mW^2/mZ^2.
"""
import math
from dataclasses import dataclass


@dataclass(frozen=True)
class Particle:
    name: str
    anti: str
    spin: int       # 1 = Dirac fermion (spin 1/2), 2 = vector
    colour: int     # 1, 3, -3, 8
    charge: float   # electric charge in units of e (particle, not antiparticle)
    t3: float       # weak isospin of the left-handed particle
    is_anti: bool   # True for antiparticles of fermions
    mass_key: str = ""
    width_key: str = ""


def _fermion_pair(name, anti, colour, charge, t3, mass_key="", width_key=""):
    return [Particle(name, anti, 1, colour, charge, t3, False, mass_key, width_key),
            Particle(anti, name, 1, -colour if colour != 1 else 1, -charge, -t3, True, mass_key, width_key)]


PARTICLES = {}
for _p in (_fermion_pair("e-", "e+", 1, -1.0, -0.5) + _fermion_pair("mu-", "mu+", 1, -1.0, -0.5)
           + _fermion_pair("ta-", "ta+", 1, -1.0, -0.5, "mta")
           + _fermion_pair("u", "u~", 3, 2.0 / 3.0, 0.5) + _fermion_pair("t", "t~", 3, 2.0 / 3.0, 0.5, "mt", "wt")
           + [Particle("g", "g", 2, 8, 0.0, 0.0, False), Particle("a", "a", 2, 1, 0.0, 0.0, False),
              Particle("z", "z", 2, 1, 0.0, 0.0, False, "mz", "wz")]):
    PARTICLES[_p.name] = _p


@dataclass(frozen=True)
class Params:
    mt: float = 173.0
    wt: float = 1.4915
    mz: float = 91.1876
    wz: float = 2.4414
    mta: float = 1.777
    alpha_em: float = 1.0 / 132.507
    gf: float = 1.16639e-5

    def mass(self, p):
        return getattr(self, p.mass_key) if p.mass_key else 0.0

    def width(self, p):
        return getattr(self, p.width_key) if p.width_key else 0.0

    @property
    def ee(self):
        return math.sqrt(4.0 * math.pi * self.alpha_em)

    @property
    def mw(self):
        mz2 = self.mz ** 2
        return math.sqrt(mz2 / 2.0 + math.sqrt(mz2 ** 2 / 4.0 - math.pi * self.alpha_em * mz2
                                               / (math.sqrt(2.0) * self.gf)))

    @property
    def sw2(self):
        return 1.0 - (self.mw / self.mz) ** 2

    def z_couplings(self, p):
        """(gL, gR) of the Z vertex -i gamma^mu (gL P_L + gR P_R) for fermion p (particle)."""
        sw = math.sqrt(self.sw2)
        cw = math.sqrt(1.0 - self.sw2)
        e = self.ee
        return (e * (p.t3 - p.charge * self.sw2) / (sw * cw), -e * p.charge * self.sw2 / (sw * cw))
