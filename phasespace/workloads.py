"""Synthetic workload recipes (flat RAMBO phase space at fixed partonic sqrt(s)).

The paper measures on madevent events (multichannel phase space with PDFs) that
are not available here; seeded flat phase space at fixed partonic energy with the
same process, multiplicity and batch sizes stands in for them.
"""
from dataclasses import dataclass
import numpy as np

from .philox import uniform01
from .rambo import rambo, incoming_beams

# Final-state masses used for phase-space generation (GeV).
_MASS = {"t": 173.0, "t~": 173.0, "ta+": 1.777, "ta-": 1.777}


@dataclass(frozen=True)
class Workload:
    name: str
    process: str
    sqrts: float
    nevt: int
    seed_momenta: int
    seed_random: int
    alpha_s: float = 0.118

    @property
    def final_state(self):
        return self.process.split(">")[1].split()

    def final_masses(self):
        return [_MASS.get(p, 0.0) for p in self.final_state]


WORKLOADS = {
    "eemumu": Workload("eemumu", "e+ e- > mu+ mu-", 500.0, 8192, 0, 1),
    "ggtt": Workload("ggtt", "g g > t t~", 1500.0, 1 << 22, 6, 7),
    "ggttg": Workload("ggttg", "g g > t t~ g", 1500.0, 1 << 20, 8, 9),
    "ggttgg": Workload("ggttgg", "g g > t t~ g g", 1500.0, 1 << 20, 2, 3),
    "ggttggg": Workload("ggttggg", "g g > t t~ g g g", 1500.0, 1 << 18, 4, 5),
    "gu_tataggu": Workload("gu_tataggu", "g u~ > ta+ ta- g g u~", 1500.0, 1 << 16, 10, 11),
}


def make_inputs(wl, nevt=None, first=0, alpha_s_range=None):
    """Momenta [nevt, npar, 4], alpha_s [nevt], r_hel [nevt], r_col [nevt] (float64, host).

    Events first..first+nevt-1 of the workload's seeded stream.  Random numbers
    are counter-based, so any sub-range reproduces the same events.  alpha_s is
    the workload's constant unless alpha_s_range = (lo, hi) is given: then each
    event draws its own value uniformly in [lo, hi) (Philox stream 3 of the
    workload's random seed), as a run with a dynamical scale would pass.
    """
    n = wl.nevt if nevt is None else nevt
    masses = wl.final_masses()
    tot = first + n
    pout, _ = rambo(tot, wl.sqrts, masses, wl.seed_momenta)
    pin = incoming_beams(tot, wl.sqrts)
    mom = np.concatenate([pin, pout], axis=1)[first:]
    if alpha_s_range is None:
        alphas = np.full(n, wl.alpha_s)
    else:
        lo, hi = alpha_s_range
        alphas = lo + (hi - lo) * uniform01(wl.seed_random, 3, tot)[first:]
    rhel = uniform01(wl.seed_random, 1, tot)[first:]
    rcol = uniform01(wl.seed_random, 2, tot)[first:]
    return np.ascontiguousarray(mom), alphas, rhel, rcol
