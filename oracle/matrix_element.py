"""|M|^2, per-helicity weights, colour-flow amplitudes (jamps) and selection.

Normalisation (MadGraph convention): me = 1/(Nspin_in * Ncol_in * S) *
sum_h sum_colours |M|^2, with Nspin_in = 4 (two helicities per incoming
parton), Ncol_in the product of the incoming colour dimensions, and S the
product of n! over identical final-state particles.

Colour: J_s(h) = sum_t k_ts A_t(h), where k_t are the coordinates of the term's
colour tensor in the flow basis b_s (solved by least squares on sampled explicit
colour configurations and verified on an independent sample); then
|M_h|^2 = Re(J^dagger C J) with the exact rational colour matrix C.  For small
processes the explicit colour sum sum_colours |sum_t A_t c_t|^2 is also given.

Selection (the paper selects one helicity and one colour flow per event for the
event record; the rule is a reading, since the paper gives none):
  helicity  = smallest canonical index k with cumsum_k(|M_h|^2) > r_hel * sum
  colour    = smallest flow index s with cumsum_s(w) > r_col * sum(w),
              w_s = sum_h |J_s(h)|^2.
"""
import math
from collections import Counter
from functools import lru_cache

import numpy as np

from .amplitudes import Process
from .colour import flow_permutations, basis_at, colour_matrix, rationalise
from .model import PARTICLES, Params


class MatrixElement:
    def __init__(self, proc, params=None, seed=12345):
        self.p = Process(proc, params)
        P = self.p
        self.perms = flow_permutations(P.gluon_legs) if P.row_leg is not None else [()]
        self.ncol = len(self.perms)
        self._decompose(seed)

    # --------------------------------------------------------------- colour
    def _decompose(self, seed):
        P = self.p
        nterm = len(P.terms)
        if P.row_leg is None:
            self.k = np.ones((nterm, 1), dtype=complex)
            self.C = np.ones((1, 1))
            self.C_exact = [[1]]
            return
        rng = np.random.default_rng(seed)
        dims = np.array([8 if leg in P.gluon_legs else 3 for leg in P.coloured_legs])
        # Most explicit colour configurations give zero (the Gell-Mann matrices are
        # sparse); keep drawing until the sampled basis rows have full column rank.
        R = 16 * self.ncol
        for _ in range(8):
            cfg1 = (rng.random((R, len(dims))) * dims).astype(np.int64)
            B1 = basis_at(cfg1, P.coloured_legs, P.gluon_legs, P.row_leg, P.col_leg, self.perms)
            if np.linalg.matrix_rank(B1) == self.ncol:
                break
            R *= 2
        else:
            raise RuntimeError("sampled colour configurations do not span the flow basis")
        cfg2 = (rng.random((R, len(dims))) * dims).astype(np.int64)
        B2 = basis_at(cfg2, P.coloured_legs, P.gluon_legs, P.row_leg, P.col_leg, self.perms)
        c1 = np.stack([P.term_colour(t, cfg1) for t in P.terms], axis=1)
        c2 = np.stack([P.term_colour(t, cfg2) for t in P.terms], axis=1)
        k, *_ = np.linalg.lstsq(B1, c1, rcond=None)
        resid = np.abs(B2 @ k - c2).max()
        if resid > 1e-10:
            raise RuntimeError(f"colour tensors are not in the flow basis span (residual {resid})")
        self.k = k.T.copy()                       # [nterm, ncol]
        Cf = colour_matrix(P.gluon_legs, self.perms, P.coloured_legs, P.row_leg, P.col_leg)
        self.C_exact = rationalise(Cf)
        self.C = np.array([[float(x) for x in row] for row in self.C_exact])

    # --------------------------------------------------------------- normalisation
    def average_factor(self):
        P = self.p
        ncol_in = 1
        for name in P.incoming:
            ncol_in *= abs(PARTICLES[name].colour)
        ident = 1
        for name, cnt in Counter(P.outgoing).items():
            ident *= math.factorial(cnt)
        return 1.0 / (4.0 * ncol_in * ident)

    # --------------------------------------------------------------- evaluation
    def jamps(self, p, alpha_s, gauge_leg=None):
        """J[nevt, nhel, ncol] (all 2^npar helicities, canonical order)."""
        A = self.p.term_amplitudes(p, alpha_s, gauge_leg)   # [nterm, nevt, nhel]
        return np.einsum("tes,tc->esc", A, self.k)

    def helicity_weights(self, J):
        """|M_h|^2 = Re(J^dagger C J): [nevt, nhel] (colour-summed, not averaged)."""
        return np.einsum("esc,cd,esd->es", J.conj(), self.C, J).real

    def evaluate(self, p, alpha_s, rnd_hel=None, rnd_col=None):
        """Dict with me, per-helicity weights, jamps, colour weights and selections."""
        J = self.jamps(p, alpha_s)
        Mh = self.helicity_weights(J)
        me = Mh.sum(axis=1) * self.average_factor()
        out = dict(me=me, mh=Mh, jamps=J, colw=(np.abs(J) ** 2).sum(axis=1))
        if rnd_hel is not None:
            out["selhel"] = select(Mh, rnd_hel)
        if rnd_col is not None:
            out["selcol"] = select(out["colw"], rnd_col)
        return out

    def condition(self, p, alpha_s, trials=4, seed=0):
        """Relative condition estimate of me per event, used to tell cancellation-limited events
        from real deviations in the float64 parity comparison: the larger of
          kappa_terms = sum_h sum_ij |C_ij| a_i(h) a_j(h) / sum_h |M_h|^2, a_i(h) = sum_t |k_ti A_t(h)|
            (relative perturbations eps of every diagram term move me by at most ~2 eps kappa_terms),
          kappa_in = max over `trials` random one-ulp sign perturbations of every momentum component
            of |me' / me - 1| / 2^-52 (the sensitivity to the rounding of the summed momenta that
            propagator denominators and vertices see, which kappa_terms does not measure).
        An event with kappa * 1e-16 > 1e-12 cannot be expected to agree to 1e-12 between two
        float64 evaluation orders: it is cancellation-limited."""
        A = self.p.term_amplitudes(p, alpha_s)               # [nterm, nevt, nhel]
        a = np.einsum("tes,tc->esc", np.abs(A), np.abs(self.k))
        bound = np.einsum("esc,cd,esd->e", a, np.abs(self.C), a)
        J = np.einsum("tes,tc->esc", A, self.k)
        me = self.helicity_weights(J).sum(axis=1)
        kappa = bound / me
        rng = np.random.default_rng(seed)
        ulp = 2.0 ** -52
        for _ in range(trials):
            q = p * (1.0 + ulp * rng.choice([-1.0, 1.0], size=p.shape))
            me2 = self.helicity_weights(self.jamps(q, alpha_s)).sum(axis=1)
            kappa = np.maximum(kappa, np.abs(me2 / me - 1.0) / ulp)
        return kappa

    def me_bruteforce_colour(self, p, alpha_s):
        """Explicit sum over every colour configuration (small processes only)."""
        P = self.p
        A = P.term_amplitudes(p, alpha_s)               # [nterm, nevt, nhel]
        if P.row_leg is None and not P.coloured_legs:
            M = A.sum(axis=0)
            return (np.abs(M) ** 2).sum(axis=1) * self.average_factor()
        c = np.stack([P.term_colour(t).reshape(-1) for t in P.terms], axis=0)   # [nterm, ncfg]
        M = np.einsum("tes,tc->esc", A, c)
        return (np.abs(M) ** 2).sum(axis=(1, 2)) * self.average_factor()

    def helicity_filter(self, p, alpha_s):
        """Canonical indices h with |M_h|^2 != 0 on any of the given events."""
        Mh = self.helicity_weights(self.jamps(p, alpha_s))
        return [h for h in range(Mh.shape[1]) if np.any(Mh[:, h] != 0.0)]


def select(weights, r):
    """Smallest index k with cumsum_k(weights) > r * total (cumsum in index order)."""
    w = np.asarray(weights, dtype=np.float64)
    cs = np.cumsum(w, axis=1)
    tot = cs[:, -1]
    target = np.asarray(r) * tot
    k = (cs <= target[:, None]).sum(axis=1)
    return np.minimum(k, w.shape[1] - 1).astype(np.int32)


def near_tie(weights, r, rel=1e-12):
    """True where some cumulative sum lies within rel*total of r*total."""
    w = np.asarray(weights, dtype=np.float64)
    cs = np.cumsum(w, axis=1)
    tot = cs[:, -1]
    return (np.abs(cs - (np.asarray(r) * tot)[:, None]) <= rel * np.abs(tot)[:, None]).any(axis=1)


@lru_cache(maxsize=None)
def get(proc):
    return MatrixElement(proc)
