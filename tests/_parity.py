"""Shared parity bar of the GPU tests: per-event relative deviation from the float64 oracle at most
1e-12, except for events whose condition estimate says no float64 evaluation order can promise
that (cancellation-limited events: reported, held to 100 x 1e-16 x kappa, and required to be rare)."""
import numpy as np

from oracle.matrix_element import get as oracle_get

TOL = 1e-12


def bounds(process, mom, a, rel):
    """Per-event bound on a relative deviation `rel` ([nevt] or [nevt, k]): TOL, except for events
    the oracle marks cancellation-limited (condition estimate kappa with kappa * 1e-16 > TOL),
    which are reported and held to 100 x 1e-16 x kappa instead.  Such events must stay rare."""
    bound = np.full(rel.shape[0], TOL)
    bad = np.flatnonzero(rel.reshape(rel.shape[0], -1).max(axis=1) > TOL)
    if bad.size:
        kappa = oracle_get(process).condition(mom[bad], a[bad])
        limited = kappa * 1e-16 > TOL
        for e, k in zip(bad, kappa):
            print(f"{process}: event {e} deviates {rel[e].max():.2e}, condition estimate {k:.3g}"
                  + (" (cancellation-limited)" if k * 1e-16 > TOL else ""))
        bound[bad[limited]] = 1e-14 * kappa[limited]
        assert limited.sum() <= max(1, rel.shape[0] // 50), "too many cancellation-limited events"
    return bound if rel.ndim == 1 else bound[:, None]
