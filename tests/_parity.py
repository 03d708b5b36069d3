"""Shared parity bar of the GPU tests: per-event relative deviation from the float64 oracle at most
1e-12, except for events whose condition estimate says no float64 evaluation order can promise
that (cancellation-limited events: reported, held to 100 x 1e-16 x kappa, and required to be rare)."""
import numpy as np

from oracle.matrix_element import get as oracle_get, near_tie

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


def check_selection(got, ref, weights, r, rel=TOL, what="selection", max_frac=0.01):
    """Selected indices equal the oracle's on every event whose cumulative weights stay more than
    rel x total away from the random threshold (reading P7); the events inside that window are
    counted, printed, and required to be at most max_frac of the sample, or one event in a sample
    of fewer than 1/max_frac (with uniform random
    numbers their expected share is about (number of weights) x 2 rel), so the comparison cannot
    become vacuous.  Returns the tie mask."""
    tie = near_tie(weights, r, rel)
    print(f"{what}: {int(tie.sum())} of {tie.size} events inside the tie window {rel:g}")
    assert tie.sum() <= max(1, int(max_frac * tie.size)), \
        f"{what}: {int(tie.sum())} of {tie.size} events excluded as near-ties"
    bad = np.flatnonzero(np.asarray(got)[~tie] != np.asarray(ref)[~tie])
    assert bad.size == 0, f"{what}: {bad.size} events differ from the oracle, first {np.flatnonzero(~tie)[bad[:5]]}"
    return tie


def check_mode(proc, got, ref, rh, rc, bound, what):
    """A reduced-precision colour sum against the float64 oracle: me and every |M_h|^2 (relative to
    the event total) within `bound`, and so every cumulative helicity weight, which makes `bound` a
    sound tie window for the helicity selection; colour weights come from the float64 jamps in
    every mode and meet the float64 bar, so the colour selection uses the float64 window."""
    assert np.all(np.isfinite(got["me"])), f"{what}: non-finite me"
    rel = np.abs(got["me"] / ref["me"] - 1.0)
    assert rel.max() <= bound, f"{what}: me max rel {rel.max():.3e}"
    good = proc.good_helicities
    tot = ref["mh"].sum(axis=1, keepdims=True)
    dmh = got["mh"] - ref["mh"][:, good]
    assert (np.abs(dmh) / tot).max() <= bound, f"{what}: |M_h|^2 max dev {(np.abs(dmh) / tot).max():.3e}"
    assert (np.abs(np.cumsum(dmh, axis=1)) / tot).max() <= bound
    check_selection(got["selhel"], ref["selhel"], ref["mh"], rh, bound, f"{what} selhel")
    return rel.max()
