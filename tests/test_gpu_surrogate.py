"""Surrogate two-stage unweighting: unbiased against the exact weighted distribution, and
fewer exact |M|^2 evaluations per unweighted event than plain hit-or-miss."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _observables(mom):
    pt_top = np.hypot(mom[:, 2, 1], mom[:, 2, 2])
    g = mom[:, 4] + mom[:, 5]
    m_gg = np.sqrt(np.maximum(g[:, 0] ** 2 - (g[:, 1:] ** 2).sum(-1), 0.0))
    return {"pt_top": pt_top, "m_gg": m_gg}


def _chi2(x_unw, w_unw, x_ref, w_ref, nbins=10):
    """chi^2 of the unweighted sample's histogram against the exact weighted distribution."""
    edges = np.quantile(x_ref, np.linspace(0, 1, nbins + 1))
    edges[0], edges[-1] = -np.inf, np.inf
    O, _ = np.histogram(x_unw, edges, weights=w_unw)
    O2, _ = np.histogram(x_unw, edges, weights=w_unw ** 2)
    R, _ = np.histogram(x_ref, edges, weights=w_ref)
    R2, _ = np.histogram(x_ref, edges, weights=w_ref ** 2)
    f = R / R.sum()
    E = f * O.sum()
    var = O2 + (O.sum() ** 2) * R2 / R.sum() ** 2
    return float(((O - E) ** 2 / var).sum()), nbins - 1


def test_two_stage_unweighting_unbiased_and_cheaper():
    from paper_2503_21935_gb300.surrogate import Unweighter
    U = Unweighter("g g > t t~ g g", 1500.0, [173.0, 173.0, 0.0, 0.0], cut_particles=[4, 5], seed=5)
    hist = U.train(1 << 18, steps=1500, batch=4096, lr=2e-3)
    assert hist[-1][1] < 0.5 * hist[0][1]
    U.calibrate(1 << 18)
    P = U.plain(1 << 21, seed=303)
    S = U.two_stage(1 << 21, seed=404)
    n_p, n_s = P["weight"].shape[0], S["weight"].shape[0]
    assert n_p > 100 and n_s > 100
    # exact ME evaluations per unweighted event: the surrogate must need fewer
    cost_p = P["exact_calls"] / P["weight"].sum().item()
    cost_s = S["exact_calls"] / S["weight"].sum().item()
    assert cost_s < cost_p, (cost_p, cost_s)
    ref_mom = P["all_momenta"].cpu().numpy()
    ref_w = P["all_weights"].cpu().numpy()
    obs_ref = _observables(ref_mom)
    for name, (mom, w) in {"plain": (P["momenta"], P["weight"]), "two-stage": (S["momenta"], S["weight"])}.items():
        obs = _observables(mom.cpu().numpy())
        for key in obs:
            chi2, ndf = _chi2(obs[key], w.cpu().numpy(), obs_ref[key], ref_w)
            assert chi2 < ndf + 5 * np.sqrt(2 * ndf), (name, key, chi2)
