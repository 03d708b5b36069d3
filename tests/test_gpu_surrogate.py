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


def test_two_rank_unweighting_equals_one_rank():
    """Data-parallel unweighting, two ranks emulated in one process (their kernels run one after the
    other; no kernel waits on another): each 'rank' calibrates on its own event range, the maxima come
    from the union of the ranks' calibration weights (what the gather collective hands every rank),
    and each rank unweights its own range.  The union of the ranks' unweighted events, with their
    weights, must be exactly the one-rank sample over all events; so must the combined (max w, sum w,
    N) of the batches."""
    import torch
    import paper_2503_21935_gb300 as pkg
    from paper_2503_21935_gb300 import dist as D
    from paper_2503_21935_gb300.surrogate import Unweighter
    U = Unweighter("g g > t t~ g g", 1500.0, [173.0, 173.0, 0.0, 0.0], cut_particles=[4, 5], seed=5)
    U.proc.set_kernel(pkg.MGX_KERNEL_THREAD)       # one kernel for every batch size: bitwise comparable
    U.train(1 << 15, steps=200, batch=2048, lr=2e-3)
    n = 1 << 16
    w_all, s_all = U.calibration_sample(2 * n, seed=202, first=0)
    one = U.set_maxima(w_all, s_all)
    parts = [U.calibration_sample(n, seed=202, first=r * n) for r in range(2)]
    two = U.set_maxima(torch.cat([p[0] for p in parts]), torch.cat([p[1] for p in parts]))
    assert one == two
    for fn, seed in ((U.plain, 303), (U.two_stage, 404)):
        single = fn(2 * n, seed=seed, first=0)
        ranks = [fn(n, seed=seed, first=r * n) for r in range(2)]
        idx = torch.cat([r["index"] for r in ranks])
        assert torch.equal(idx, single["index"]), fn.__name__
        assert torch.equal(torch.cat([r["weight"] for r in ranks]), single["weight"])
        assert torch.equal(torch.cat([r["momenta"] for r in ranks]), single["momenta"])
        assert single["index"].numel() > 20
        if fn is U.plain:
            assert D.combine_weight_stats([(r["max_w"], r["sum_w"], r["n_events"]) for r in ranks])[0] == single["max_w"]
            sw = D.combine_weight_stats([(r["max_w"], r["sum_w"], r["n_events"]) for r in ranks])[1]
            assert abs(sw / single["sum_w"] - 1) < 1e-12


def test_data_parallel_training_step_equals_full_batch():
    """Two replicas' gradients of their half batches, averaged as the all-reduce does, then one Adam
    step: the parameters equal those of one replica's train step on the whole batch (float32
    accumulation order differs, so within float32 rounding of the gradient)."""
    import torch
    import paper_2503_21935_gb300 as pkg
    from paper_2503_21935_gb300 import dist as D
    rng = np.random.default_rng(8)
    x = rng.normal(size=(1024, 24)).astype(np.float32)
    t = rng.normal(size=1024).astype(np.float32)
    a, b = pkg.Mlp(seed=9), pkg.Mlp(seed=9)
    p0 = a.get_params()
    assert np.array_equal(p0, b.get_params())
    a.train_step(x, t, lr=1e-3)
    g = D.combine_gradients([b.device_gradients(x[:512], t[:512]), b.device_gradients(x[512:], t[512:])], [512, 512])
    b.adam_step(g, lr=1e-3)
    torch.cuda.synchronize()
    pa, pb = a.get_params().astype(np.float64), b.get_params().astype(np.float64)
    step = np.abs(pa - p0)
    # Adam's first step moves each parameter by about lr; a float32-rounding difference of the
    # gradient changes that only where the gradient is tiny against its own rounding
    assert np.median(np.abs(pa - pb)) <= 1e-9 and np.quantile(np.abs(pa - pb), 0.99) <= 2e-5
    assert np.median(step) > 5e-4


def test_tiny_batches_and_empty_stages():
    """Batches of 1 to 64 events, and maxima so large that a stage keeps nothing: every call of the
    chain (indexed RAMBO, cuts, exact |M|^2, accept, compaction, outputs) runs on the empty case and
    the outputs stay consistent."""
    from paper_2503_21935_gb300.surrogate import Unweighter
    U = Unweighter("g g > t t~ g g", 1500.0, [173.0, 173.0, 0.0, 0.0], cut_particles=[4, 5], seed=5)
    U.train(1 << 12, steps=20, batch=512, lr=2e-3)
    U.calibrate(1 << 12)
    for n in (1, 8, 64):
        for fn in (U.plain, U.two_stage):
            r = fn(n, seed=77, first=1000)
            m = r["weight"].shape[0]
            assert r["index"].shape[0] == m and r["momenta"].shape == (m, 6, 4)
            if m:
                assert bool((r["weight"] >= 1).all())
                assert bool((r["index"] >= 1000).all()) and bool((r["index"] < 1000 + n).all())
    U.w_max = U.s_max = U.r_max = 1e300
    for fn in (U.plain, U.two_stage):
        r = fn(256, seed=78)
        assert r["weight"].shape[0] == 0 and r["momenta"].shape == (0, 6, 4)
    assert U.two_stage(256, seed=78)["stage1"] == 0
