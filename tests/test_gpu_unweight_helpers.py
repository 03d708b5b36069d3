"""The unweighting's helper kernels through the C ABI against numpy: training targets, moments,
standardisation, the unweighted events' weights and indices, and the calibration maxima."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lib():
    import paper_2503_21935_gb300 as pkg
    return pkg.lib(), pkg._ptr


def pkg_len():
    import paper_2503_21935_gb300 as pkg
    return pkg.MGX_MOMENTS_LEN


def _ok(rc):
    import paper_2503_21935_gb300 as pkg
    assert rc == pkg.MGX_OK, pkg.status_string(rc)


def test_targets_moments_standardisation():
    import torch
    lib, ptr = _lib()
    rng = np.random.default_rng(3)
    n = 100003
    me = np.exp(3.0 * rng.normal(size=n))
    me[::7] = 0.0
    me[5], me[11], me[13] = np.inf, -1.0, np.nan
    ok = (rng.random(n) < 0.8).astype(np.uint8)
    d = lambda a: torch.from_numpy(a).cuda()
    dme, dok = d(me), d(ok)
    logme = torch.empty(n, dtype=torch.float64, device="cuda")
    keep = torch.empty(n, dtype=torch.uint8, device="cuda")
    _ok(lib.mgx_log_targets(n, ptr(dme), ptr(dok), ptr(logme), ptr(keep), None))
    torch.cuda.synchronize()
    k_ref = (ok == 1) & (me > 0) & np.isfinite(me)
    assert np.array_equal(keep.cpu().numpy().astype(bool), k_ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        l_ref = np.where(k_ref, np.log(me), 0.0)
    assert np.max(np.abs(logme.cpu().numpy() - l_ref)) <= 1e-14
    y = l_ref[k_ref]
    dy = d(y)
    sums = torch.empty(pkg_len(), dtype=torch.float64, device="cuda")
    _ok(lib.mgx_moments(y.size, ptr(dy), ptr(sums), None))
    s1, s2, mx = sums.cpu().numpy()[:3]
    import math
    assert abs(s1 - math.fsum(y)) <= 1e-12 * math.fsum(np.abs(y))
    assert abs(s2 - math.fsum(y * y)) <= 1e-12 * math.fsum(y * y)
    assert mx == y.max()
    again = torch.empty(pkg_len(), dtype=torch.float64, device="cuda")
    _ok(lib.mgx_moments(y.size, ptr(dy), ptr(again), None))
    assert torch.equal(sums[:3], again[:3])            # fixed order: the same bits
    mean, sd = s1 / y.size, 1.7
    t = torch.empty(y.size, dtype=torch.float32, device="cuda")
    _ok(lib.mgx_standardize_f32(y.size, ptr(dy), mean, sd, ptr(t), None))
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy(), ((y - mean) / sd).astype(np.float32))
    empty = torch.empty(pkg_len(), dtype=torch.float64, device="cuda")
    _ok(lib.mgx_moments(0, None, ptr(empty), None))
    assert empty.cpu().numpy()[2] == -np.inf and empty.cpu().numpy()[0] == 0.0


def test_unweighted_out_both_stages():
    import torch
    lib, ptr = _lib()
    rng = np.random.default_rng(5)
    n1 = 50000
    idx1 = np.sort(rng.choice(n1, 20000, replace=False)).astype(np.int32)
    idx2 = np.sort(rng.choice(idx1.size, 7000, replace=False)).astype(np.int32)
    over1 = np.maximum(1.0, rng.exponential(size=n1) * 2)
    over2 = np.maximum(1.0, rng.exponential(size=idx1.size) * 2)
    d = lambda a: torch.from_numpy(a).cuda()
    first = 12345678901
    # device copies held in variables for as long as the kernel may read them (a temporary's block
    # returns to the caching allocator at once and the next copy may overwrite it)
    di2, di1, do1, do2 = d(idx2), d(idx1), d(over1), d(over2)
    for two in (True, False):
        m = idx2.size
        w = torch.empty(m, dtype=torch.float64, device="cuda")
        ix = torch.empty(m, dtype=torch.int64, device="cuda")
        _ok(lib.mgx_unweighted_out(m, ptr(di2), ptr(di1) if two else None, ptr(do1), ptr(do2) if two else None,
                                   first, ptr(w), ptr(ix), None))
        torch.cuda.synchronize()
        ev = idx1[idx2] if two else idx2
        w_ref = over1[ev] * over2[idx2] if two else over1[ev]
        assert np.array_equal(w.cpu().numpy(), w_ref)
        assert np.array_equal(ix.cpu().numpy(), first + ev.astype(np.int64))


@pytest.mark.parametrize("q", [0.999, 0.5, 1.0])
def test_unweighting_maxima_are_the_quantiles(q):
    import torch
    lib, ptr = _lib()
    rng = np.random.default_rng(7)
    n = 200001
    w = rng.exponential(size=n) * (rng.random(n) < 0.7)
    s = rng.exponential(size=n) * (rng.random(n) < 0.9)
    out = (ctypes.c_double * 3)()
    dw, ds = torch.from_numpy(w).cuda(), torch.from_numpy(s).cuda()
    _ok(lib.mgx_unweighting_maxima(n, ptr(dw), ptr(ds), q, ctypes.cast(out, ctypes.c_void_p), None))
    sel = (w > 0) & (s > 0)
    ref = [np.quantile(v, q) for v in (w[sel], s[sel], w[sel] / s[sel])]
    for got, want in zip(out, ref):
        assert abs(got - want) <= 1e-15 * abs(want), (q, got, want)
