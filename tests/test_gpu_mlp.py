"""GPU MLP kernels (tcgen05 bf16 GEMMs + SIMT) against the float64 CPU reference."""
import ctypes

import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


def _net(seed=3):
    import paper_2503_21935_gb300 as pkg
    return pkg.Mlp(seed=seed)


@pytest.mark.parametrize("n", [300, 2112, 4096])
def test_gradients_match_cpu_reference(n):
    """300 rows: one batch chunk per contraction slice; 2112: slices past the last chunk are empty
    (they must contribute zero); 4096: two chunks per slice."""
    import torch
    net = _net()
    rng = np.random.default_rng(1)
    x = rng.normal(size=(n, 24)).astype(np.float32)
    t = rng.normal(size=n).astype(np.float32)
    loss, g = net.gradients(x, t)
    p = net.get_params().astype(np.float64)
    rloss, rg = ref.gradients(p, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - rloss) <= 1e-4 * abs(rloss)
    # per parameter block: relative L2 error well below one bfloat16 ulp (3.9e-3)
    o = 0
    for l in range(ref.DEPTH):
        kin = ref.K0 if l == 0 else ref.WIDTH
        for size in (ref.WIDTH * kin, ref.WIDTH):
            a, b = g[o:o + size], rg[o:o + size]
            assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b) + 1e-12, (l, size)
            o += size
    a, b = g[o:], rg[o:]
    assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b)


def test_forward_matches_cpu_reference_many_rows():
    net = _net(seed=5)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(70000, 24)).astype(np.float32)      # two inference chunks, ragged tail
    y = net.forward(x)
    ry, _, _ = ref.forward(net.get_params().astype(np.float64), x.astype(np.float64))
    d = np.abs(y - ry) / (np.abs(ry).max() + 1.0)
    # float32 vs float64 accumulation (~1e-7 relative) flips a bfloat16 rounding of a hidden
    # activation (one ulp = 0.4%) with probability ~1e-7/4e-3 per rounding, ~1000 roundings a
    # row: a few percent of the rows move by up to a fraction of a percent, the rest agree
    assert np.median(d) < 1e-6 and np.quantile(d, 0.9) < 1e-5 and d.max() < 2e-2


def test_adam_step_matches_cpu():
    """One train step: the parameters move exactly as float32 Adam on the reference gradient."""
    net = _net(seed=7)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(512, 24)).astype(np.float32)
    t = rng.normal(size=512).astype(np.float32)
    p0 = net.get_params().astype(np.float64)
    _, g = net.gradients(x, t)
    net.train_step(x, t, lr=1e-3)
    p1 = net.get_params().astype(np.float64)
    m = 0.1 * g
    v = 0.001 * g * g
    step = -1e-3 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    assert np.abs((p1 - p0) - step).max() <= 1e-6


def test_training_fits_smooth_function():
    """Adam on a smooth 24-dimensional target: the loss must fall by a large factor."""
    net = _net(seed=11)
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, size=(32768, 24)).astype(np.float32)
    a = rng.normal(size=24)
    t = (np.sin(x @ a / 3.0) + 0.5 * (x[:, 0] * x[:, 1])).astype(np.float32)
    t = (t - t.mean()) / t.std()
    first = net.gradients(x[:4096], t[:4096])[0]
    for step in range(400):
        idx = rng.choice(len(x), 1024, replace=False)
        net.train_step(x[idx], t[idx], lr=1e-3)
    last = net.gradients(x[:4096], t[:4096])[0]
    assert last < 0.1 * first, (first, last)


def test_inference_from_momenta_and_across_passes():
    """The fused inference path: from float64 momenta it equals the float32-feature path bit for bit
    (both round momenta / scale to float32, then to bf16), and rows of a second pass (beyond 2^22
    rows) equal the same rows evaluated on their own (every row's result is independent of the
    tiling)."""
    import torch
    net = _net(seed=13)
    rng = np.random.default_rng(6)
    n = (1 << 22) + 300
    mom = torch.from_numpy(rng.normal(scale=500.0, size=(n, 6, 4))).cuda()
    scale = 750.0
    y_mom = net.forward_momenta(mom, scale)
    x = (mom.reshape(n, 24) / scale).to(torch.float32)
    y_x = net.forward(x)
    torch.cuda.synchronize()
    assert torch.equal(y_mom, y_x)
    tail = net.forward(x[(1 << 22) - 100:].contiguous())
    assert torch.equal(tail, y_x[(1 << 22) - 100:])
    assert torch.isfinite(y_x).all()


def test_sampled_training_step_draws_the_documented_rows():
    """mgx_mlp_train_step_sampled is mgx_mlp_train_step on the rows its header documents: batch row
    r takes example floor(w0 ntotal / 2^32), w0 the first word of Philox-4x32-10 with counter
    (r, step, 0x4D4C5053, 0) under the seed (computed here by the host generator), bit for bit."""
    import torch
    from phasespace.philox import philox4x32_10
    rng = np.random.default_rng(4)
    ntotal, batch, seed, step = 5000, 1024, 0x123456789ABC, 7
    x = rng.normal(size=(ntotal, 24)).astype(np.float32)
    t = rng.normal(size=ntotal).astype(np.float32)
    r = np.arange(batch, dtype=np.uint64)
    ctr = np.stack([r & np.uint64(0xFFFFFFFF), np.full(batch, step, np.uint64), np.full(batch, 0x4D4C5053, np.uint64),
                    r >> np.uint64(32)], axis=-1).astype(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    w0 = philox4x32_10(ctr, key)[:, 0].astype(np.uint64)
    idx = ((w0 * np.uint64(ntotal)) >> np.uint64(32)).astype(np.int64)
    assert len(np.unique(idx)) > 0.8 * batch
    a, b = _net(seed=5), _net(seed=5)
    a.train_step_sampled(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), batch, seed, step, lr=1e-3)
    b.train_step(x[idx], t[idx], lr=1e-3)
    torch.cuda.synchronize()
    assert np.array_equal(a.get_params(), b.get_params())
