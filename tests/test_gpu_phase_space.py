"""Device Philox / RAMBO / cuts against the host generators (which the oracle-side tests pin)."""
import numpy as np
import pytest

from phasespace import rambo, uniform01, incoming_beams

pytestmark = pytest.mark.gpu


def test_uniforms_bit_exact():
    import paper_2503_21935_gb300 as pkg
    for seed, sid, first in [(3, 1, 0), (12345678901, 2, 1000)]:
        d = pkg.uniforms(5000, seed, sid, first=first).cpu().numpy()
        h = uniform01(seed, sid, first + 5000)[first:]
        assert np.array_equal(d, h)


@pytest.mark.parametrize("masses", [[0.0, 0.0], [173.0, 173.0, 0.0, 0.0], [173.0, 173.0, 0.0, 0.0, 0.0]])
def test_rambo_matches_host(masses):
    import paper_2503_21935_gb300 as pkg
    n, sqrts, seed = 4096, 1500.0, 17
    mom, wt = pkg.rambo(n, sqrts, masses, seed, first=100)
    po, hw = rambo(n + 100, sqrts, masses, seed)
    hmom = np.concatenate([incoming_beams(n + 100, sqrts), po], axis=1)[100:]
    d = mom.cpu().numpy()
    # CUDA and host libm (log, sin, cos) differ by ~1 ulp; RAMBO's boost of the random massless
    # momenta amplifies that by its condition number (Q0/M)^2 of the summed vector, so the bound
    # is per event: 1e-15 x cond (with a floor of 1e-13)
    r = np.asarray([0.0])
    dev = (np.abs(d - hmom) / sqrts).max(axis=(1, 2))
    from phasespace.philox import uniform_open01
    u = uniform_open01(seed, 0, n + 100, 4 * len(masses)).reshape(n + 100, len(masses), 4)[100:]
    c = 2 * u[..., 0] - 1
    s_ = np.sqrt(1 - c * c)
    f = 2 * np.pi * u[..., 1]
    q0 = -np.log(u[..., 2] * u[..., 3])
    Q = np.stack([q0.sum(1), (q0 * s_ * np.cos(f)).sum(1), (q0 * s_ * np.sin(f)).sum(1), (q0 * c).sum(1)], 1)
    cond = Q[:, 0] ** 2 / (Q[:, 0] ** 2 - (Q[:, 1:] ** 2).sum(1))
    assert np.all(dev <= np.maximum(1e-13, 1e-15 * cond))
    assert np.abs(wt.cpu().numpy() / hw[100:] - 1).max() < 1e-9
    # the device momenta themselves are physical: after the repair step, conservation and mass
    # shells hold to rounding whatever the boost's conditioning
    assert np.abs(d[:, 2:].sum(1) - d[:, :2].sum(1)).max() < 1e-14 * sqrts
    m2 = d[:, 2:, 0] ** 2 - (d[:, 2:, 1:] ** 2).sum(-1)
    rel = np.abs(m2 - np.asarray(masses) ** 2) / d[:, 2:, 0] ** 2
    assert rel.max() <= 1e-14


def test_cuts_match_numpy():
    import torch
    import paper_2503_21935_gb300 as pkg
    n = 20000
    mom, _ = pkg.rambo(n, 1500.0, [173.0, 173.0, 0.0, 0.0], 5)
    got = pkg.cuts(mom, [4, 5], 20.0, 5.0, 0.4).cpu().numpy().astype(bool)
    p = mom.cpu().numpy()
    g = p[:, [4, 5]]
    pt = np.hypot(g[..., 1], g[..., 2])
    pp = np.sqrt(pt ** 2 + g[..., 3] ** 2)
    eta = 0.5 * np.log((pp + g[..., 3]) / (pp - g[..., 3]))
    phi = np.arctan2(g[..., 2], g[..., 1])
    dphi = np.abs(phi[:, 0] - phi[:, 1])
    dphi = np.where(dphi > np.pi, 2 * np.pi - dphi, dphi)
    dr = np.sqrt((eta[:, 0] - eta[:, 1]) ** 2 + dphi ** 2)
    ref = (pt > 20).all(axis=1) & (np.abs(eta) < 5).all(axis=1) & (dr > 0.4)
    assert np.array_equal(got, ref)
    assert 0.3 < ref.mean() < 0.99


@pytest.mark.parametrize("masses", [[0.0, 0.0, 0.0], [173.0, 173.0, 0.0, 0.0]])
def test_rambo_indexed_and_float32(masses):
    """Float64 regeneration of selected events equals the corresponding rows bit for bit; the
    float32 proposals are the same events to float32 accuracy (momenta relative to sqrt(s), weights)."""
    import torch
    import paper_2503_21935_gb300 as pkg
    n, sqrts, seed, first = 1 << 16, 1500.0, 23, 77
    mom, wt = pkg.rambo(n, sqrts, masses, seed, first=first)
    idx = torch.tensor(np.sort(np.random.default_rng(0).choice(n, 999, replace=False)).astype(np.int32), device="cuda")
    mi, wi = pkg.rambo_indexed(idx, first, sqrts, masses, seed)
    assert torch.equal(mi, mom[idx.long()]) and torch.equal(wi, wt[idx.long()])
    m32, w32 = pkg.rambo_f32(n, sqrts, masses, seed, first=first)
    dev = ((m32.double() - mom).abs() / sqrts).amax(dim=(1, 2))
    assert dev.median().item() < 1e-6 and dev.max().item() < 1e-3
    assert ((w32.double() / wt - 1).abs().median()).item() < 1e-5


def test_float32_cuts_with_margin_contain_float64_cuts():
    """Every event the float64 cuts accept is accepted by the float32 cuts with the proposal margin
    (so stage-1 proposals cover the exact support); the widened band is a small fraction."""
    import torch
    import paper_2503_21935_gb300 as pkg
    from paper_2503_21935_gb300.surrogate import PROPOSAL_CUT_MARGIN
    n, sqrts, seed = 1 << 21, 1500.0, 31
    masses = [173.0, 173.0, 0.0, 0.0]
    mom, _ = pkg.rambo(n, sqrts, masses, seed)
    m32, _ = pkg.rambo_f32(n, sqrts, masses, seed)
    exact = pkg.cuts(mom, [4, 5], 20.0, 5.0, 0.4).bool()
    wide = pkg.cuts_f32(m32, [4, 5], 20.0, 5.0, 0.4, PROPOSAL_CUT_MARGIN).bool()
    assert not (exact & ~wide).any()
    band = (wide & ~exact).float().mean().item()
    assert band < 0.02, band
    same = pkg.cuts_f32(m32, [4, 5], 20.0, 5.0, 0.4, 0.0).bool()
    assert (same != exact).float().mean().item() < 1e-4
