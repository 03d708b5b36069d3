"""CPU checks of the float64 MLP reference itself (no GPU): finite differences and bf16 rounding."""
import numpy as np

from oracle import mlp


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.1415926, 0.0])
    r = mlp.bf16(x)
    assert r[0] == 1.0 and r[4] == 0.0
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8 + 1e-300)
    assert mlp.bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7          # exactly representable
    assert mlp.bf16(1.0 + 2 ** -9) == 1.0                     # tie to even


def test_gradient_matches_finite_differences_without_rounding(monkeypatch):
    # with rounding disabled the analytic gradient must match central differences of the loss
    monkeypatch.setattr(mlp, "bf16", lambda x: np.asarray(x, dtype=np.float64))
    rng = np.random.default_rng(0)
    n = sum(256 * k + 256 for k in (32, 256, 256, 256)) + 257
    p = rng.normal(scale=0.05, size=n)
    x = rng.normal(size=(7, 24))
    t = rng.normal(size=7)
    loss, g = mlp.gradients(p, x, t)
    for idx in rng.choice(n, 40, replace=False):
        if 24 <= idx % 32 < 32 and idx < 256 * 32:
            continue
        e = np.zeros(n)
        e[idx] = 1e-6
        fd = (mlp.gradients(p + e, x, t)[0] - mlp.gradients(p - e, x, t)[0]) / 2e-6
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), idx
