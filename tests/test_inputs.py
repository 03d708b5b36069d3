"""Seeded input generators: Philox known answers, RAMBO properties, determinism."""
import math
import os

import numpy as np
import pytest

from phasespace import philox4x32_10, rambo, make_inputs, WORKLOADS, uniform01
from phasespace.rambo import rambo_massless_weight

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not l.startswith("#")]
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox4x32_10(np.array(v[:4], np.uint32), np.array(v[4:6], np.uint32))
        assert [int(x) for x in out] == v[6:10]


@pytest.mark.parametrize("masses", [[0.0, 0.0, 0.0, 0.0], [173.0, 173.0, 0.0, 0.0, 0.0]])
def test_rambo_conservation_and_shell(masses):
    p, w = rambo(20000, 1500.0, masses, seed=3)
    tot = p.sum(axis=1)
    # to rounding level (the repair step), including the nearly collinear events whose boost
    # loses digits
    assert np.abs(tot[:, 0] - 1500.0).max() < 1e-14 * 1500.0
    assert np.abs(tot[:, 1:]).max() < 1e-14 * 1500.0
    m2 = p[..., 0] ** 2 - (p[..., 1:] ** 2).sum(-1)
    assert (np.abs(m2 - np.asarray(masses) ** 2) / p[..., 0] ** 2).max() < 1e-14
    assert np.all(w > 0)


def test_rambo_massless_weight_constant():
    p, w = rambo(100, 1000.0, [0.0] * 3, seed=1)
    assert np.all(w == w[0])
    # two-body massless phase space volume is 1/(8 pi)
    assert math.isclose(rambo_massless_weight(2, 91.0), 1.0 / (8.0 * math.pi), rel_tol=1e-14)


def test_rambo_isotropic_two_body():
    p, _ = rambo(200000, 100.0, [0.0, 0.0], seed=5)
    cth = p[:, 0, 3] / p[:, 0, 0]
    hist, _ = np.histogram(cth, bins=10, range=(-1, 1))
    expected = len(cth) / 10
    chi2 = ((hist - expected) ** 2 / expected).sum()
    assert chi2 < 40.0


def test_inputs_independent_of_batching():
    wl = WORKLOADS["ggttgg"]
    a = make_inputs(wl, 64)
    b = make_inputs(wl, 32, first=32)
    for x, y in zip(a, b):
        assert np.array_equal(x[32:], y)
    r = uniform01(9, 1, 100000)
    assert r.min() >= 0.0 and r.max() < 1.0 and abs(r.mean() - 0.5) < 0.01
