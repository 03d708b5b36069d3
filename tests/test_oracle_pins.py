"""Pins of the float64 oracle against closed forms, exact colour algebra,
independent algorithms and symmetries (no GPU)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from phasespace import WORKLOADS, make_inputs, rambo, incoming_beams
from oracle import closed_forms as cf
from oracle.berends_giele import jamps_ggttng
from oracle.colour import colour_matrix, flow_permutations, rationalise
from oracle.diagrams import enumerate_diagrams, parse_process
from oracle.matrix_element import MatrixElement, get, select, near_tie
from oracle.model import Params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    return [l.rstrip("\n") for l in open(os.path.join(GOLDEN, name)) if l.strip() and not l.startswith("#")]


def _split(line):
    proc, rest = line.split(">")
    parts = rest.split()
    # process string keeps its particle names; the numeric fields follow
    names = [x for x in parts if not x[0].isdigit()]
    nums = [x for x in parts if x[0].isdigit()]
    return proc.strip() + " > " + " ".join(names), nums


def test_diagram_counts():
    for line in _golden("diagram_counts.txt"):
        proc, nums = _split(line)
        _, d = enumerate_diagrams(*parse_process(proc))
        assert len(d) == int(nums[0]), proc


def _exact_2to2(p, mass=0.0):
    """Rebuild exactly on-shell, back-to-back final momenta along the first final
    particle's direction (RAMBO roundoff leaves ~1e-13 inconsistencies, which forward
    kinematics amplify); the pins then measure the amplitude code, not the inputs."""
    q = p.copy()
    e = 0.5 * (p[:, 0, 0] + p[:, 1, 0])
    d = p[:, 2, 1:] / np.sqrt((p[:, 2, 1:] ** 2).sum(-1))[:, None]
    k = np.sqrt(e * e - mass * mass)
    q[:, 2, 0] = q[:, 3, 0] = e
    q[:, 2, 1:] = k[:, None] * d
    q[:, 3, 1:] = -k[:, None] * d
    return q


def _boost(p, beta):
    b = np.asarray(beta, float)
    b2 = b @ b
    g = 1.0 / math.sqrt(1.0 - b2)
    bp = p[..., 1:] @ b
    out = np.empty_like(p)
    out[..., 0] = g * (p[..., 0] + bp)
    out[..., 1:] = p[..., 1:] + ((g - 1.0) * bp / b2 + g * p[..., 0])[..., None] * b
    return out


def _rotate(p, axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    R = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
    out = p.copy()
    out[..., 1:] = p[..., 1:] @ R.T
    return out


def test_eemumu_per_helicity_closed_form():
    p, a, _, _ = make_inputs(WORKLOADS["eemumu"], 256)
    p = _exact_2to2(p)
    me = get("e+ e- > mu+ mu-")
    r = me.evaluate(p, a)
    ref = cf.eemumu_helicity(p)
    assert np.all((ref == 0) == (r["mh"] == 0))            # exact chirality zeros
    # relative to the event's largest helicity: (1 -+ cos th)^2 itself loses digits near th = 0, pi
    assert (np.abs(r["mh"] - ref) / ref.max(axis=1, keepdims=True)).max() < 1e-13
    assert sorted(me.helicity_filter(p[:16], a[:16])) == [5, 6, 9, 10]


def test_ggtt_combridge():
    me = MatrixElement("g g > t t~", Params(wt=0.0))
    p, a, _, _ = make_inputs(WORKLOADS["ggtt"], 256)
    p = _exact_2to2(p, 173.0)
    r = me.evaluate(p, a)
    assert np.abs(r["me"] / cf.ggQQ_average(p, a, 173.0) - 1).max() < 1e-12


def test_ggtt_massless_limit_textbook():
    me = MatrixElement("g g > t t~", Params(mt=0.0, wt=0.0))
    po, _ = rambo(64, 1500.0, [0.0, 0.0], seed=21)
    p = _exact_2to2(np.concatenate([incoming_beams(64, 1500.0), po], axis=1))
    a = np.full(64, 0.118)
    s = 2 * (p[:, 0, 0] * p[:, 1, 0] - (p[:, 0, 1:] * p[:, 1, 1:]).sum(-1))
    t = -2 * (p[:, 0, 0] * p[:, 2, 0] - (p[:, 0, 1:] * p[:, 2, 1:]).sum(-1))
    u = -s - t
    g4 = (4 * math.pi * 0.118) ** 2
    # textbook g g -> q qbar (massless), spin/colour averaged
    ref = g4 * ((t * t + u * u) / (6 * t * u) - 3.0 / 8.0 * (t * t + u * u) / (s * s))
    assert np.abs(me.evaluate(p, a)["me"] / ref - 1).max() < 1e-12


def test_gggg_textbook():
    me = get("g g > g g")
    po, _ = rambo(64, 1500.0, [0.0, 0.0], seed=11)
    p = _exact_2to2(np.concatenate([incoming_beams(64, 1500.0), po], axis=1))
    a = np.full(64, 0.118)
    # me includes the 1/2! identical-gluon factor; the textbook form does not
    assert np.abs(2.0 * me.me_bruteforce_colour(p, a) / cf.gggg_average(p, a) - 1).max() < 1e-12


def test_colour_matrices_exact():
    for line in _golden("colour_matrices.txt"):
        proc, nums = _split(line)
        n = int(nums[0])
        diag = Fraction(nums[1])
        gl = list(range(n))
        perms = flow_permutations(gl)
        if n <= 4:
            C = rationalise(colour_matrix(gl, perms, gl + [n, n + 1], n, n + 1))
            assert all(C[i][i] == diag for i in range(len(perms)))
            assert all(C[i][j] == C[j][i] for i in range(len(perms)) for j in range(len(perms)))
            ev = np.linalg.eigvalsh(np.array([[float(x) for x in r] for r in C]))
            assert ev.min() > 0
            if len(nums) > 2:
                full = [[Fraction(x) for x in row.split(",")] for row in nums[2].split(";")]
                assert C == full
        assert diag == Fraction(3) * Fraction(4, 3) ** n


def test_flow_decomposition_vs_bruteforce_colour_sum():
    for proc, wl, n in [("g g > t t~", "ggtt", 32), ("g g > t t~ g", "ggttg", 16), ("g g > t t~ g g", "ggttgg", 2)]:
        me = get(proc)
        p, a, _, _ = make_inputs(WORKLOADS[wl], n)
        r = me.evaluate(p, a)
        assert np.abs(me.me_bruteforce_colour(p, a) / r["me"] - 1).max() < 1e-13, proc


def test_berends_giele_equals_interpreter_jamps():
    for proc, wl, n in [("g g > t t~", "ggtt", 16), ("g g > t t~ g", "ggttg", 8), ("g g > t t~ g g", "ggttgg", 2)]:
        me = get(proc)
        p, a, _, _ = make_inputs(WORKLOADS[wl], n)
        J = me.jamps(p, a)
        perms, Jbg = jamps_ggttng(p, a)
        assert perms == me.perms
        assert np.abs(Jbg - J).max() / np.abs(J).max() < 1e-13, proc


def test_berends_giele_equals_interpreter_jamps_five_gluons():
    """g g > t t~ g g g, the 1240-diagram process of the large workload: every jamp of all 128
    helicities from the diagram interpreter equals the colour-ordered recursion's (one event; the
    recursion sums gluon currents over splittings and never forms a diagram), and |M|^2 is
    symmetric under a relabelling of the final gluons."""
    me = get("g g > t t~ g g g")
    p, a, _, _ = make_inputs(WORKLOADS["ggttggg"], 1)
    J = me.jamps(p, a)
    perms, Jbg = jamps_ggttng(p, a)
    assert perms == me.perms and J.shape == (1, 128, 120)
    assert np.abs(Jbg - J).max() / np.abs(J).max() < 1e-13
    # Bose symmetry of the three final gluons: a cyclic relabelling leaves |M|^2 unchanged only if
    # the enumeration misses no diagram and the flow decomposition is right
    q = p.copy()
    q[:, [4, 5, 6]] = p[:, [5, 6, 4]]
    r = me.evaluate(p, a)["me"]
    assert np.abs(me.evaluate(q, a)["me"] / r - 1).max() < 1e-13


def test_lorentz_invariance():
    # a boost changes the polarisation vectors by terms proportional to k, so the
    # helicity sum is frame independent only where the Ward identity holds: zero width
    me = MatrixElement("g g > t t~ g g", Params(wt=0.0))
    p, a, _, _ = make_inputs(WORKLOADS["ggttgg"], 4)
    r0 = me.evaluate(p, a)["me"]
    q = _rotate(_boost(p, [0.3, -0.2, 0.5]), [1.0, 2.0, -0.5], 0.7)
    r1 = me.evaluate(q, a)["me"]
    assert np.abs(r1 / r0 - 1).max() < 1e-11


def test_gauge_invariance_zero_width():
    me = MatrixElement("g g > t t~ g g", Params(wt=0.0))
    p, a, _, _ = make_inputs(WORKLOADS["ggttgg"], 3)
    J = me.jamps(p, a)
    scale = np.abs(J).max()
    for leg in (0, 1, 4, 5):
        Jg = me.jamps(p, a, gauge_leg=leg)
        assert np.abs(Jg).max() / (scale * p[:, leg, 0].max()) < 1e-13, leg


def test_alpha_s_scaling_and_bose_symmetry():
    me = get("g g > t t~ g")
    p, a, _, _ = make_inputs(WORKLOADS["ggttg"], 8)
    r1 = me.evaluate(p, a)["me"]
    r2 = me.evaluate(p, 2.0 * a)["me"]
    assert np.abs(r2 / r1 - 2.0 ** 3).max() < 1e-13
    me4 = get("g g > t t~ g g")
    p, a, _, _ = make_inputs(WORKLOADS["ggttgg"], 3)
    q = p.copy()
    q[:, [4, 5]] = p[:, [5, 4]]
    assert np.abs(me4.evaluate(q, a)["me"] / me4.evaluate(p, a)["me"] - 1).max() < 1e-13


def test_helicity_filter_keeps_full_sum():
    me = get("e+ e- > mu+ mu-")
    p, a, _, _ = make_inputs(WORKLOADS["eemumu"], 64)
    r = me.evaluate(p, a)
    good = me.helicity_filter(p[:16], a[:16])
    assert np.array_equal(r["mh"][:, good].sum(axis=1), r["mh"].sum(axis=1)) or \
        np.abs(r["mh"][:, good].sum(axis=1) / r["mh"].sum(axis=1) - 1).max() < 1e-15


def test_selection_rule_bruteforce():
    rng = np.random.default_rng(0)
    w = rng.random((500, 7)) * (rng.random((500, 7)) > 0.3)
    w[:, 0] += 1e-3
    r = rng.random(500)
    got = select(w, r)
    for e in range(500):
        tot = w[e].sum()
        acc = 0.0
        for k in range(7):
            acc += w[e, k]
            if acc > r[e] * tot:
                break
        assert got[e] == k


def test_near_tie_constructed_cases():
    """The mask that drops an event from the bit-exact selection comparison (reading P7: some
    cumulative weight within rel * total of r * total).  Integer weights make every cumulative sum
    and the total exact, so the distance of r * total to each cumulative sum is known by
    construction: exactly on a cumulative sum (a tie), half a step inside the window (a tie), four
    window widths away (not a tie) and halfway between two cumulative sums (not a tie).  A widened,
    narrowed, inverted or off-by-one mask fails one of these."""
    rng = np.random.default_rng(11)
    n, k = 400, 6
    w = rng.integers(1, 100, size=(n, k)).astype(np.float64)
    cs = np.cumsum(w, axis=1)
    tot = cs[:, -1]
    rel = 1e-12
    col = rng.integers(0, k - 1, size=n)          # an interior cumulative sum per event
    c = cs[np.arange(n), col]
    prev = np.where(col > 0, cs[np.arange(n), np.maximum(col - 1, 0)], 0.0)
    exact = c / tot                                # r * total lands on cs[col] up to one rounding
    inside = (c + 0.5 * rel * tot) / tot           # half a window above it
    outside = (c + 4.0 * rel * tot) / tot          # four windows above it
    below = (c - 4.0 * rel * tot) / tot
    midway = 0.5 * (prev + c) / tot                # between two cumulative sums (steps are >= 1)
    assert near_tie(w, exact, rel).all()
    assert near_tie(w, inside, rel).all()
    assert not near_tie(w, outside, rel).any()
    assert not near_tie(w, below, rel).any()
    assert not near_tie(w, midway, rel).any()
    # the window scales with the total, not with the weights' magnitude
    assert near_tie(1e-30 * w, exact, rel).all() and not near_tie(1e-30 * w, midway, rel).any()
    # a tie on the last cumulative sum (r -> 1) counts too; the default window is 1e-12
    assert near_tie(w, 1.0 - 0.5 * rel * np.ones(n)).all()
    assert not near_tie(w, 1.0 - 4.0 * rel * np.ones(n)).any()
    # mixed rows: exactly the constructed ties are flagged, row by row
    pick = rng.random(n) < 0.3
    r = np.where(pick, inside, midway)
    assert np.array_equal(near_tie(w, r, rel), pick)
    # uniform random r: ties have probability ~ k * 2e-12 per event, so none in this sample
    assert not near_tie(w, rng.random(n), rel).any()


def test_selection_frequencies_follow_weights():
    me = get("g g > t t~")
    p, a, _, _ = make_inputs(WORKLOADS["ggtt"], 1)
    pp = np.repeat(p, 20000, axis=0)
    aa = np.repeat(a, 20000)
    rng = np.random.default_rng(3)
    r = me.evaluate(pp[:1], aa[:1])
    mh = r["mh"][0]
    sel = select(np.repeat(r["mh"], 20000, axis=0), rng.random(20000))
    counts = np.bincount(sel, minlength=16)
    expect = 20000 * mh / mh.sum()
    m = expect > 5
    chi2 = ((counts[m] - expect[m]) ** 2 / expect[m]).sum()
    assert chi2 < 3 * m.sum() + 30
    assert np.all(counts[~m] <= 20)


def test_ew_qcd_process_colour_and_gauge():
    """g u~ > ta+ ta- g g u~ (photon/Z to a massive tau pair, one quark line, three gluons):
    flow decomposition vs the explicit colour sum, and the gluon Ward identity (no top width)."""
    me = get("g u~ > ta+ ta- g g u~")
    p, a, _, _ = make_inputs(WORKLOADS["gu_tataggu"], 4)
    assert np.abs(me.me_bruteforce_colour(p[:2], a[:2]) / me.evaluate(p[:2], a[:2])["me"] - 1).max() < 1e-13
    J = me.jamps(p, a)
    for leg in (0, 4, 5):
        assert np.abs(me.jamps(p, a, gauge_leg=leg)).max() / (np.abs(J).max() * p[:, leg, 0].max()) < 1e-13


def test_condition_estimate():
    """The parity tests' condition estimate: at least 1 (triangle inequality on the diagram sum),
    modest for the two-diagram e+e- -> mu+mu-, and larger where a propagator nearly goes on shell
    (a gluon pair made nearly collinear in g g > t t~ g g)."""
    me = get("e+ e- > mu+ mu-")
    p, a, _, _ = make_inputs(WORKLOADS["eemumu"], 64)
    k = me.condition(p, a)
    assert np.all(k >= 1.0) and k.max() < 1e3
    me4 = get("g g > t t~ g g")
    p, a, _, _ = make_inputs(WORKLOADS["ggttgg"], 8)
    k0 = me4.condition(p, a)
    q = p.copy()
    # rotate gluon 5 onto gluon 4's direction up to 1e-6 rad, keeping its energy; the top pair
    # absorbs the three-momentum change (energy conservation is irrelevant to the estimate)
    d = q[:, 4, 1:] / np.linalg.norm(q[:, 4, 1:], axis=1, keepdims=True)
    perp = np.cross(d, [0.0, 0.0, 1.0])
    perp /= np.linalg.norm(perp, axis=1, keepdims=True)
    n5 = d + 1e-6 * perp
    n5 /= np.linalg.norm(n5, axis=1, keepdims=True)
    new5 = q[:, 5, :1] * n5
    shift = (new5 - q[:, 5, 1:]) / 2
    q[:, 5, 1:] = new5
    for t in (2, 3):
        q[:, t, 1:] -= shift
        q[:, t, 0] = np.sqrt(173.0 ** 2 + (q[:, t, 1:] ** 2).sum(-1))
    k1 = me4.condition(q, a)
    assert np.all(k0 >= 1.0) and np.median(k1) > 100 * np.median(k0)
