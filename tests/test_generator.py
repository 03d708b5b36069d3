"""Host logic of the process compiler (gen/): its colour algebra against the oracle's independent
one, diagram counts, and structural invariants of the op tables the kernels execute."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2503_21935_gb300.gen import program as pg
from paper_2503_21935_gb300.gen.emit import BUILTIN


@pytest.fixture(scope="module")
def programs():
    return {p: pg.build_program(p) for p in BUILTIN}


@pytest.mark.parametrize("proc", ["g g > t t~", "g g > t t~ g", "g g > t t~ g g", "g g > t t~ g g g"])
def test_colour_matrix_equals_oracle(proc, programs):
    """Symbolic Fierz reduction (compiler) against explicit colour-index sums (oracle), exactly."""
    from oracle.matrix_element import get
    P = programs[proc]
    m = get(proc)
    assert [tuple(x) for x in P.perms] == [tuple(x) for x in m.perms]
    assert [[Fraction(x) for x in row] for row in P.colour] == [[Fraction(x) for x in row] for row in m.C_exact]


def test_five_gluon_colour_matrix_properties(programs):
    C = programs["g g > t t~ g g g"].colour
    n = len(C)
    assert n == 120
    assert all(C[i][i] == Fraction(1024, 81) for i in range(n))
    assert all(C[i][j] == C[j][i] for i in range(n) for j in range(i))
    assert np.linalg.eigvalsh(np.array([[float(x) for x in r] for r in C])).min() > 0.0


def test_diagram_counts_and_gs_power(programs):
    expect = {"e+ e- > mu+ mu-": (2, 0), "g g > t t~": (3, 2), "g g > t t~ g": (16, 3), "g g > t t~ g g": (123, 4),
              "g g > t t~ g g g": (1240, 5), "g u~ > ta+ ta- g g u~": (None, 3)}
    for proc, (nd, gsp) in expect.items():
        P = programs[proc]
        if nd is not None:
            assert P.ndiagrams == nd, proc
        assert P.gs_power == gsp, proc


def _terms(P, start, count):
    return [P.terms[8 * k: 8 * k + 8] for k in range(start, start + count)]


def test_op_table_invariants(programs):
    for proc, P in programs.items():
        full = (1 << P.npar) - 1
        seen_first = set()
        for op in P.ops:
            if op[0] == pg.OP_AMP:
                # every term closes all legs exactly once: bilinear legs and other-operand legs
                for t in _terms(P, op[11], op[12]):
                    assert t[1] & t[3] == 0 and t[1] | t[3] == full, proc
                    assert t[4] in (0, 1, 2, 3) and t[5] in (0, 1)
                # flows: valid index, one first-write flag per flow, at its first occurrence
                for k in range(op[9], op[9] + op[10]):
                    f, code = P.flows[2 * k], P.flows[2 * k + 1]
                    assert 0 <= f < P.ncol
                    first = bool(code & pg.FLOW_FIRST)
                    assert first == (f not in seen_first), proc
                    seen_first.add(f)
            elif op[0] == pg.OP_SUM:
                # summands cover exactly the sum current's legs
                for t in _terms(P, op[11], op[12]):
                    assert t[1] == op[5], proc
        assert P.jamp_zero == (0 if len(seen_first) == P.ncol else 1)


def _fp64_work(P, ngood):
    """Float64 instructions per event of a program under the kernels' per-op counts (the model the
    library's roofline uses; colour sum and weights left out, they do not depend on the closure)."""
    c = P.flop_counts
    per_var = (64 * (c["var_ffv_f"] + c["var_ffv_fb"]) + 72 * c["var_ffv_v"] + 56 * c["var_vvv"]
               + 32 * c["var_vvvv"] + 56 * c["var_bil"] + 32 * c["var_rbil"])
    amp = ngood * (16 * c["amp_runs"] + 8 * (c["amp_terms"] - c["amp_runs"]) + 2 * (c["amp_runs"] - c["amp"])
                   + 2 * (c["amp_flows"] - P.ncol))
    hdr = 8 * c["sum_adds"] + 8 * c["vvv_hdr"] + 18 * c["vvvv_hdr"] + 8 * c["slash_hdr"] + 16 * c["slash_pref_hdr"]
    return per_var + amp + hdr


@pytest.mark.parametrize("proc", BUILTIN)
def test_flow_major_closure_only_where_it_saves_work(proc, programs, monkeypatch):
    """The flow-major closure changes the amplitude stage only: every current op of the group-major
    program is still there, and the modelled float64 work per event never grows.  For
    g g > t t~ g g it closes exactly the four row bilinears whose 15 groups reach 6 flows each
    (105 -> 69 products per helicity)."""
    P = programs[proc]
    monkeypatch.setattr(pg, "_flow_major_bilinears", lambda B, groups, gruns: {})
    G = pg.build_program(proc)
    key = lambda op: (op[0], op[5], op[6], op[7], op[8], op[9], op[10])
    cur_ops = lambda Q: sorted(key(op) for op in Q.ops if op[0] not in (pg.OP_AMP, pg.OP_SUM))
    assert cur_ops(P) == cur_ops(G)
    ngood = 1 << P.npar
    assert _fp64_work(P, ngood) <= _fp64_work(G, ngood)
    if proc == "g g > t t~ g g":
        assert (G.flop_counts["amp"], P.flop_counts["amp"]) == (105, 69)
        assert (G.flop_counts["amp_flows"], P.flop_counts["amp_flows"]) == (336, 240)
        single = [op for op in P.ops if op[0] == pg.OP_AMP and op[10] == 1 and op[12] == 1]
        assert len(single) == 24                      # 4 bilinears x 6 flows
        assert _fp64_work(P, ngood) < 0.9 * _fp64_work(G, ngood)
    if proc in ("e+ e- > mu+ mu-", "g g > t t~"):
        assert P.ops == G.ops and P.flows == G.flows and P.terms == G.terms
