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


@pytest.mark.parametrize("proc", ["g g > t t~", "g g > t t~ g", "g g > t t~ g g"])
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
