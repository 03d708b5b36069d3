"""Explicit SU(3) colour algebra by brute force (numpy, complex128).

T^a = lambda^a / 2 (Gell-Mann matrices), Tr(T^a T^b) = delta^ab / 2,
f^abc = -2i Tr([T^a, T^b] T^c).  The colour-flow basis of a process with one
quark line (barred end i, unbarred end j) and gluons a_1..a_n is the set of
strings b_s = (T^{a_s1} ... T^{a_sn})_{ij}, s running over the permutations of
the gluon legs in lexicographic order.  The colour matrix is the explicit sum
C_st = sum_{all colour indices} conj(b_s) b_t  (the colour-matrix quadratic
form J^dagger C J of the paper's Sec. 3 acts with this C).
"""
import itertools
from fractions import Fraction

import numpy as np


def gell_mann_T():
    lam = np.zeros((8, 3, 3), dtype=complex)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam / 2


T = gell_mann_T()
F = (-2j * (np.einsum("aij,bjk,cki->abc", T, T, T) - np.einsum("bij,ajk,cki->abc", T, T, T))).real.copy()


def flow_permutations(gluon_legs):
    return list(itertools.permutations(gluon_legs))


def basis_at(configs, coloured_legs, gluon_legs, row_leg, col_leg, perms):
    """b_s evaluated at explicit colour configurations.

    configs: int array [R, len(coloured_legs)] of colour indices per coloured leg.
    Returns complex [R, len(perms)].
    """
    pos = {leg: k for k, leg in enumerate(coloured_legs)}
    R = configs.shape[0]
    out = np.zeros((R, len(perms)), dtype=complex)
    if row_leg is None:
        return np.ones((R, 1), dtype=complex)
    i = configs[:, pos[row_leg]]
    j = configs[:, pos[col_leg]]
    for s, perm in enumerate(perms):
        m = np.broadcast_to(np.eye(3, dtype=complex), (R, 3, 3)).copy()
        for leg in perm:
            m = m @ T[configs[:, pos[leg]]]
        out[:, s] = m[np.arange(R), i, j]
    return out


def basis_full(gluon_legs, perms, coloured_legs, row_leg, col_leg, first_gluon_index=None):
    """All b_s as a dense [nperm, ncolourconfigs] matrix (configs in coloured-leg order).

    With first_gluon_index set, only configurations whose first coloured gluon has
    that adjoint index (a slice used to bound memory).
    """
    dims = [8 if leg in gluon_legs else 3 for leg in coloured_legs]
    if first_gluon_index is not None:
        g0 = coloured_legs.index(gluon_legs[0])
        ranges = [range(d) if k != g0 else [first_gluon_index] for k, d in enumerate(dims)]
    else:
        ranges = [range(d) for d in dims]
    cfg = np.array(list(itertools.product(*ranges)), dtype=np.int64)
    return basis_at(cfg, coloured_legs, gluon_legs, row_leg, col_leg, perms).T, cfg


def colour_matrix(gluon_legs, perms, coloured_legs, row_leg, col_leg):
    """C_st = sum over all colour indices of conj(b_s) b_t, float64 (exactly rational)."""
    n = len(perms)
    C = np.zeros((n, n), dtype=complex)
    for a in range(8):
        B, _ = basis_full(gluon_legs, perms, coloured_legs, row_leg, col_leg, first_gluon_index=a)
        C += B.conj() @ B.T
    return C


def rationalise(M, max_den=10 ** 6, tol=1e-9):
    """Exact Fractions for a real matrix known to be rational (checked to tol)."""
    out = []
    for row in np.asarray(M).real:
        r = []
        for x in row:
            f = Fraction(float(x)).limit_denominator(max_den)
            if abs(float(f) - x) > tol * max(1.0, abs(x)):
                raise ValueError(f"entry {x} is not a simple rational")
            r.append(f)
        out.append(r)
    if np.abs(np.asarray(M).imag).max(initial=0.0) > tol:
        raise ValueError("colour matrix is not real")
    return out
