"""Colour-ordered Berends-Giele recursion for g g -> t tbar + n g (independent tier).

Berends & Giele, Nucl. Phys. B306 (1988) 759.  For one quark line the amplitude
decomposes as M = sum_s (T^{a_s1} ... T^{a_sn})_{i_t j_tbar} A(s); each A(s) is
obtained from off-shell currents with colour-ordered rules derived from the
same Feynman rules as the diagram interpreter, f^{xyz} T^z = -i [T^x, T^y]:
  3-gluon, ordered (L, R):      -i g_s V^{mnr}(kL, kR, -(kL+kR))
  4-gluon, ordered (L, M, R):   -i g_s^2 [ -(g^mr g^ns - g^ms g^nr) + (g^mn g^rs - g^mr g^ns) ]
  quark-gluon:                   i g_s gamma^mu
Gluon currents J(B) of consecutive ordered gluons are summed over all splittings
(no individual Feynman diagrams appear), so this tier shares the physics but not
the algorithm of the diagram interpreter.  Works in all-incoming momenta.
"""
import itertools
import math

import numpy as np

from . import lorentz as L
from .model import Params


def _vvv(k1, k2, k3):
    g = L.METRIC
    return (np.einsum("mn,er->emnr", g, k1 - k2) + np.einsum("nr,em->emnr", g, k2 - k3)
            + np.einsum("rm,en->emnr", g, k3 - k1)).astype(complex)


_G = L.METRIC
_G1 = np.einsum("mr,ns->mnrs", _G, _G) - np.einsum("ms,nr->mnrs", _G, _G)
_G3 = np.einsum("mn,rs->mnrs", _G, _G) - np.einsum("mr,ns->mnrs", _G, _G)
_V4_ORDERED = (_G3 - _G1).astype(complex)


def jamps_ggttng(p, alpha_s, params=None, helicity=None):
    """Ordered amplitudes A[nevt, nhel, n!] for g g > t t~ g^n (legs g, g, t, t~, g...).

    Permutations of the gluon legs in lexicographic order; all 2^npar helicities
    unless `helicity` (a canonical index) is given.
    """
    prm = params or Params()
    nevt, npar, _ = p.shape
    gl = [0, 1] + list(range(4, npar))
    q = p.copy()
    q[:, 2:] *= -1.0                      # incoming momenta
    gs = np.sqrt(4.0 * math.pi * np.asarray(alpha_s, dtype=float)) * np.ones(nevt)
    m, w = prm.mt, prm.wt
    eps = {}
    for i in gl:
        e = L.polarisation(p[:, i])
        if i >= 2:
            e = e.conj()
        eps[i] = e @ L.METRIC             # lowered, [nevt, 2, 4]
    ubar_t = L.bar(L.u_spinor(p[:, 2], m))  # [nevt, 2, 4]
    v_tb = L.v_spinor(p[:, 3], m)
    hels = range(2 ** npar) if helicity is None else [helicity]
    perms = list(itertools.permutations(gl))
    out = np.zeros((nevt, len(hels), len(perms)), dtype=complex)
    for hi, h in enumerate(hels):
        bits = [(h >> (npar - 1 - k)) & 1 for k in range(npar)]
        for si, perm in enumerate(perms):
            out[:, hi, si] = _ordered(perm, bits, q, eps, ubar_t, v_tb, gs, m, w)
    return perms, out


def _ordered(perm, bits, q, eps, ubar_t, v_tb, gs, m, w):
    n = len(perm)
    nevt = q.shape[0]
    # gluon currents for blocks perm[i:j]
    J = {}
    K = {}
    for i in range(n):
        J[(i, i + 1)] = eps[perm[i]][np.arange(nevt), bits[perm[i]]]
        K[(i, i + 1)] = q[:, perm[i]]
    for size in range(2, n + 1):
        for i in range(0, n - size + 1):
            j = i + size
            P = sum(q[:, perm[x]] for x in range(i, j))
            K[(i, j)] = P
            acc = np.zeros((nevt, 4), dtype=complex)
            for k in range(i + 1, j):
                V = _vvv(K[(i, k)], K[(k, j)], -P)
                acc += -1j * gs[:, None] * np.einsum("emnr,em,en->er", V, J[(i, k)], J[(k, j)])
            for k in range(i + 1, j):
                for l in range(k + 1, j):
                    acc += -1j * (gs * gs)[:, None] * np.einsum("mnrs,em,en,er->es", _V4_ORDERED,
                                                                J[(i, k)], J[(k, l)], J[(l, j)])
            P2 = L.minkowski(P, P)
            J[(i, j)] = (-1j / P2)[:, None] * (acc @ L.METRIC)
    # quark line from the ubar(t) end
    hb_t, hb_tb = bits[2], bits[3]
    psi = {0: ubar_t[np.arange(nevt), hb_t]}
    amp = np.zeros(nevt, dtype=complex)
    qt = q[:, 2]
    for k in range(1, n + 1):
        acc = np.zeros((nevt, 4), dtype=complex)
        for j in range(0, k):
            vert = 1j * gs[:, None, None] * np.einsum("mab,em->eab", L.GAMMA, J[(j, k)])
            acc += np.einsum("ea,eab->eb", psi[j], vert)
        if k < n:
            kk = -(qt + sum(q[:, perm[x]] for x in range(k)))
            k2 = L.minkowski(kk, kk)
            S = 1j * (L.slash(kk) + m * np.eye(4)[None]) / (k2 - m * m + 1j * m * w)[:, None, None]
            psi[k] = np.einsum("ea,eab->eb", acc, S)
        else:
            amp = np.einsum("ea,ea->e", acc, v_tb[np.arange(nevt), hb_tb])
    return -1j * amp
