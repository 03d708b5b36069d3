"""Dirac algebra and external wavefunctions (float64 / complex128, numpy).

Conventions (Peskin & Schroeder; chiral representation; metric (+,-,-,-)):
  gamma^mu = [[0, sigma^mu], [sigmabar^mu, 0]],  sigma^mu = (1, s),  sigmabar^mu = (1, -s)
  gamma^5 = diag(-1,-1,+1,+1);  P_L = (1 - gamma^5)/2 selects the upper two components.

External states are helicity eigenstates in the frame where momenta are given
(HELAS, KEK-91-11: two-component helicity spinors chi_lambda(p) and
polarisation vectors built from the unit vectors e1, e2 orthogonal to p):
  u(p, l)  = ( sqrt(E - l|p|) chi_l ,  sqrt(E + l|p|) chi_l )
  v(p, l)  = ( sqrt(E + l|p|) chi_-l , -sqrt(E - l|p|) chi_-l )   (l = physical helicity)
  eps(k, l) = ( -l e1 - i e2 ) / sqrt(2)
Barred spinors are psi^dagger gamma^0; an outgoing vector uses eps^*.
All functions take momenta [nevt, 4] and return [nevt, 2, 4] arrays whose axis 1
is the helicity index (0 -> helicity -1, 1 -> helicity +1).
"""
import numpy as np

METRIC = np.diag([1.0, -1.0, -1.0, -1.0])

_S = [np.eye(2, dtype=complex), np.array([[0, 1], [1, 0]], dtype=complex),
      np.array([[0, -1j], [1j, 0]], dtype=complex), np.array([[1, 0], [0, -1]], dtype=complex)]


def _gamma():
    g = np.zeros((4, 4, 4), dtype=complex)
    for mu in range(4):
        sig = _S[mu]
        sbar = _S[mu] if mu == 0 else -_S[mu]
        g[mu, :2, 2:] = sig
        g[mu, 2:, :2] = sbar
    return g


GAMMA = _gamma()                                      # GAMMA[mu] = gamma^mu (upper index)
GAMMA5 = np.diag([-1.0, -1.0, 1.0, 1.0]).astype(complex)
PL = np.diag([1.0, 1.0, 0.0, 0.0]).astype(complex)
PR = np.diag([0.0, 0.0, 1.0, 1.0]).astype(complex)


def slash(k):
    """k-slash = gamma^mu k_mu for k [nevt, 4] (upper components) -> [nevt, 4, 4]."""
    klow = k @ METRIC
    return np.einsum("nm,mab->nab", klow.astype(complex), GAMMA)


def minkowski(a, b):
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


def _chi(p):
    """Two-component helicity eigenstates chi_-(p), chi_+(p): [nevt, 2(hel), 2]."""
    px, py, pz = p[:, 1], p[:, 2], p[:, 3]
    pp = np.sqrt(px * px + py * py + pz * pz)
    n = p.shape[0]
    chi = np.zeros((n, 2, 2), dtype=complex)
    a = pp + pz
    reg = a > 0.0
    norm = np.sqrt(2.0 * pp[reg] * a[reg])
    chi[reg, 1, 0] = a[reg] / norm
    chi[reg, 1, 1] = (px[reg] + 1j * py[reg]) / norm
    chi[reg, 0, 0] = (-px[reg] + 1j * py[reg]) / norm
    chi[reg, 0, 1] = a[reg] / norm
    # p along -z: theta = pi, phi = 0
    back = (~reg) & (pp > 0.0)
    chi[back, 1] = (0.0, 1.0)
    chi[back, 0] = (-1.0, 0.0)
    # p = 0: quantise along +z
    rest = pp == 0.0
    chi[rest, 1] = (1.0, 0.0)
    chi[rest, 0] = (0.0, 1.0)
    return chi, pp


def _weights(e, pp, lam, mass):
    """sqrt(E - lam|p|), sqrt(E + lam|p|); for a massless particle E = |p| is used
    exactly, so the wrong-chirality half of the spinor is an exact zero."""
    if mass == 0.0:
        z = np.zeros_like(e)
        s = np.sqrt(2.0 * e)
        return (z, s) if lam > 0 else (s, z)
    return np.sqrt(np.maximum(e - lam * pp, 0.0)), np.sqrt(np.maximum(e + lam * pp, 0.0))


def u_spinor(p, mass):
    chi, pp = _chi(p)
    e = p[:, 0]
    out = np.zeros((p.shape[0], 2, 4), dtype=complex)
    for h, lam in ((0, -1.0), (1, 1.0)):
        wm, wp = _weights(e, pp, lam, mass)
        out[:, h, :2] = wm[:, None] * chi[:, h]
        out[:, h, 2:] = wp[:, None] * chi[:, h]
    return out


def v_spinor(p, mass):
    chi, pp = _chi(p)
    e = p[:, 0]
    out = np.zeros((p.shape[0], 2, 4), dtype=complex)
    for h, lam in ((0, -1.0), (1, 1.0)):
        c = chi[:, 1 - h]
        wm, wp = _weights(e, pp, lam, mass)
        out[:, h, :2] = wp[:, None] * c
        out[:, h, 2:] = -wm[:, None] * c
    return out


def bar(psi):
    """psi^dagger gamma^0 for spinors [..., 4]."""
    return np.einsum("...a,ab->...b", psi.conj(), GAMMA[0])


def polarisation(k):
    """eps^mu(k, l) for l = -1, +1 (upper index): [nevt, 2, 4]."""
    kx, ky, kz = k[:, 1], k[:, 2], k[:, 3]
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    pt = np.sqrt(kx * kx + ky * ky)
    cth = np.where(kk > 0, kz / np.where(kk > 0, kk, 1.0), 1.0)
    sth = np.where(kk > 0, pt / np.where(kk > 0, kk, 1.0), 0.0)
    cph = np.where(pt > 0, kx / np.where(pt > 0, pt, 1.0), 1.0)
    sph = np.where(pt > 0, ky / np.where(pt > 0, pt, 1.0), 0.0)
    n = k.shape[0]
    e1 = np.zeros((n, 4))
    e2 = np.zeros((n, 4))
    e1[:, 1], e1[:, 2], e1[:, 3] = cth * cph, cth * sph, -sth
    e2[:, 1], e2[:, 2] = -sph, cph
    out = np.zeros((n, 2, 4), dtype=complex)
    for h, lam in ((0, -1.0), (1, 1.0)):
        out[:, h] = (-lam * e1 - 1j * e2) / np.sqrt(2.0)
    return out
