"""Flat n-body phase space by RAMBO (Kleiss, Stirling, Ellis, Comput. Phys. Commun.
40 (1986) 359), vectorised over events.

Momenta are returned as float64 arrays [nevt, n, 4] holding (E, px, py, pz) in GeV
in the partonic centre-of-mass frame.  Massive final states are obtained from
the massless configuration by the common rescaling factor xi solved with Newton
iterations, as in the RAMBO paper.  A final repair step restores momentum
conservation and the mass shells to rounding level.
"""
import math
import numpy as np

from .philox import uniform_open01


def incoming_beams(nevt, sqrts):
    """Two massless incoming partons along +z and -z, each with energy sqrt(s)/2."""
    e = 0.5 * sqrts
    p = np.zeros((nevt, 2, 4))
    p[:, 0] = (e, 0.0, 0.0, e)
    p[:, 1] = (e, 0.0, 0.0, -e)
    return p


def rambo_massless_weight(n, sqrts):
    """Constant massless n-body phase-space volume element returned by RAMBO."""
    po2 = 0.5 * math.pi
    w = po2 ** (n - 1) * sqrts ** (2 * n - 4) / (math.gamma(n) * math.gamma(n - 1))
    return w * (2.0 * math.pi) ** (4 - 3 * n)


def _repair(p, masses, sqrts):
    """Restore exact kinematics to rounding level.  The RAMBO boost loses digits when the
    generated massless momenta are nearly collinear (Q nearly lightlike): the outgoing momenta
    then miss momentum conservation and the mass shell by up to ~1e-11 relative, and amplitudes
    evaluated from them depend at that level on which momenta a formula uses.  Step 1 removes
    the residual three-momentum in proportion to the energies; step 2 rescales all
    three-momenta by the factor xi with sum_i sqrt(m_i^2 + xi^2 |p_i|^2) = sqrt(s) (Newton,
    from xi = 1) and recomputes every energy from its three-momentum."""
    p = p.copy()
    r = p[..., 1:].sum(axis=1)
    p[..., 1:] -= r[:, None, :] * (p[..., 0] / p[..., 0].sum(axis=1, keepdims=True))[..., None]
    k2 = (p[..., 1:] ** 2).sum(axis=-1)
    m2 = np.asarray(masses, dtype=np.float64)[None, :] ** 2
    xi = np.ones(p.shape[0])
    for _ in range(8):
        e = np.sqrt(m2 + xi[:, None] ** 2 * k2)
        step = (e.sum(axis=1) - sqrts) / (xi[:, None] * k2 / e).sum(axis=1)
        xi = xi - step
    p[..., 1:] *= xi[:, None, None]
    p[..., 0] = np.sqrt(m2 + (p[..., 1:] ** 2).sum(axis=-1))
    return p


def rambo(nevt, sqrts, masses, seed, stream=0):
    """Generate nevt events of len(masses) outgoing particles at total energy sqrts.

    Returns (momenta[nevt, n, 4], weight[nevt]).  The random numbers of event i
    are Philox words with counter (i, block, stream) and key seed, so the output
    does not depend on batching or thread count.
    """
    masses = np.asarray(masses, dtype=np.float64)
    n = masses.shape[0]
    r = uniform_open01(seed, stream, nevt, 4 * n).reshape(nevt, n, 4)
    c = 2.0 * r[..., 0] - 1.0
    s = np.sqrt(np.maximum(0.0, 1.0 - c * c))
    f = 2.0 * math.pi * r[..., 1]
    q0 = -np.log(r[..., 2] * r[..., 3])
    q = np.stack([q0, q0 * s * np.cos(f), q0 * s * np.sin(f), q0 * c], axis=-1)
    Q = q.sum(axis=1)
    M = np.sqrt(Q[:, 0] ** 2 - (Q[:, 1:] ** 2).sum(axis=1))
    b = -Q[:, 1:] / M[:, None]
    g = Q[:, 0] / M
    a = 1.0 / (1.0 + g)
    x = sqrts / M
    bq = (b[:, None, :] * q[..., 1:]).sum(axis=-1)
    p = np.empty_like(q)
    p[..., 0] = x[:, None] * (g[:, None] * q[..., 0] + bq)
    p[..., 1:] = x[:, None, None] * (q[..., 1:] + b[:, None, :] * q[..., :1]
                                     + a[:, None, None] * bq[..., None] * b[:, None, :])
    w = np.full(nevt, rambo_massless_weight(n, sqrts))
    if not np.any(masses > 0.0):
        return _repair(p, masses, sqrts), w
    if masses.sum() >= sqrts:
        raise ValueError("final-state masses exceed sqrt(s)")
    # Newton iteration for xi: sum_i sqrt(m_i^2 + xi^2 E_i^2) = sqrts (massless |p_i| = E_i)
    m2 = masses[None, :] ** 2
    e0 = p[..., 0]
    xi = np.full(nevt, math.sqrt(1.0 - (masses.sum() / sqrts) ** 2))
    for _ in range(60):
        e = np.sqrt(m2 + (xi[:, None] * e0) ** 2)
        fval = e.sum(axis=1) - sqrts
        dfdx = (xi[:, None] * e0 ** 2 / e).sum(axis=1)
        step = fval / dfdx
        xi = xi - step
        if np.all(np.abs(step) <= 1e-15 * xi):
            break
    k = np.empty_like(p)
    k[..., 1:] = xi[:, None, None] * p[..., 1:]
    k[..., 0] = np.sqrt(m2 + (xi[:, None] * e0) ** 2)
    k = _repair(k, masses, sqrts)
    kabs = np.sqrt((k[..., 1:] ** 2).sum(axis=-1))
    wt = (kabs.sum(axis=1) / sqrts) ** (2 * n - 3)
    wt = wt * np.prod(kabs / k[..., 0], axis=1) * sqrts / (kabs ** 2 / k[..., 0]).sum(axis=1)
    return k, w * wt
