"""Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11,
"Parallel random numbers: as easy as 1, 2, 3").

Each output block of four 32-bit words is a pure function of (counter, key), so
an event's random numbers depend only on its index and the seed, never on how
many threads or chunks produced them.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Apply the 10-round Philox-4x32 bijection.

    ctr: uint32 array [..., 4]; key: uint32 array broadcastable to [..., 2].
    Returns uint32 array [..., 4].
    """
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.broadcast_to(np.asarray(key, dtype=np.uint32), c.shape[:-1] + (2,))
    c0, c1, c2, c3 = (c[..., i].astype(np.uint64) for i in range(4))
    k0 = k[..., 0].astype(np.uint32).copy()
    k1 = k[..., 1].astype(np.uint32).copy()
    with np.errstate(over="ignore"):
        for r in range(10):
            if r:
                k0 = k0 + _W0
                k1 = k1 + _W1
            p0 = _M0 * c0
            p1 = _M1 * c2
            hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
            hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
            c0, c1, c2, c3 = (hi1 ^ c1 ^ k0.astype(np.uint64), lo1,
                              hi0 ^ c3 ^ k1.astype(np.uint64), lo0)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def _blocks(seed, stream, nevt, nblocks):
    """Raw words for events 0..nevt-1: counter = (event, block, stream, 0), key = seed."""
    ev = np.arange(nevt, dtype=np.uint64)
    blk = np.arange(nblocks, dtype=np.uint32)
    ctr = np.zeros((nevt, nblocks, 4), dtype=np.uint32)
    ctr[..., 0] = (ev & np.uint64(0xFFFFFFFF)).astype(np.uint32)[:, None]
    ctr[..., 1] = blk[None, :]
    ctr[..., 2] = np.uint32(stream)
    ctr[..., 3] = (ev >> np.uint64(32)).astype(np.uint32)[:, None]
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    return philox4x32_10(ctr, key)


def uniform_open01(seed, stream, nevt, n):
    """n uniforms per event in the open interval (0,1) (24+ bits; safe for log)."""
    nb = (n + 3) // 4
    w = _blocks(seed, stream, nevt, nb).reshape(nevt, nb * 4)[:, :n]
    return (w.astype(np.float64) + 0.5) * (1.0 / 4294967296.0)


def uniform01(seed, stream, nevt):
    """One 53-bit uniform per event in [0,1)."""
    w = _blocks(seed, stream, nevt, 1)[:, 0, :]
    hi = (w[:, 0] >> np.uint32(5)).astype(np.float64)
    lo = (w[:, 1] >> np.uint32(6)).astype(np.float64)
    return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0)
