"""Float64 CPU reference of the MLP surrogate (forward and backward), for the gradient check.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network: 24 inputs (zero-padded to 32) -> 4 hidden layers of 256 with SiLU -> 1.  Mean squared
error loss.  The GPU kernels multiply bfloat16 operands exactly and accumulate in float32; this
reference rounds to bfloat16 at the same points (inputs, weights used in products, hidden
activations, back-propagated pre-activation gradients) and accumulates in float64, so the two
differ only by accumulation order (and the rare bfloat16 rounding flip that causes).

Parameter layout (flat float32 vector): per hidden layer W_l [256][kin_l] then b_l [256]
(kin_0 = 32), then w_out [256], b_out [1].
"""
import numpy as np

NIN, K0, WIDTH, DEPTH = 24, 32, 256, 4


def bf16(x):
    """Round to bfloat16 (nearest, ties to even) and return as float64."""
    a = np.asarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    Ws, bs, o = [], [], 0
    for l in range(DEPTH):
        kin = K0 if l == 0 else WIDTH
        Ws.append(p[o:o + WIDTH * kin].reshape(WIDTH, kin))
        o += WIDTH * kin
        bs.append(p[o:o + WIDTH])
        o += WIDTH
    w4 = p[o:o + WIDTH]
    b4 = p[o + WIDTH]
    return Ws, bs, w4, b4


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(p, x):
    Ws, bs, w4, b4 = unpack(p)
    n = x.shape[0]
    xin = np.zeros((n, K0))
    xin[:, :NIN] = x
    h = bf16(xin)
    cache = [h]
    zs = []
    for l in range(DEPTH):
        z = h @ bf16(Ws[l]).T + bs[l]
        zs.append(z)
        h = bf16(z * sigmoid(z))
        cache.append(h)
    y = h @ w4 + b4
    return y, zs, cache


def gradients(p, x, t):
    """Mean-squared-error loss and its gradient (flat, same layout as p)."""
    Ws, bs, w4, b4 = unpack(p)
    n = x.shape[0]
    y, zs, hs = forward(p, x)
    loss = np.mean((y - t) ** 2)
    dy = 2.0 * (y - t) / n
    grads_W, grads_b = [None] * DEPTH, [None] * DEPTH
    dw4 = hs[DEPTH].T @ dy
    db4 = dy.sum()

    def silu_grad(z):
        s = sigmoid(z)
        return s * (1.0 + z * (1.0 - s))
    dz = bf16(dy[:, None] * w4[None, :] * silu_grad(zs[DEPTH - 1]))
    for l in range(DEPTH - 1, -1, -1):
        grads_W[l] = dz.T @ hs[l]
        grads_b[l] = dz.sum(axis=0)
        if l == 0:
            break
        dz = bf16((dz @ bf16(Ws[l])) * silu_grad(zs[l - 1]))
    out = []
    for l in range(DEPTH):
        out += [grads_W[l].ravel(), grads_b[l]]
    out += [dw4, np.array([db4])]
    return loss, np.concatenate(out)
