"""CPU oracle of the learned pressure-Poisson correction: a 3-level 3-D convolutional U-Net.

TEST INFRASTRUCTURE: plain FP64 NumPy, forward and backward written out from the definitions.
The paper has no learned component; the architecture is fixed as follows (3 levels,
16/32/64 channels, 3x3x3 kernels, per-element inputs and outputs):

  c1 (Cin -> 16), c2 (16 -> 16)                         level 0, n^3 voxels   -> skip a2
  avg-pool 2, c3 (16 -> 32), c4 (32 -> 32)              level 1, (n/2)^3      -> skip a4
  avg-pool 2, c5 (32 -> 64), c6 (64 -> 64)              level 2, (n/4)^3
  nearest-upsample 2, concat [up, a4] (96), c7 (96 -> 32), c8 (32 -> 32)
  nearest-upsample 2, concat [up, a2] (48), c9 (48 -> 16), c10 (16 -> 16)
  c11 (16 -> Cout), linear output;   ReLU after c1..c10;  zero padding.

Tensors are [D][H][W][C] (x fastest among the spatial axes, channels contiguous), voxel
(ex, ey, ez) of an n^3 element grid.  Convolution taps t = (dx+1) + 3 (dy+1) + 9 (dz+1),
weights W[t][ci][co], bias b[co]:  y[v][co] = b[co] + sum_t sum_ci W[t][ci][co] x[v + d_t][ci].
Parameters are flattened layer by layer as (W then b).  Loss: mean squared error.
"""
from __future__ import annotations

import numpy as np

LAYERS_TEMPLATE = [("c1", None, 16), ("c2", 16, 16), ("c3", 16, 32), ("c4", 32, 32), ("c5", 32, 64),
                   ("c6", 64, 64), ("c7", 96, 32), ("c8", 32, 32), ("c9", 48, 16), ("c10", 16, 16),
                   ("c11", 16, None)]


def layer_shapes(cin: int, cout: int):
    """[(name, Cin, Cout)] for an input of `cin` channels and an output of `cout` channels."""
    out = []
    for name, ci, co in LAYERS_TEMPLATE:
        out.append((name, cin if ci is None else ci, cout if co is None else co))
    return out


def n_params(cin: int, cout: int) -> int:
    return sum(27 * ci * co + co for _, ci, co in layer_shapes(cin, cout))


def unflatten(theta: np.ndarray, cin: int, cout: int):
    params, off = {}, 0
    for name, ci, co in layer_shapes(cin, cout):
        w = theta[off: off + 27 * ci * co].reshape(27, ci, co)
        off += 27 * ci * co
        b = theta[off: off + co]
        off += co
        params[name] = (w, b)
    assert off == theta.size
    return params


def flatten(grads: dict, cin: int, cout: int) -> np.ndarray:
    return np.concatenate([np.concatenate([grads[name][0].ravel(), grads[name][1].ravel()])
                           for name, _, _ in layer_shapes(cin, cout)])


def _taps():
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                yield dx, dy, dz


def _shift(x, dx, dy, dz):
    """s[z][y][x] = x[z+dz][y+dy][x+dx] with zeros outside."""
    D, H, W = x.shape[:3]
    s = np.zeros_like(x)
    zs, zd = (slice(dz, D), slice(0, D - dz)) if dz >= 0 else (slice(0, D + dz), slice(-dz, D))
    ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
    xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
    s[zd, yd, xd] = x[zs, ys, xs]
    return s


def conv3d(x, w, b):
    y = np.broadcast_to(b, x.shape[:3] + (w.shape[2],)).astype(np.float64).copy()
    for t, (dx, dy, dz) in enumerate(_taps()):
        y += _shift(x, dx, dy, dz) @ w[t]
    return y


def conv3d_backward(x, w, gy):
    """Gradients of sum(gy * conv3d(x, w, b)) w.r.t. x, w, b."""
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for t, (dx, dy, dz) in enumerate(_taps()):
        xs = _shift(x, dx, dy, dz)
        gw[t] = xs.reshape(-1, x.shape[3]).T @ gy.reshape(-1, gy.shape[3])
        gx += _shift(gy @ w[t].T, -dx, -dy, -dz)
    gb = gy.reshape(-1, gy.shape[3]).sum(axis=0)
    return gx, gw, gb


def pool(x):
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def pool_backward(gp):
    return np.repeat(np.repeat(np.repeat(gp, 2, 0), 2, 1), 2, 2) / 8.0


def upsample(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def upsample_backward(gu):
    D, H, W, C = gu.shape
    return gu.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def forward(theta, x, cin, cout):
    """Returns (y, cache).  x: [n][n][n][cin]."""
    P = unflatten(theta, cin, cout)
    c = {}

    def cr(name, inp):
        z = conv3d(inp, *P[name])
        c[name] = (inp, z)
        return np.maximum(z, 0.0)

    a1 = cr("c1", x)
    a2 = cr("c2", a1)
    a3 = cr("c3", pool(a2))
    a4 = cr("c4", a3)
    a5 = cr("c5", pool(a4))
    a6 = cr("c6", a5)
    a7 = cr("c7", np.concatenate([upsample(a6), a4], axis=3))
    a8 = cr("c8", a7)
    a9 = cr("c9", np.concatenate([upsample(a8), a2], axis=3))
    a10 = cr("c10", a9)
    y = conv3d(a10, *P["c11"])
    c["c11"] = (a10, y)
    return y, c


def loss_and_grad(theta, x, target, cin, cout):
    """MSE loss mean((y - target)^2) and its gradient w.r.t. the flat parameters."""
    P = unflatten(theta, cin, cout)
    y, c = forward(theta, x, cin, cout)
    diff = y - target
    loss = float(np.mean(diff ** 2))
    g = {}
    gy = 2.0 * diff / diff.size

    def back(name, gz, relu=True):
        inp, z = c[name]
        if relu:
            gz = gz * (z > 0)
        gx, gw, gb = conv3d_backward(inp, P[name][0], gz)
        g[name] = (gw, gb)
        return gx

    g10 = back("c11", gy, relu=False)
    g9 = back("c10", g10)
    gcat2 = back("c9", g9)
    g8 = upsample_backward(gcat2[..., :32])
    ga2 = gcat2[..., 32:]
    g7 = back("c8", g8)
    gcat1 = back("c7", g7)
    g6 = upsample_backward(gcat1[..., :64])
    ga4 = gcat1[..., 64:]
    g5 = back("c6", g6)
    ga4 = ga4 + pool_backward(back("c5", g5))
    g3 = back("c4", ga4)
    ga2 = ga2 + pool_backward(back("c3", g3))
    g1 = back("c2", ga2)
    back("c1", g1)
    return loss, flatten(g, cin, cout)


def adam_step(theta, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
