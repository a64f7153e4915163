"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic (no viscosity formula, no operator, no solver step).

The multi-sinker benchmark of Sec. 2.1 places n sinkers at "precomputed random
points" that the paper does not publish, so seeded stand-ins are drawn here:
SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) turned into 53-bit uniforms u in [0, 1), mapped to
c = lo + (hi - lo) * u, drawn in the order sinker i, then x, y, z.
"""
from __future__ import annotations

import numpy as np

_MASK64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64_stream(seed: int, count: int) -> list[int]:
    """Return the first `count` 64-bit outputs of SplitMix64 seeded with `seed`."""
    state = seed & _MASK64
    out = []
    for _ in range(count):
        state = (state + _GOLDEN) & _MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        out.append(z ^ (z >> 31))
    return out


def uniform01(seed: int, count: int) -> np.ndarray:
    """`count` doubles in [0, 1) from the top 53 bits of SplitMix64 outputs."""
    vals = splitmix64_stream(seed, count)
    return np.array([(v >> 11) * (1.0 / (1 << 53)) for v in vals], dtype=np.float64)


def sinker_centres(seed: int, n_sinkers: int, lo: float = 0.1, hi: float = 0.9) -> np.ndarray:
    """Sinker centres c_i, shape (n_sinkers, 3), uniform in [lo, hi]^3 (Sec. 2.1 stand-in)."""
    u = uniform01(seed, 3 * n_sinkers).reshape(n_sinkers, 3)
    return lo + (hi - lo) * u


def normal_vector(seed: int, size: int) -> np.ndarray:
    """Standard-normal float64 vector of length `size` (a seeded numpy Generator)."""
    return np.random.default_rng(seed).standard_normal(size)


def uniform_vector(seed: int, size: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform float64 vector of length `size` in [lo, hi) (a seeded numpy Generator)."""
    return np.random.default_rng(seed).uniform(lo, hi, size)


def unet_init_params(seed: int, cin: int, cout: int, scale: float = 1.0) -> np.ndarray:
    """He-normal initial U-Net parameters (weights N(0, 2 / (27 cin)), biases 0), flat float32.

    Layer order and shapes follow the parameter layout of the learned correction
    (c1..c11, W[27][cin][cout] then b[cout]).
    """
    chans = [(cin, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (96, 32), (32, 32), (48, 16),
             (16, 16), (16, cout)]
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in chans:
        parts.append(rng.standard_normal(27 * ci * co) * np.sqrt(2.0 / (27 * ci)) * scale)
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


# Workload definitions: the multi-sinker problems of Sec. 2.1 at the sizes the
# tests and the bench run.  omega is the sinker diameter, delta the Gaussian
# decay, dr the dynamic ratio max(mu)/min(mu).
WORKLOADS = {
    "8^3-Q2-S4-DR1e4": dict(n=8, k=2, n_sinkers=4, omega=0.1, delta=200.0, dr=1e4, seed=0),
    "32^3-Q2-S24-DR1e6": dict(n=32, k=2, n_sinkers=24, omega=0.05, delta=200.0, dr=1e6, seed=0),
    "24^3-Q3-S32-DR1e8": dict(n=24, k=3, n_sinkers=32, omega=0.1, delta=200.0, dr=1e8, seed=0),
    "64^3-Q2-S64-DR1e10": dict(n=64, k=2, n_sinkers=64, omega=0.04, delta=400.0, dr=1e10, seed=0),
    # the size of Table 3a's refinement level 7 (59.3M DOF) with its S16, DR 1e6 problem
    "128^3-Q2-S16-DR1e6": dict(n=128, k=2, n_sinkers=16, omega=0.1, delta=200.0, dr=1e6, seed=0),
}


# Mapped (non-affine) hexahedral meshes.  Both generators move the nodes of a brick mesh: they take
# the brick's nodal coordinates X0 (n_nodes, 3) and return the moved coordinates, which then define
# each element's isoparametric map.  Nodes on the brick's faces stay where they are, so the domain
# stays the brick.

def deform_vertices(X0: np.ndarray, n_el: tuple[int, int, int], lengths: tuple[float, float, float],
                    amp: float, seed: int) -> np.ndarray:
    """Straight-edged, non-affine elements: every interior element vertex moves by a seeded uniform
    offset in [-amp, amp] h per axis (vertices on the boundary stay), and every node moves by the
    trilinear interpolant of its brick element's vertex offsets.  amp < 1/6 keeps det J > 0
    everywhere: every entry of (2/h) J - I is an average of edge-offset differences, at most 2 amp
    in magnitude, so its norm stays below 1."""
    nx, ny, nz = n_el
    h = np.array(lengths, dtype=np.float64) / np.array([nx, ny, nz])
    rng = np.random.default_rng(seed)
    off = rng.uniform(-amp, amp, size=(nz + 1, ny + 1, nx + 1, 3)) * h
    off[0, :, :] = off[-1, :, :] = 0.0
    off[:, 0, :] = off[:, -1, :] = 0.0
    off[:, :, 0] = off[:, :, -1] = 0.0
    t = X0 / h                                           # brick coordinates in element units
    e = np.minimum(np.floor(t + 1e-12).astype(np.int64), np.array([nx, ny, nz]) - 1)
    s = np.clip(t - e, 0.0, 1.0)
    out = X0.astype(np.float64).copy()
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                wgt = ((s[:, 0] if cx else 1 - s[:, 0]) * (s[:, 1] if cy else 1 - s[:, 1])
                       * (s[:, 2] if cz else 1 - s[:, 2]))
                out += wgt[:, None] * off[e[:, 2] + cz, e[:, 1] + cy, e[:, 0] + cx]
    return out


def deform_smooth(X0: np.ndarray, lengths: tuple[float, float, float], amp: float) -> np.ndarray:
    """Curved elements: x -> x + amp L b(x) v, b(x) = prod_d sin(pi x_d / L_d), v = (1, -1, 1) / 2
    scaled per axis by L_d; b vanishes on the boundary.  The Jacobian of the move is I plus a rank-one
    term, det = 1 + amp L v . grad b >= 1 - 1.5 pi amp, so amp < 0.2 keeps it positive."""
    L = np.array(lengths, dtype=np.float64)
    b = np.prod(np.sin(np.pi * X0 / L), axis=1)
    return X0 + amp * b[:, None] * (L * np.array([0.5, -0.5, 0.5]))[None, :]
