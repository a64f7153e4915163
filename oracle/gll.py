"""1-D reference-element tables for the Q_k x P_{k-1}^disc pair (Sec. 1.2).

The paper fixes a continuous nodal Q_k velocity and a discontinuous modal
P_{k-1} pressure but not the nodes, quadrature or modal basis.  The readings
used here: Gauss-Lobatto-Legendre (GLL) nodes, (k+1)-point GLL collocated
quadrature, and monomials xi^a eta^b zeta^c (a+b+c <= k-1) ordered by total
degree and then lexicographically descending in (a, b, c).
"""
from __future__ import annotations

import itertools

import numpy as np
from numpy.polynomial import Polynomial
from numpy.polynomial.legendre import Legendre


def gll_nodes_weights(k: int) -> tuple[np.ndarray, np.ndarray]:
    """GLL nodes and weights on [-1, 1] with k+1 points.

    Nodes: -1, the roots of P_k', +1.  Weights: 2 / (k (k+1) P_k(x_i)^2).
    The roots are polished with Newton steps on P_k'.
    """
    if k < 1:
        raise ValueError("k >= 1 required")
    pk = Legendre.basis(k)
    dpk = pk.deriv()
    d2pk = dpk.deriv()
    inner = np.sort(dpk.roots().real) if k > 1 else np.zeros(0)
    for _ in range(5):
        inner = inner - dpk(inner) / d2pk(inner)
    x = np.concatenate([[-1.0], inner, [1.0]])
    w = 2.0 / (k * (k + 1) * pk(x) ** 2)
    return x, w


def lagrange_polys(x: np.ndarray) -> list[Polynomial]:
    """Lagrange basis polynomials l_j with l_j(x_i) = delta_ij."""
    polys = []
    for j in range(len(x)):
        p = Polynomial([1.0])
        for m in range(len(x)):
            if m != j:
                p = p * Polynomial([-x[m], 1.0]) / (x[j] - x[m])
        polys.append(p)
    return polys


def lagrange_eval(x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Matrix L[s, j] = l_j(t_s) of the Lagrange basis on nodes x."""
    polys = lagrange_polys(x)
    t = np.asarray(t, dtype=np.float64)
    return np.stack([p(t) for p in polys], axis=-1)


def derivative_matrix(x: np.ndarray) -> np.ndarray:
    """D[i, j] = l_j'(x_i): derivative at node i of the j-th Lagrange polynomial."""
    polys = lagrange_polys(x)
    return np.stack([p.deriv()(x) for p in polys], axis=-1)


def pressure_exponents(k: int) -> list[tuple[int, int, int]]:
    """Exponents (a, b, c) of the P_{k-1} monomials, a+b+c <= k-1.

    Ordered by total degree, then lexicographically descending.  The count is
    k(k+1)(k+2)/6, the per-element pressure DOF count behind Table 3.
    """
    out = []
    for deg in range(k):
        same = [t for t in itertools.product(range(deg + 1), repeat=3) if sum(t) == deg]
        out.extend(sorted(same, reverse=True))
    return out


def pressure_basis_at_points(k: int, pts: np.ndarray) -> np.ndarray:
    """Psi[q, m] = psi_m(pts[q]) for reference points pts of shape (nq, 3)."""
    ex = pressure_exponents(k)
    pts = np.asarray(pts, dtype=np.float64)
    return np.stack([pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c for (a, b, c) in ex], axis=-1)


def tensor_points(x: np.ndarray) -> np.ndarray:
    """Reference points of the tensor grid x^3, index q = i + n (j + n l)."""
    n = len(x)
    l, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.stack([x[i.ravel()], x[j.ravel()], x[l.ravel()]], axis=-1)


def tensor_weights(w: np.ndarray) -> np.ndarray:
    """Tensor-product weights W[q] = w_i w_j w_l, index q = i + n (j + n l)."""
    return np.einsum("l,j,i->lji", w, w, w).ravel()
