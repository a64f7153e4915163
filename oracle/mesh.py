"""Structured hexahedral brick mesh with Q_k nodes (Sec. 1.2, Sec. 2.2).

Elements: e = ex + nx (ey + ny ez).  Global Q_k nodes: (k nx + 1) x (k ny + 1)
x (k nz + 1), index ix + NX (iy + NY iz).  Element-local node / quadrature
point q = i + n (j + n l), n = k + 1, sits at global node (k ex + i, k ey + j,
k ez + l).  Velocity vectors are component-major: [u_x(all nodes), u_y, u_z].
Pressure vectors are element-major: p[e * Np + m].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import gll


@dataclass
class Mesh:
    nx: int
    ny: int
    nz: int
    k: int
    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0

    def __post_init__(self):
        self.n = self.k + 1
        self.NX = self.k * self.nx + 1
        self.NY = self.k * self.ny + 1
        self.NZ = self.k * self.nz + 1
        self.n_nodes = self.NX * self.NY * self.NZ
        self.n_elem = self.nx * self.ny * self.nz
        self.Np = self.k * (self.k + 1) * (self.k + 2) // 6
        self.h = np.array([self.lx / self.nx, self.ly / self.ny, self.lz / self.nz])
        self.detJ = float(np.prod(self.h / 2.0))
        self.xi, self.w1 = gll.gll_nodes_weights(self.k)
        self.D1 = gll.derivative_matrix(self.xi)
        self.W = gll.tensor_weights(self.w1)           # (n^3,)
        self.ref_pts = gll.tensor_points(self.xi)       # (n^3, 3)

    @property
    def n_u(self) -> int:
        return 3 * self.n_nodes

    @property
    def n_p(self) -> int:
        return self.n_elem * self.Np

    def element_coords(self) -> np.ndarray:
        """(n_elem, 3) integer element coordinates (ex, ey, ez)."""
        ez, ey, ex = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx), indexing="ij")
        return np.stack([ex.ravel(), ey.ravel(), ez.ravel()], axis=-1)

    def local_ijk(self) -> np.ndarray:
        """(n^3, 3) local tensor indices (i, j, l) of point q."""
        n = self.n
        l, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        return np.stack([i.ravel(), j.ravel(), l.ravel()], axis=-1)

    def point_to_node(self) -> np.ndarray:
        """(n_elem, n^3) global node index of every element-local point."""
        ec = self.element_coords()
        lq = self.local_ijk()
        g = self.k * ec[:, None, :] + lq[None, :, :]
        return g[..., 0] + self.NX * (g[..., 1] + self.NY * g[..., 2])

    def node_coords(self) -> np.ndarray:
        """(n_nodes, 3) physical coordinates of the global GLL nodes."""
        def axis(ne, hh):
            pts = [0.0]
            for e in range(ne):
                pts.extend(e * hh + (self.xi[1:] + 1.0) * hh / 2.0)
            return np.array(pts)
        X, Y, Z = axis(self.nx, self.h[0]), axis(self.ny, self.h[1]), axis(self.nz, self.h[2])
        zz, yy, xx = np.meshgrid(Z, Y, X, indexing="ij")
        return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=-1)

    def boundary_node_mask(self) -> np.ndarray:
        """True for nodes on the boundary of the brick (Dirichlet nodes, Eq. dir-bc)."""
        iz, iy, ix = np.meshgrid(np.arange(self.NZ), np.arange(self.NY), np.arange(self.NX), indexing="ij")
        b = (ix == 0) | (ix == self.NX - 1) | (iy == 0) | (iy == self.NY - 1) | (iz == 0) | (iz == self.NZ - 1)
        return b.ravel()

    def boundary_element_mask(self) -> np.ndarray:
        """True for elements whose closure touches the boundary (the set D of Eq. bdramp)."""
        ec = self.element_coords()
        nn = np.array([self.nx, self.ny, self.nz])
        return np.any((ec == 0) | (ec == nn - 1), axis=1)

    def interior_dof_mask(self) -> np.ndarray:
        """Velocity DOF mask (3 n_nodes,), True for non-Dirichlet DOFs."""
        return np.tile(~self.boundary_node_mask(), 3)

    def coarsen(self) -> "Mesh":
        return Mesh(self.nx // 2, self.ny // 2, self.nz // 2, self.k, self.lx, self.ly, self.lz)


def table3_dof_counts(level: int, k: int) -> tuple[int, int]:
    """Velocity and pressure DOF counts of the uniform level-`level` mesh (N = 2^level).

    Velocity counts include the Dirichlet nodes, as Table 3 does.
    """
    m = Mesh(2 ** level, 2 ** level, 2 ** level, k)
    return m.n_u, m.n_p
