"""CPU check of the arithmetic scheme of the FP64 Q2 row-segment element passes (q2_fp64.cu).

The kernels replace the table-driven 3-term derivative sums by constant expressions of the Q2
GLL derivative matrix D = Dt / 2, Dt = [[-3, 4, -1], [-1, 0, 1], [1, -4, 3]], fold the mesh scale
kappa = 1/h into the point weights on isotropic meshes, and assemble x-line partials per
32-element row segment (node 2m = point 0 of element m + point 2 of element m - 1) before a node
pass over the (up to 2 x 2) y/z lines and the segment seams.  This test restates that scheme in
NumPy, lane-vectorised like the kernels, and compares A, B^T, B and the fused K against the
oracle's assembled operators (Sec. 1.2).  It runs no GPU code.
"""
import numpy as np
import pytest

from oracle import mesh as M
from oracle import operators as op
from oracle import sinker
from paper_1607_03936_gb300 import inputs

SEG, LD = 32, 66
XS = (-1.0, 0.0, 1.0)   # GLL nodes of Q2 on [-1, 1]


def pt(i, j, l):
    return i + 3 * (j + 3 * l)


def slot(c, d):
    return c if c == d else (3 if c + d == 1 else (4 if c + d == 2 else 5))


def dfw(P, v0, v1, v2):
    """Row P of Dt applied to a line (the kernels' constant forms)."""
    return [4.0 * v1 - 3.0 * v0 - v2, v2 - v0, 3.0 * v2 - 4.0 * v1 + v0][P]


def dbw(P, s0, s1, s2):
    """Column P of Dt applied to a line: (-3, -1, 1), (4, 0, -4), (-1, 1, 3)."""
    return [-3.0 * s0 - s1 + s2, 4.0 * (s0 - s2), -s0 + s1 + 3.0 * s2][P]


def scheme(m, mu, u, p, ops, iso):
    nx, ny, nz = m.nx, m.ny, m.nz
    NX, NY, NZ = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
    nn = NX * NY * NZ
    h = (m.lx / nx, m.ly / ny, m.lz / nz)
    kap = [1.0 / x for x in h]
    detJ = h[0] * h[1] * h[2] / 8.0
    w1 = (1.0 / 3.0, 4.0 / 3.0, 1.0 / 3.0)
    W = [w1[q % 3] * w1[(q // 3) % 3] * w1[q // 9] * detJ for q in range(27)]
    H = [W[q] * kap[0] ** 2 if iso else W[q] for q in range(27)]
    T = [W[q] * kap[0] if iso else W[q] for q in range(27)]
    DA, DBT, DB = ops & 1, ops & 2, ops & 4
    nseg = (nx + SEG - 1) // SEG
    R = np.zeros((nseg, nz, ny, 9, 3, LD))
    Bu = np.zeros(nx * ny * nz * 4)
    uu = u.reshape(3, nn)
    bnd = np.zeros((NZ, NY, NX), bool)
    bnd[[0, -1], :, :] = bnd[:, [0, -1], :] = bnd[:, :, [0, -1]] = True
    bnd = bnd.ravel()
    for ez in range(nz):
        for ey in range(ny):
            for seg in range(nseg):
                ex = np.arange(seg * SEG, min(nx, seg * SEG + SEG))   # lanes of the segment
                nl = len(ex)
                e = ex + nx * (ey + ny * ez)
                su = np.zeros((3, 27, nl))
                mus = np.zeros((27, nl))
                for q in range(27):
                    i, j, l = q % 3, (q // 3) % 3, q // 9
                    n = (2 * ex + i) + NX * ((2 * ey + j) + NY * (2 * ez + l))
                    su[:, q] = uu[:, n] * ~bnd[n]
                    mus[q] = mu[n]
                sp = p.reshape(-1, 4)[e].T   # [4][lane]
                sS = np.zeros((6, 27, nl))
                sdiv = np.zeros((27, nl))
                for q in range(27):
                    I, J, L = q % 3, (q // 3) % 3, q // 9
                    g = np.zeros((3, 3, nl))
                    for c in range(3):
                        g[c, 0] = dfw(I, *[su[c, pt(a, J, L)] for a in range(3)])
                        g[c, 1] = dfw(J, *[su[c, pt(I, a, L)] for a in range(3)])
                        g[c, 2] = dfw(L, *[su[c, pt(I, J, a)] for a in range(3)])
                    if DB:
                        tr = g[0, 0] + g[1, 1] + g[2, 2] if iso else kap[0] * g[0, 0] + kap[1] * g[1, 1] + kap[2] * g[2, 2]
                        sdiv[q] = T[q] * tr
                    t = T[q] * (sp[0] + XS[I] * sp[1] + XS[J] * sp[2] + XS[L] * sp[3]) if DBT else 0.0
                    if DA:
                        hh = H[q] * mus[q]
                        if iso:
                            for c in range(3):
                                sS[c, q] = 2.0 * hh * g[c, c] - t
                            sS[3, q] = hh * (g[0, 1] + g[1, 0])
                            sS[4, q] = hh * (g[0, 2] + g[2, 0])
                            sS[5, q] = hh * (g[1, 2] + g[2, 1])
                        else:
                            hk = [hh * kap[d] for d in range(3)]
                            for c in range(3):
                                sS[c, q] = 2.0 * hk[c] * g[c, c] - t
                            sS[3, q] = hk[1] * g[0, 1] + hk[0] * g[1, 0]
                            sS[4, q] = hk[2] * g[0, 2] + hk[0] * g[2, 0]
                            sS[5, q] = hk[2] * g[1, 2] + hk[1] * g[2, 1]
                    elif DBT:
                        sS[0, q] = -t
                sY = np.zeros((3, 27, nl))
                for q in range(27):
                    I, J, L = q % 3, (q // 3) % 3, q // 9
                    pos = (I, J, L)
                    lines = [[pt(a, J, L) for a in range(3)], [pt(I, a, L) for a in range(3)],
                             [pt(I, J, a) for a in range(3)]]
                    for c in range(3):
                        if DA:
                            parts = [dbw(pos[d], *[sS[slot(c, d), qq] for qq in lines[d]]) for d in range(3)]
                            sY[c, q] = sum(parts) if iso else sum(kap[d] * parts[d] for d in range(3))
                        elif DBT:
                            sY[c, q] = dbw(pos[c], *[sS[0, qq] for qq in lines[c]]) * (1.0 if iso else kap[c])
                if DA or DBT:
                    last = nl - 1
                    for jl in range(9):
                        y0, y1, y2 = sY[:, 3 * jl], sY[:, 3 * jl + 1], sY[:, 3 * jl + 2]   # [c][lane]
                        row = R[seg, ez, ey, jl]
                        row[:, 1:2 * last + 2:2] = y1
                        row[:, 0:2 * last + 1:2] = y0
                        row[:, 2:2 * last + 3:2] += y2
                if DB:
                    Tl = np.stack([sdiv[3 * jl] + sdiv[3 * jl + 1] + sdiv[3 * jl + 2] for jl in range(9)])
                    Xl = np.stack([sdiv[3 * jl + 2] - sdiv[3 * jl] for jl in range(9)])
                    vals = [Tl.sum(0), Xl.sum(0), sum(Tl[2 + 3 * l] - Tl[3 * l] for l in range(3)),
                            sum(Tl[j + 6] - Tl[j] for j in range(3))]
                    for mo in range(4):
                        Bu[e * 4 + mo] = -vals[mo]
    # node pass: y/z lines through the node, x from the segment row (and the previous segment's
    # last entry at a seam)
    y = np.zeros((3, nn))
    for iz in range(NZ):
        zr = [(iz >> 1, 1)] if iz & 1 else [r for r in ([((iz >> 1) - 1, 2)] if iz > 0 else []) +
                                             ([(iz >> 1, 0)] if (iz >> 1) < nz else [])]
        for iy in range(NY):
            yr = [(iy >> 1, 1)] if iy & 1 else [r for r in ([((iy >> 1) - 1, 2)] if iy > 0 else []) +
                                                 ([(iy >> 1, 0)] if (iy >> 1) < ny else [])]
            ix = np.arange(NX)
            s, X = ix >> 6, ix & 63            # segment and entry of each node of the row
            prev = (X == 0) & (s > 0)          # a segment's first node is the previous one's last
            cur = s < nseg                     # (the mesh's last node after a full segment: prev only)
            acc = np.zeros((3, NX))
            for (zz, zl) in zr:
                for (yy, yl) in yr:
                    jl = 3 * zl + yl
                    acc[:, cur] += R[s[cur], zz, yy, jl, :, X[cur]].T
                    acc[:, prev] += R[s[prev] - 1, zz, yy, jl, :, 64].T
            n = ix + NX * (iy + NY * iz)
            y[:, n] = acc * ~bnd[n]
    return y.ravel(), Bu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("shape", [(5, 4, 3, (1.0, 0.7, 1.3)), (6, 5, 4, (1.5, 1.25, 1.0)),
                                   (33, 2, 1, (8.25, 0.5, 0.25)), (32, 1, 2, (8.0, 0.25, 0.5))])
def test_fp64_row_scheme_matches_assembled_operators(shape):
    nx, ny, nz, L = shape
    m = M.Mesh(nx, ny, nz, 2, *L)
    mu = sinker.viscosity(m.node_coords(), inputs.sinker_centres(0, 4), 0.1, 200.0, 1e4)
    rng = np.random.default_rng(1)
    u, p = rng.standard_normal(m.n_u), rng.standard_normal(m.n_p)
    A = op.assemble_A(m, op.point_values(m, mu))
    B = op.assemble_B(m)
    iso = m.lx / nx == m.ly / ny == m.lz / nz
    for ops in (1, 2, 4, 7):
        for form in ([True, False] if (iso and ops & 1) else [False]):
            yu, yp = scheme(m, mu, u, p, ops, form)
            if ops & 3:
                ref = (A @ u if ops & 1 else 0.0) + (B.T @ p if ops & 2 else 0.0)
                assert rel(yu, ref) < 1e-13, (ops, form)
            if ops & 4:
                assert rel(yp, B @ u) < 1e-13, (ops, form)
