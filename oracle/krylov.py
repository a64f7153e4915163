"""Right-preconditioned flexible GMRES(m) (Saad, SIAM J. Sci. Comput. 14, 1993).

The paper solves the preconditioned system (Eq. precond-stokes) with GMRES,
restarted every 100 iterations, to a 1e-6 relative Euclidean residual; the
flexible variant keeps z_j = P^-1 v_j so that a varying preconditioner is
allowed.  Modified Gram-Schmidt, Givens rotations, x0 = 0, convergence when
||r_j|| <= rtol ||r_0|| with r_0 the residual of the first cycle.  At every
restart the residual is recomputed as f - K x.
"""
from __future__ import annotations

import numpy as np


def fgmres(K, P, f, rtol=1e-6, restart=50, maxit=1000, x0=None, history=None):
    """Solve K x = f.  K, P: callables on float64 vectors.  Returns (x, iters, rel_res).

    rel_res is the true relative residual ||f - K x|| / ||f - K x0|| at exit.
    """
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - K(x)
    beta0 = np.linalg.norm(r)
    if beta0 == 0.0:
        return x, 0, 0.0
    its = 0
    while True:
        beta = np.linalg.norm(r)
        m = restart
        V = np.zeros((m + 1, f.size))
        Z = np.zeros((m, f.size))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        converged = False
        for j in range(m):
            Z[j] = P(V[j])
            w = K(Z[j])
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            if history is not None:
                history.append(abs(g[j + 1]) / beta0)
            if abs(g[j + 1]) <= rtol * beta0 or its >= maxit:
                converged = abs(g[j + 1]) <= rtol * beta0
                break
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        x = x + Z[:j_done].T @ y
        r = f - K(x)
        rel = np.linalg.norm(r) / beta0
        if converged and rel <= rtol:
            return x, its, rel
        if its >= maxit:
            return x, its, rel
