"""CPU check of the blocked symmetric Gauss-Jordan scheme of the coarsest inverses (vec_ops.cu).

The kernels invert SPD matrices in place, pivot block by pivot block (32 wide): P = inv(A_JJ),
A_JK <- P A_JK, A_IK <- A_IK - A_IJ A_JK (I, K outside J), A_IJ <- -A_IJ P, A_JJ <- P.  The
trailing update is computed only on 32 x 32 tiles on or above the tile diagonal; the tiles below
are restored from the invariant of the sweep, A[k][i] = s(i) s(k) A[i][k] with s = -1 on
indices already pivoted and +1 otherwise.  This test restates the scheme in NumPy, tile by tile
as the kernels run it, and compares with a dense inverse, including a ragged last tile and a
matrix whose first row and column are pinned to the identity (the singular Neumann Poisson
coarsest matrices).  It runs no GPU code.
"""
import numpy as np
import pytest

B = 32


def sweep(A0):
    A = A0.copy()
    n = A.shape[0]
    nt = (n + B - 1) // B
    for J0 in range(0, n, B):
        bb = min(B, n - J0)
        Jr = np.arange(J0, J0 + bb)
        P = np.linalg.inv(A[np.ix_(Jr, Jr)])
        notJ = np.r_[0:J0, J0 + bb:n]
        colJ = A[:, Jr].copy()
        A[np.ix_(Jr, notJ)] = P @ A[np.ix_(Jr, notJ)]
        for it in range(nt):
            for kt in range(it, nt):      # tiles on or above the diagonal
                I = np.arange(it * B, min(n, it * B + B))
                K = np.arange(kt * B, min(n, kt * B + B))
                I = I[(I < J0) | (I >= J0 + bb)]
                K = K[(K < J0) | (K >= J0 + bb)]
                if len(I) and len(K):
                    A[np.ix_(I, K)] -= colJ[I] @ A[np.ix_(Jr, K)]
        for it in range(nt):
            for kt in range(it):          # tiles below: mirrored with the sign pattern
                i0, k0 = it * B, kt * B
                if J0 <= i0 < J0 + bb or J0 <= k0 < J0 + bb:
                    continue
                I = np.arange(i0, min(n, i0 + B))
                K = np.arange(k0, min(n, k0 + B))
                sg = np.where((I[:, None] < J0) != (K[None, :] < J0), -1.0, 1.0)
                A[np.ix_(I, K)] = sg * A[np.ix_(K, I)].T
        A[np.ix_(notJ, Jr)] = -colJ[notJ] @ P
        A[np.ix_(Jr, Jr)] = P
    return A


@pytest.mark.parametrize("n,pin", [(64, False), (100, False), (129, True)])
def test_symmetric_sweep_inverts_spd(n, pin):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    if pin:
        A[0, :] = 0.0
        A[:, 0] = 0.0
        A[0, 0] = 1.0
    X = sweep(A)
    ref = np.linalg.inv(A)
    assert np.abs(X - ref).max() / np.abs(ref).max() < 1e-13
    assert np.abs(X - X.T).max() / np.abs(ref).max() < 1e-13
