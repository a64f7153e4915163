// Launchers of the vector, reduction, Krylov and dense-coarse-solve kernels.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

// out[0] = sum_i x[i*stride] * y[i*stride] (y == nullptr: sum of x), deterministic; sqrt_out takes sqrt.
// part: >= 592 doubles of workspace.
template <typename A, typename B>
cudaError_t launch_dot(const A* x, const B* y, long long n, long long stride, double* part, double* out, int sqrt_out,
                       cudaStream_t st);

// Chebyshev-Jacobi pieces (Saad, Iterative Methods, Alg. 12.1, with D^-1):
//  init0: r = b, d = dinv r / theta, x = d                    (zero initial guess)
//  init1: r = b - Mx, d = dinv r / theta, x += d
//  step : r -= Md, d = a d + bc dinv r, x += d
template <typename T>
cudaError_t launch_cheb_init0(long long n, const T* b, const T* dinv, T inv_theta, T* r, T* d, T* x, cudaStream_t st);
template <typename T>
cudaError_t launch_cheb_init1(long long n, const T* b, const T* mx, const T* dinv, T inv_theta, T* r, T* d, T* x,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_cheb_step(long long n, const T* md, const T* dinv, T a, T bc, T* r, T* d, T* x, cudaStream_t st);
template <typename T>
cudaError_t launch_sub(long long n, const T* a, T* r, cudaStream_t st);
template <typename T>
cudaError_t launch_axpby(long long n, T a, const T* x, T b, const T* y, T* z, cudaStream_t st);
template <typename T>
cudaError_t launch_mul(long long n, const T* a, const T* b, T* z, cudaStream_t st);
template <typename T>
cudaError_t launch_scale(long long n, T s, const T* x, T* z, cudaStream_t st);
// z = x / s[0] with the divisor read from device memory (no host round trip).
template <typename T>
cudaError_t launch_scale_by_inv(long long n, const double* s, const T* x, T* z, cudaStream_t st);
template <typename A, typename B>
cudaError_t launch_cast(long long n, const A* x, B* y, cudaStream_t st);

// dst = src with the constant-mode mean removed (Euclidean projection against 1_psi).
template <typename T>
cudaError_t launch_project_pressure(long long ne, int np, const T* src, T* dst, double* part, double* sum,
                                    cudaStream_t st);

// Coarsest-level solve: gather b through map (node -> dense index, -1 eliminated), x = Ainv b in FP64,
// neumann: b[0] pinned to 0 and the mean of x removed; scatter to x (0 on eliminated nodes).
template <typename T>
cudaError_t launch_coarse_solve(int nn, int ncomp, const int* map, int nfree_nodes, int ndense, const double* Ainv,
                                int neumann, const T* b, T* x, double* bf, double* xf, cudaStream_t st);

// In-place inverses of up to 4 SPD matrices M[z] (n[z] x n[z], row-major) by blocked Gauss-Jordan
// (32-pivot blocks, 4 launches per block for all matrices together); pin_first[z]: replace row and
// column 0 by the identity first.  pwork: 4 * 32 * 32 doubles.  flag[0] != 0 afterwards if a pivot
// was not positive (a matrix is not SPD).
cudaError_t launch_dense_inverse_batch(int count, double* const* M, const int* n, const int* pin_first,
                                       double* pwork, int* flag, cudaStream_t st);

// FGMRES: out[c] = V[c] . w for c < ncols (deterministic); w -= V^T-weighted sum; x += Z y.
cudaError_t launch_mdot(const double* V, long long ld, int ncols, const double* w, long long n, double* part,
                        double* out, cudaStream_t st);
cudaError_t launch_gemv_sub(const double* V, long long ld, int ncols, const double* h, double* w, long long n,
                            cudaStream_t st);
cudaError_t launch_gemv_add(const double* Z, long long ld, int ncols, const double* y, double* x, long long n,
                            cudaStream_t st);
cudaError_t launch_add_vec(long long n, const double* a, double* h, cudaStream_t st);
