// The inverse-viscosity pressure mass Schur approximation (Sec. 1.3, Eq. lumping): the baseline
// the paper compares w-BFBT against (Sec. 4, Table 1).
//
//   [M_p(1/mu)]_ij = int psi_i psi_j / mu,   M~_p(1/mu) = diag(M_p(1/mu) 1_psi),
//
// 1_psi being the coefficient vector of the constant function.  The lumping is taken in the
// element basis of non-negative monomials s^a t^b u^c, s = (1 + xi)/2 (and t, u alike), a + b + c
// <= k - 1: there d'_j = int_e phi'_j / mu > 0.  (In the solver's centred basis xi^a eta^b zeta^c
// the same formula gives int_e xi / mu, which vanishes for constant mu: no usable diagonal.)  The
// solver's pressure coefficients p relate to the non-negative basis by p = T p', so the
// approximation acts on a residual r (dual, transforms by T^T) as
//
//   y = T diag(1/d') T^T r       per element,
//
// with T[m][j] = 2^-(a+b+c) C(a, a_m) C(b, b_m) C(c, c_m) (binomial expansion of s^a t^b u^c).
// Integrals use the (k+1)^3-point GLL quadrature with mu at the nodes, as everywhere else.
//
// A second variant (diag = 1) takes the diagonal of M_p(1/mu) in the centred basis instead,
// S_e = diag(1 / int_e psi_m^2 / mu): for k = 2 that basis is orthogonal under a constant
// weight, so this is the exact inverse mass wherever mu is constant on the element.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace {

__device__ inline double binom(int n, int r) {
  if (r < 0 || r > n) return 0.0;
  double v = 1.0;
  for (int i = 1; i <= r; ++i) v = v * (n - r + i) / i;
  return v;
}

// One thread per element: d'_j by quadrature, then S_e = T diag(1/d') T^T into S[e][Np][Np] (FP64);
// with diag = 1, d_m = int_e psi_m^2 / mu and S_e = diag(1/d).
__global__ void k_mass_lumped_inv(Grid g, int k, const RefTables* __restrict__ tab, const double* __restrict__ mu,
                                  int diag, double* __restrict__ S) {
  pdl_entry();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ne) return;
  const int n = k + 1, np = tab->np;
  const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
  double d[WB_MAXNP];
  for (int j = 0; j < np; ++j) d[j] = 0.0;
  for (int l = 0; l < n; ++l)
    for (int jj = 0; jj < n; ++jj)
      for (int i = 0; i < n; ++i) {
        const int node = (k * ex + i) + g.NX * ((k * ey + jj) + g.NY * (k * ez + l));
        const double wq = tab->w[i] * tab->w[jj] * tab->w[l] * g.detJ / mu[node];
        const double s = 0.5 * (1.0 + tab->x[i]), t = 0.5 * (1.0 + tab->x[jj]), u = 0.5 * (1.0 + tab->x[l]);
        for (int j = 0; j < np; ++j) {
          double v = 1.0;
          if (diag) {   // psi_j^2 at the point, centred monomials
            v = tab->pw[i][tab->ex[j][0]] * tab->pw[jj][tab->ex[j][1]] * tab->pw[l][tab->ex[j][2]];
            v *= v;
          } else {      // phi'_j, monomials of the non-negative coordinates
            for (int a = 0; a < tab->ex[j][0]; ++a) v *= s;
            for (int b = 0; b < tab->ex[j][1]; ++b) v *= t;
            for (int c = 0; c < tab->ex[j][2]; ++c) v *= u;
          }
          d[j] += wq * v;
        }
      }
  double* Se = S + (size_t)e * np * np;
  if (diag) {
    for (int m = 0; m < np; ++m)
      for (int m2 = 0; m2 < np; ++m2) Se[m * np + m2] = m == m2 ? 1.0 / d[m] : 0.0;
    return;
  }
  for (int m = 0; m < np; ++m)
    for (int m2 = 0; m2 < np; ++m2) {
      double acc = 0.0;
      for (int j = 0; j < np; ++j) {
        const int a = tab->ex[j][0], b = tab->ex[j][1], c = tab->ex[j][2];
        const double sc = 1.0 / (double)(1 << (a + b + c));
        const double t1 = sc * binom(a, tab->ex[m][0]) * binom(b, tab->ex[m][1]) * binom(c, tab->ex[m][2]);
        const double t2 = sc * binom(a, tab->ex[m2][0]) * binom(b, tab->ex[m2][1]) * binom(c, tab->ex[m2][2]);
        acc += t1 * t2 / d[j];
      }
      Se[m * np + m2] = acc;
    }
}

// y[e][m] = sum_m2 S[e][m][m2] r[e][m2]: one thread per output coefficient.
template <typename T>
__global__ void k_block_apply(long long rows, int np, const T* __restrict__ S, const T* __restrict__ r,
                              T* __restrict__ y) {
  pdl_entry();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows) return;
  const long long e = t / np;
  const int m = (int)(t % np);
  const T* Sr = S + (size_t)e * np * np + (size_t)m * np;
  const T* re = r + (size_t)e * np;
  T acc = T(0);
  for (int j = 0; j < np; ++j) acc += Sr[j] * re[j];
  y[t] = acc;
}

}  // namespace

cudaError_t launch_mass_lumped_inv(const Grid& g, int k, const RefTables* dtab, const double* mu, int diag,
                                   double* S, cudaStream_t st) {
  wb_launch(k_mass_lumped_inv, (unsigned)((g.ne + 127) / 128), 128, 0, st, g, k, dtab, mu, diag, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_block_apply(long long ne, int np, const T* S, const T* r, T* y, cudaStream_t st) {
  const long long rows = ne * np;
  wb_launch(k_block_apply<T>, (unsigned)((rows + 255) / 256), 256, 0, st, rows, np, S, r, y);
  return cudaGetLastError();
}

template cudaError_t launch_block_apply<double>(long long, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_block_apply<float>(long long, int, const float*, const float*, float*, cudaStream_t);
