// Vector kernels of the solver: deterministic reductions, Chebyshev-Jacobi updates,
// projections, casts, FGMRES Gram-Schmidt kernels, and the FP64 dense coarsest
// solve (blocked Gauss-Jordan explicit inverse at setup, GEMV per V-cycle).
//
// Reductions are two-stage with a grid that depends only on the vector length and
// a fixed tree inside each block, so repeated runs give bitwise-identical sums.
#include "vec_ops.h"

namespace {

constexpr int RB = 256;          // reduction block size
constexpr int RMAX = 592;        // max partial blocks (4 x 148-SM-multiple, also 152 x 4 = 608 is close)

inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

__device__ inline double block_sum(double v) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = threadIdx.x < nw ? sh[threadIdx.x] : 0.0;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;  // valid in thread 0
}

template <typename A, typename B>
__global__ void k_dot_partial(const A* __restrict__ x, const B* __restrict__ y, long long n, long long stride,
                              double* __restrict__ part) {
  pdl_entry();
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double a = (double)x[i * stride];
    acc += y ? a * (double)y[i * stride] : a;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_final(const double* __restrict__ part, int np, int ncols, double* __restrict__ out, int sqrt_out) {
  pdl_entry();
  // one block per column; partials of column c at part[c * np + b]
  double acc = 0.0;
  for (int b = threadIdx.x; b < np; b += blockDim.x) acc += part[(size_t)blockIdx.x * np + b];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[blockIdx.x] = sqrt_out ? sqrt(acc) : acc;
}

// Partial blocks of a single dot product: about 3300 entries per block (measured best on GB300
// between 0.96M and 7.5M entries), at most RMAX.
int dot_blocks(long long n) {
  long long b = (n + 3299) / 3300;
  const long long cap = (n + RB - 1) / RB;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : (b > RMAX ? RMAX : b));
}

// Blocks per column of the multi-column dot V^T w: about 4864 blocks in total (measured best for
// 25 columns of 0.96M and 7.5M entries), at most RMAX and at most one per 256 entries.
int mdot_blocks(long long n, int ncols) {
  long long b = 4864 / (ncols > 0 ? ncols : 1);
  const long long cap = (n + RB - 1) / RB;
  if (b > cap) b = cap;
  return (int)(b < 16 ? (cap < 16 ? cap : 16) : (b > RMAX ? RMAX : b));
}

template <typename T>
__global__ void k_cheb_init0(long long n, const T* __restrict__ b, const T* __restrict__ dinv, T inv_theta,
                             T* __restrict__ r, T* __restrict__ d, T* __restrict__ x) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T rv = b[i];
  const T dv = dinv[i] * rv * inv_theta;
  r[i] = rv;
  d[i] = dv;
  x[i] = dv;
}

template <typename T>
__global__ void k_cheb_init1(long long n, const T* __restrict__ b, const T* __restrict__ mx, const T* __restrict__ dinv,
                             T inv_theta, T* __restrict__ r, T* __restrict__ d, T* __restrict__ x) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T rv = b[i] - mx[i];
  const T dv = dinv[i] * rv * inv_theta;
  r[i] = rv;
  d[i] = dv;
  x[i] += dv;
}

template <typename T>
__global__ void k_cheb_step(long long n, const T* __restrict__ md, const T* __restrict__ dinv, T a, T bc,
                            T* __restrict__ r, T* __restrict__ d, T* __restrict__ x) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T rv = r[i] - md[i];
  const T dv = a * d[i] + bc * (dinv[i] * rv);
  r[i] = rv;
  d[i] = dv;
  x[i] += dv;
}

template <typename T>
__global__ void k_sub(long long n, const T* __restrict__ a, T* __restrict__ r) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] -= a[i];
}

template <typename T>
__global__ void k_axpby(long long n, T a, const T* __restrict__ x, T b, const T* __restrict__ y, T* __restrict__ z) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = a * x[i] + b * y[i];
}

template <typename T>
__global__ void k_mul(long long n, const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ z) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = a[i] * b[i];
}

template <typename T>
__global__ void k_scale(long long n, T s, const T* __restrict__ x, T* __restrict__ z) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = x[i] * s;
}

template <typename T>
__global__ void k_scale_by_inv(long long n, const double* __restrict__ s, const T* __restrict__ x, T* __restrict__ z) {
  pdl_entry();
  __shared__ double inv;   // one FP64 reciprocal per block
  if (threadIdx.x == 0) inv = 1.0 / s[0];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = T((double)x[i] * inv);
}

template <typename A, typename B>
__global__ void k_cast(long long n, const A* __restrict__ x, B* __restrict__ y) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (B)x[i];
}

// p[e * np] -= sum / count, sum from device memory (the constant-mode total)
template <typename T>
__global__ void k_sub_const_mode(long long count, int np, const double* __restrict__ sum, T* __restrict__ p) {
  pdl_entry();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) p[e * np] = T((double)p[e * np] - sum[0] / (double)count);
}

template <typename T>
__global__ void k_copy_proj(long long count, int np, const double* __restrict__ sum, const T* __restrict__ src,
                            T* __restrict__ dst) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count * np) return;
  T v = src[i];
  if (i % np == 0) v = T((double)v - sum[0] / (double)count);
  dst[i] = v;
}

// ---------------------------------------------------------------- coarse dense solve

template <typename T>
__global__ void k_coarse_gather(int nn, int ncomp, const int* __restrict__ map, int nfree, const T* __restrict__ b,
                                double* __restrict__ bf, int pin0) {
  pdl_entry();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int m = map[n];
  if (m < 0) return;
  for (int c = 0; c < ncomp; ++c) {
    const int idx = c * nfree + m;
    bf[idx] = (pin0 && idx == 0) ? 0.0 : (double)b[(size_t)c * nn + n];
  }
}

// xf = Ainv bf, one warp per row
__global__ void k_gemv_rows(const double* __restrict__ Ainv, int n, const double* __restrict__ bf,
                            double* __restrict__ xf) {
  pdl_entry();
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = Ainv + (size_t)row * n;
  double acc = 0.0;
  for (int c = lane; c < n; c += 32) acc += a[c] * bf[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) xf[row] = acc;
}

// single block: xf -= mean(xf)
__global__ void k_sub_mean_small(int n, double* __restrict__ xf) {
  pdl_entry();
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += xf[i];
  acc = block_sum(acc);
  __shared__ double mean;
  if (threadIdx.x == 0) mean = acc / n;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) xf[i] -= mean;
}

template <typename T>
__global__ void k_coarse_scatter(int nn, int ncomp, const int* __restrict__ map, int nfree, const double* __restrict__ xf,
                                 T* __restrict__ x) {
  pdl_entry();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int m = map[n];
  for (int c = 0; c < ncomp; ++c) x[(size_t)c * nn + n] = m < 0 ? T(0) : T(xf[c * nfree + m]);
}

__global__ void k_pin_first(double* M, int n) {
  pdl_entry();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  M[t] = t == 0 ? 1.0 : 0.0;            // row 0
  M[(size_t)t * n] = t == 0 ? 1.0 : 0.0; // column 0
}

// Blocked in-place Gauss-Jordan inversion of SPD matrices (no pivoting; every pivot block is a
// Schur complement of an SPD matrix, hence SPD).  For the pivot block J = [J0, J0 + bb):
//   P     <- inv(A[J][J])                       (one block per matrix, GJ in shared memory)
//   A[J][K] <- P A[J][K]              (K not in J)
//   A[I][K] <- A[I][K] - A[I][J] A[J][K]   (I, K not in J; A[J][K] already updated)
//   A[I][J] <- -A[I][J] P            (I not in J);   A[J][J] <- P
// After the last block A holds inv(A).  Several matrices run in one launch (grid.z / grid.x).
constexpr int GJB = 32;

struct GjJobs {
  double* A[4];
  int n[4];
  double* P[4];   // GJB x GJB workspace per matrix
};

__global__ void k_bgj_pivot(GjJobs jobs, int J0, int* __restrict__ flag) {
  pdl_entry();
  const int z = blockIdx.x;
  const int n = jobs.n[z];
  if (J0 >= n) return;
  const int bb = min(GJB, n - J0);
  double* A = jobs.A[z];
  __shared__ double S[GJB][GJB + 1];
  __shared__ double rowp[GJB], colj[GJB], s_ip;
  __shared__ int s_ok;
  const int r = threadIdx.y, c = threadIdx.x;   // 32 x 32 threads
  if (r < bb && c < bb) S[r][c] = A[(size_t)(J0 + r) * n + J0 + c];
  __syncthreads();
  for (int j = 0; j < bb; ++j) {
    // one reciprocal per step, the scaled pivot row and the pivot column shared by all threads
    if (r == 0 && c == 0) {
      const double p = S[j][j];
      if (!(p > 0.0) || !isfinite(p)) flag[0] = J0 + j + 1;
      s_ok = p > 0.0;
      s_ip = s_ok ? 1.0 / p : 0.0;
    }
    __syncthreads();
    if (!s_ok) return;   // uniform across the block
    const double ip = s_ip;
    if (r == 0 && c < bb) rowp[c] = S[j][c] * ip;
    if (r == 1 && c < bb) colj[c] = S[c][j];
    __syncthreads();
    if (r < bb && c < bb) {
      if (r != j && c != j) S[r][c] -= colj[r] * rowp[c];
      else if (r == j && c != j) S[r][c] = rowp[c];
      else if (r != j && c == j) S[r][c] = -colj[r] * ip;
      else S[r][c] = ip;
    }
    __syncthreads();
  }
  if (r < bb && c < bb) jobs.P[z][r * GJB + c] = S[r][c];
}

// A[J][k] <- P A[J][k] for k not in J.  Block (32 columns, 8 row groups): every thread of a column
// reads the column's pivot rows, the block synchronises, then each writes 4 of the rows.
__global__ void k_bgj_rows(GjJobs jobs, int J0) {
  pdl_entry();
  const int z = blockIdx.y;
  const int n = jobs.n[z];
  if (J0 >= n) return;
  const int bb = min(GJB, n - J0);
  const int k = blockIdx.x * 32 + threadIdx.x;
  __shared__ double P[GJB * GJB];
  for (int t = threadIdx.y * 32 + threadIdx.x; t < GJB * GJB; t += 256) P[t] = jobs.P[z][t];
  double* A = jobs.A[z];
  const bool valid = k < n && !(k >= J0 && k < J0 + bb);
  double col[GJB];
#pragma unroll
  for (int s = 0; s < GJB; ++s) col[s] = (valid && s < bb) ? A[(size_t)(J0 + s) * n + k] : 0.0;
  __syncthreads();   // every read of the column precedes any write to it
  if (!valid) return;
#pragma unroll
  for (int t = 0; t < GJB / 8; ++t) {
    const int r = threadIdx.y + 8 * t;
    if (r >= bb) continue;
    double v = 0.0;
#pragma unroll
    for (int s = 0; s < GJB; ++s) v += P[r * GJB + s] * col[s];
    A[(size_t)(J0 + r) * n + k] = v;
  }
}

// A[i][k] -= sum_s A[i][J0+s] A[J0+s][k] for i, k not in J (32 x 8 threads, 32 x 32 tile), on
// the tiles on or above the tile diagonal only.  Symmetry: at every stage of the sweep
// A[k][i] = s(i) s(k) A[i][k] with s = -1 for indices already pivoted and +1 otherwise (the
// pivoted part holds the inverse of its leading block, the cross blocks P A and -A P), and the
// update keeps that relation; k_bgj_mirror restores the tiles below the diagonal from it, so
// the FP64 work of the trailing update is halved.
__global__ void k_bgj_update(GjJobs jobs, int J0) {
  pdl_entry();
  const int z = blockIdx.z;
  const int n = jobs.n[z];
  if (J0 >= n) return;
  const int bb = min(GJB, n - J0);
  double* A = jobs.A[z];
  const int k0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  if (k0 >= n || i0 >= n || i0 > k0) return;
  __shared__ double Rj[GJB][33];   // A[J0+s][k0+x]
  __shared__ double Ci[32][GJB + 1];   // A[i0+y][J0+s]
  for (int t = threadIdx.y * 32 + threadIdx.x; t < GJB * 32; t += 256) {
    const int s = t / 32, x = t % 32;
    Rj[s][x] = (s < bb && k0 + x < n) ? A[(size_t)(J0 + s) * n + k0 + x] : 0.0;
    const int y = t / GJB, s2 = t % GJB;
    Ci[y][s2] = (s2 < bb && i0 + y < n) ? A[(size_t)(i0 + y) * n + J0 + s2] : 0.0;
  }
  __syncthreads();
  const int k = k0 + threadIdx.x;
  if (k >= n || (k >= J0 && k < J0 + bb)) return;
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int i = i0 + yy;
    if (i >= n || (i >= J0 && i < J0 + bb)) continue;
    double acc = 0.0;
#pragma unroll
    for (int s = 0; s < GJB; ++s) acc += Ci[yy][s] * Rj[s][threadIdx.x];
    A[(size_t)i * n + k] -= acc;
  }
}

// Tiles below the diagonal (i0 > k0, neither in J) from their transposes after the update:
// A[i][k] = s(i) s(k) A[k][i], s(x) = -1 for x < J0 (pivoted before this block), else +1.
__global__ void k_bgj_mirror(GjJobs jobs, int J0) {
  pdl_entry();
  const int z = blockIdx.z;
  const int n = jobs.n[z];
  if (J0 >= n) return;
  const int bb = min(GJB, n - J0);
  double* A = jobs.A[z];
  const int k0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  if (k0 >= n || i0 >= n || i0 <= k0 || (i0 >= J0 && i0 < J0 + bb) || (k0 >= J0 && k0 < J0 + bb)) return;
  __shared__ double T[32][33];
  // T[x][y] = A[k0 + x][i0 + y] (coalesced reads along y)
  for (int x = threadIdx.y; x < 32; x += 8) {
    const int k = k0 + x, i = i0 + threadIdx.x;
    T[x][threadIdx.x] = (k < n && i < n) ? A[(size_t)k * n + i] : 0.0;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int i = i0 + y, k = k0 + threadIdx.x;
    if (i < n && k < n) {
      const double sg = ((i < J0) != (k < J0)) ? -1.0 : 1.0;
      A[(size_t)i * n + k] = sg * T[threadIdx.x][y];
    }
  }
}

// A[i][J] <- -A[i][J] P for i not in J; A[J][J] <- P.  Block (32 rows, 8 column groups): every
// thread of a row reads the row's pivot columns, the block synchronises, then each writes 4.
__global__ void k_bgj_cols(GjJobs jobs, int J0) {
  pdl_entry();
  const int z = blockIdx.y;
  const int n = jobs.n[z];
  if (J0 >= n) return;
  const int bb = min(GJB, n - J0);
  double* A = jobs.A[z];
  __shared__ double P[GJB * GJB];
  for (int t = threadIdx.y * 32 + threadIdx.x; t < GJB * GJB; t += 256) P[t] = jobs.P[z][t];
  const int i = blockIdx.x * 32 + threadIdx.x;
  const bool in_range = i < n;
  const bool pivot_row = in_range && i >= J0 && i < J0 + bb;
  double* row = A + (size_t)(in_range ? i : 0) * n + J0;
  double a[GJB];
#pragma unroll
  for (int s = 0; s < GJB; ++s) a[s] = (in_range && !pivot_row && s < bb) ? row[s] : 0.0;
  __syncthreads();   // P is loaded and every read of the row precedes any write to it
  if (!in_range) return;
#pragma unroll
  for (int t = 0; t < GJB / 8; ++t) {
    const int cc = threadIdx.y + 8 * t;
    if (cc >= bb) continue;
    if (pivot_row) {
      row[cc] = P[(i - J0) * GJB + cc];
      continue;
    }
    double v = 0.0;
#pragma unroll
    for (int s = 0; s < GJB; ++s) v += a[s] * P[s * GJB + cc];
    row[cc] = -v;
  }
}

// ---------------------------------------------------------------- FGMRES (FP64)

__global__ void k_mdot_partial(const double* __restrict__ V, long long ld, const double* __restrict__ w, long long n,
                               int np, double* __restrict__ part) {
  pdl_entry();
  const double* v = V + (size_t)blockIdx.y * ld;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)np * blockDim.x)
    acc += v[i] * w[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * np + blockIdx.x] = acc;
}

__global__ void k_gemv_sub(const double* __restrict__ V, long long ld, int ncols, const double* __restrict__ h,
                           double* __restrict__ w, long long n) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = w[i];
  for (int c = 0; c < ncols; ++c) acc -= h[c] * V[(size_t)c * ld + i];
  w[i] = acc;
}

__global__ void k_gemv_add(const double* __restrict__ Z, long long ld, int ncols, const double* __restrict__ y,
                           double* __restrict__ x, long long n) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = x[i];
  for (int c = 0; c < ncols; ++c) acc += y[c] * Z[(size_t)c * ld + i];
  x[i] = acc;
}

__global__ void k_add2(long long n, const double* __restrict__ a, double* __restrict__ h) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) h[i] += a[i];
}

}  // namespace

// ================================================================== launchers

template <typename A, typename B>
cudaError_t launch_dot(const A* x, const B* y, long long n, long long stride, double* part, double* out, int sqrt_out,
                       cudaStream_t st) {
  const int np = dot_blocks(n);
  wb_launch(k_dot_partial<A, B>, np, RB, 0, st, x, y, n, stride, part);
  wb_launch(k_final, 1, RB, 0, st, part, np, 1, out, sqrt_out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cheb_init0(long long n, const T* b, const T* dinv, T inv_theta, T* r, T* d, T* x, cudaStream_t st) {
  wb_launch(k_cheb_init0<T>, nblk(n, 256), 256, 0, st, n, b, dinv, inv_theta, r, d, x);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cheb_init1(long long n, const T* b, const T* mx, const T* dinv, T inv_theta, T* r, T* d, T* x,
                              cudaStream_t st) {
  wb_launch(k_cheb_init1<T>, nblk(n, 256), 256, 0, st, n, b, mx, dinv, inv_theta, r, d, x);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cheb_step(long long n, const T* md, const T* dinv, T a, T bc, T* r, T* d, T* x, cudaStream_t st) {
  wb_launch(k_cheb_step<T>, nblk(n, 256), 256, 0, st, n, md, dinv, a, bc, r, d, x);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_sub(long long n, const T* a, T* r, cudaStream_t st) {
  wb_launch(k_sub<T>, nblk(n, 256), 256, 0, st, n, a, r);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_axpby(long long n, T a, const T* x, T b, const T* y, T* z, cudaStream_t st) {
  wb_launch(k_axpby<T>, nblk(n, 256), 256, 0, st, n, a, x, b, y, z);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_mul(long long n, const T* a, const T* b, T* z, cudaStream_t st) {
  wb_launch(k_mul<T>, nblk(n, 256), 256, 0, st, n, a, b, z);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_scale(long long n, T s, const T* x, T* z, cudaStream_t st) {
  wb_launch(k_scale<T>, nblk(n, 256), 256, 0, st, n, s, x, z);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_scale_by_inv(long long n, const double* s, const T* x, T* z, cudaStream_t st) {
  wb_launch(k_scale_by_inv<T>, nblk(n, 256), 256, 0, st, n, s, x, z);
  return cudaGetLastError();
}

template <typename A, typename B>
cudaError_t launch_cast(long long n, const A* x, B* y, cudaStream_t st) {
  wb_launch(k_cast<A, B>, nblk(n, 256), 256, 0, st, n, x, y);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_project_pressure(long long ne, int np, const T* src, T* dst, double* part, double* sum,
                                    cudaStream_t st) {
  cudaError_t e = launch_dot<T, T>(src, (const T*)nullptr, ne, np, part, sum, 0, st);
  if (e != cudaSuccess) return e;
  wb_launch(k_copy_proj<T>, nblk(ne * np, 256), 256, 0, st, ne, np, sum, src, dst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve(int nn, int ncomp, const int* map, int nfree_nodes, int ndense, const double* Ainv,
                                int neumann, const T* b, T* x, double* bf, double* xf, cudaStream_t st) {
  wb_launch(k_coarse_gather<T>, nblk(nn, 256), 256, 0, st, nn, ncomp, map, nfree_nodes, b, bf, neumann);
  wb_launch(k_gemv_rows, nblk((long long)ndense * 32, 256), 256, 0, st, Ainv, ndense, bf, xf);
  if (neumann) wb_launch(k_sub_mean_small, 1, 1024, 0, st, ndense, xf);
  wb_launch(k_coarse_scatter<T>, nblk(nn, 256), 256, 0, st, nn, ncomp, map, nfree_nodes, xf, x);
  return cudaGetLastError();
}

cudaError_t launch_dense_inverse_batch(int count, double* const* M, const int* n, const int* pin_first,
                                       double* pwork, int* flag, cudaStream_t st) {
  if (count < 1 || count > 4) return cudaErrorInvalidValue;
  GjJobs jobs{};
  int nmax = 0;
  for (int z = 0; z < count; ++z) {
    jobs.A[z] = M[z];
    jobs.n[z] = n[z];
    jobs.P[z] = pwork + (size_t)z * GJB * GJB;
    if (n[z] > nmax) nmax = n[z];
    if (pin_first[z]) wb_launch(k_pin_first, nblk(n[z], 256), 256, 0, st, M[z], n[z]);
  }
  for (int J0 = 0; J0 < nmax; J0 += GJB) {
    wb_launch(k_bgj_pivot, count, dim3(32, 32), 0, st, jobs, J0, flag);
    wb_launch(k_bgj_rows, dim3((nmax + 31) / 32, count), dim3(32, 8), 0, st, jobs, J0);
    wb_launch(k_bgj_update, dim3((nmax + 31) / 32, (nmax + 31) / 32, count), dim3(32, 8), 0, st, jobs, J0);
    wb_launch(k_bgj_mirror, dim3((nmax + 31) / 32, (nmax + 31) / 32, count), dim3(32, 8), 0, st, jobs, J0);
    wb_launch(k_bgj_cols, dim3((nmax + 31) / 32, count), dim3(32, 8), 0, st, jobs, J0);
  }
  return cudaGetLastError();
}

cudaError_t launch_mdot(const double* V, long long ld, int ncols, const double* w, long long n, double* part,
                        double* out, cudaStream_t st) {
  const int np = mdot_blocks(n, ncols);
  wb_launch(k_mdot_partial, dim3(np, ncols), RB, 0, st, V, ld, w, n, np, part);
  wb_launch(k_final, ncols, RB, 0, st, part, np, ncols, out, 0);
  return cudaGetLastError();
}

cudaError_t launch_gemv_sub(const double* V, long long ld, int ncols, const double* h, double* w, long long n,
                            cudaStream_t st) {
  wb_launch(k_gemv_sub, nblk(n, 256), 256, 0, st, V, ld, ncols, h, w, n);
  return cudaGetLastError();
}

cudaError_t launch_gemv_add(const double* Z, long long ld, int ncols, const double* y, double* x, long long n,
                            cudaStream_t st) {
  wb_launch(k_gemv_add, nblk(n, 256), 256, 0, st, Z, ld, ncols, y, x, n);
  return cudaGetLastError();
}

cudaError_t launch_add_vec(long long n, const double* a, double* h, cudaStream_t st) {
  wb_launch(k_add2, nblk(n, 256), 256, 0, st, n, a, h);
  return cudaGetLastError();
}

#define WB_VINST(T)                                                                                                   \
  template cudaError_t launch_cheb_init0<T>(long long, const T*, const T*, T, T*, T*, T*, cudaStream_t);              \
  template cudaError_t launch_cheb_init1<T>(long long, const T*, const T*, const T*, T, T*, T*, T*, cudaStream_t);    \
  template cudaError_t launch_cheb_step<T>(long long, const T*, const T*, T, T, T*, T*, T*, cudaStream_t);            \
  template cudaError_t launch_sub<T>(long long, const T*, T*, cudaStream_t);                                          \
  template cudaError_t launch_axpby<T>(long long, T, const T*, T, const T*, T*, cudaStream_t);                        \
  template cudaError_t launch_mul<T>(long long, const T*, const T*, T*, cudaStream_t);                                \
  template cudaError_t launch_scale<T>(long long, T, const T*, T*, cudaStream_t);                                     \
  template cudaError_t launch_scale_by_inv<T>(long long, const double*, const T*, T*, cudaStream_t);                  \
  template cudaError_t launch_project_pressure<T>(long long, int, const T*, T*, double*, double*, cudaStream_t);      \
  template cudaError_t launch_coarse_solve<T>(int, int, const int*, int, int, const double*, int, const T*, T*,       \
                                              double*, double*, cudaStream_t);                                        \
  template cudaError_t launch_dot<T, T>(const T*, const T*, long long, long long, double*, double*, int, cudaStream_t);
WB_VINST(double)
WB_VINST(float)
template cudaError_t launch_cast<double, float>(long long, const double*, float*, cudaStream_t);
template cudaError_t launch_cast<float, double>(long long, const float*, double*, cudaStream_t);
template cudaError_t launch_cast<double, double>(long long, const double*, double*, cudaStream_t);
template cudaError_t launch_cast<float, float>(long long, const float*, float*, cudaStream_t);
