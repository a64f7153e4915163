// Device helpers shared by the element-operator kernels: per-order sizes, reference tables
// staged in shared memory, and the node -> adjacent-elements walk of the structured mesh.
#pragma once

#include "common.cuh"

namespace wb {

template <int N> struct Cfg {
  static constexpr int N3 = N * N * N;
  static constexpr int NP = (N - 1) * N * (N + 1) / 6;
  static constexpr int EPB = N3 >= 100 ? 1 : (N3 >= 64 ? 2 : 4);
  static constexpr int THREADS = EPB * N3;
};

template <typename T, int N>
struct SmTab {
  T D[N][N];
  T w[N];
  T pw[N][N];
  int ex[Cfg<N>::NP][3];
};

template <typename T, int N>
__device__ inline void load_tab(SmTab<T, N>& s, const RefTables* __restrict__ tab) {
  for (int t = threadIdx.x; t < N * N; t += blockDim.x) {
    s.D[t / N][t % N] = (T)tab->D[t / N][t % N];
    s.pw[t / N][t % N] = (T)tab->pw[t / N][t % N];
  }
  for (int t = threadIdx.x; t < N; t += blockDim.x) s.w[t] = (T)tab->w[t];
  for (int t = threadIdx.x; t < Cfg<N>::NP * 3; t += blockDim.x) s.ex[t / 3][t % 3] = tab->ex[t / 3][t % 3];
}

template <typename T, int N>
__device__ inline T psi(const SmTab<T, N>& s, int m, int i, int j, int l) {
  return s.pw[i][s.ex[m][0]] * s.pw[j][s.ex[m][1]] * s.pw[l][s.ex[m][2]];
}

__device__ inline int sym_index(int c, int d) {
  // xx, yy, zz, xy, xz, yz
  if (c == d) return c;
  int lo = c < d ? c : d, hi = c < d ? d : c;
  return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}

// Operator tables in shared memory for the hot kernels: derivative matrices pre-scaled by
// 2/h per axis, tensor quadrature weights (with and without |J|), the pressure basis at the
// points, the inverse reference pressure mass and the per-child 1-D interpolation weights.
// Built once per level on the host (make_optab) in the kernel's precision, so blocks only copy
// them into shared memory: no per-block arithmetic, and no FP64 arithmetic in FP32 kernels.
template <typename T, int N>
struct OpTab {
  T Ds[3][N][N];             // Ds[d][i][a] = (2 / h_d) l_a'(x_i)
  T W3[Cfg<N>::N3];          // W_q |J|
  T Wref[Cfg<N>::N3];        // W_q (reference element)
  T Psi[Cfg<N>::N3][Cfg<N>::NP];
  T Minv[Cfg<N>::NP][Cfg<N>::NP];
  T P1[2][N][N];             // P1[s][a][b] = l_b((x_a + 2s - 1) / 2)
};

template <typename T, int N>
inline void make_optab(const RefTables& t, const Grid& g, OpTab<T, N>* o) {
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP;
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < N; ++a) o->Ds[d][i][a] = T(g.s[d] * t.D[i][a]);
  for (int q = 0; q < N3; ++q) {
    const int i = q % N, j = (q / N) % N, l = q / (N * N);
    const double w = t.w[i] * t.w[j] * t.w[l];
    o->W3[q] = T(w * g.detJ);
    o->Wref[q] = T(w);
    for (int m = 0; m < NP; ++m) o->Psi[q][m] = T(t.pw[i][t.ex[m][0]] * t.pw[j][t.ex[m][1]] * t.pw[l][t.ex[m][2]]);
  }
  for (int m = 0; m < NP; ++m)
    for (int mp = 0; mp < NP; ++mp) o->Minv[m][mp] = T(t.minv[m][mp]);
  for (int s2 = 0; s2 < 2; ++s2)
    for (int a = 0; a < N; ++a)
      for (int b = 0; b < N; ++b) o->P1[s2][a][b] = T(t.P1[s2][a][b]);
}

// Block-wide copy of a table from global memory into shared memory (32-bit words).
template <typename Tab>
__device__ inline void copy_tab(Tab& dst, const Tab* __restrict__ src) {
  static_assert(sizeof(Tab) % 4 == 0, "table size must be a multiple of 4 bytes");
  const unsigned* s = reinterpret_cast<const unsigned*>(src);
  unsigned* d = reinterpret_cast<unsigned*>(&dst);
  for (int t = threadIdx.x; t < (int)(sizeof(Tab) / 4); t += blockDim.x) d[t] = s[t];
}

// Calls f(e, ex, ey, ez, a0, a1, a2) for every element containing node (ix, iy, iz), in a fixed order.
template <typename F>
__device__ inline void for_elements_of_node(const Grid& g, int K, int ix, int iy, int iz, F f) {
  int lo[3], hi[3];
  const int idx[3] = {ix, iy, iz}, ne[3] = {g.nx, g.ny, g.nz};
  for (int d = 0; d < 3; ++d) {
    int e = idx[d] / K;
    if (idx[d] % K == 0) {
      lo[d] = e - 1 < 0 ? 0 : e - 1;
      hi[d] = e > ne[d] - 1 ? ne[d] - 1 : e;
    } else {
      lo[d] = hi[d] = e;
    }
  }
  for (int ez = lo[2]; ez <= hi[2]; ++ez)
    for (int ey = lo[1]; ey <= hi[1]; ++ey)
      for (int ex = lo[0]; ex <= hi[0]; ++ex)
        f(ex + g.nx * (ey + g.ny * ez), ex, ey, ez, ix - K * ex, iy - K * ey, iz - K * ez);
}

}  // namespace wb
