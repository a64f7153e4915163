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
// 2/h per axis, tensor quadrature weights times |J|, and the pressure basis at the points,
// so that the per-point work is only the sum-factorisation FMAs and the pointwise physics.
template <typename T, int N>
struct OpTab {
  T Ds[3][N][N];             // Ds[d][i][a] = (2 / h_d) l_a'(x_i)
  T W3[Cfg<N>::N3];          // W_q |J|
  T Psi[Cfg<N>::N3][Cfg<N>::NP];
};

template <typename T, int N>
__device__ inline void load_optab(OpTab<T, N>& s, const RefTables* __restrict__ tab, const Grid& g, bool need_psi) {
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP;
  for (int t = threadIdx.x; t < 3 * N * N; t += blockDim.x) {
    const int d = t / (N * N), r = t % (N * N);
    s.Ds[d][r / N][r % N] = T(g.s[d] * tab->D[r / N][r % N]);
  }
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    const int i = q % N, j = (q / N) % N, l = q / (N * N);
    s.W3[q] = T(tab->w[i] * tab->w[j] * tab->w[l] * g.detJ);
    if (need_psi)
      for (int m = 0; m < NP; ++m)
        s.Psi[q][m] = T(tab->pw[i][tab->ex[m][0]] * tab->pw[j][tab->ex[m][1]] * tab->pw[l][tab->ex[m][2]]);
  }
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
