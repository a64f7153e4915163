// The weighted pressure Poisson operator K_w = B C_w^-1 B^T (Sec. 6; C_w = lumped velocity mass
// weighted by a(e) sqrt(mu), diagonal) as an assembled block stencil.
//
// On the structured mesh every element has the same local divergence matrix
//   B_e[m][(a, c)] = -sum_q W_q |J| psi_m(q) d_c phi_a(q)        (Sec. 1.2, b(v,q) = -int q div v)
// so (K_w p)_e = sum over the 27 neighbours e' of e (sharing at least one node) of the Np x Np
// block  K[e][e'][m][m'] = sum over shared nodes n and components c of
//   B_e[m][(n, c)] C^-1(n) B_e'[m'][(n, c)].
// The blocks depend on mu only through C^-1 and are assembled once per setup (FP64 sums, stored
// in the preconditioner precision as [o][m][m'][e], o = (dx+1) + 3 (dy+1) + 9 (dz+1)); an apply
// is then one pass over the stencil with the fused pressure epilogue instead of a B^T element
// pass, a node pass and a B element pass.
#include "elem_common.cuh"
#include "epi.cuh"
#include "fused.h"
#include "kernels.h"

namespace {

using namespace wb;

// bref[(m * N3 + a) * 3 + c] = B_e[m][(a, c)] (reference element scaled to the grid).
template <int N>
__global__ void k_kw_bref(Grid g, const RefTables* __restrict__ tab, double* __restrict__ bref) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NP * N3 * 3) return;
  const int c = t % 3, a = (t / 3) % N3, m = t / (3 * N3);
  const int ai[3] = {a % N, (a / N) % N, a / (N * N)};
  double b = 0.0;
  for (int ii = 0; ii < N; ++ii) {   // d_c phi_a is nonzero only at points sharing a's other indices
    int qq[3] = {ai[0], ai[1], ai[2]};
    qq[c] = ii;
    const double Wq = tab->w[qq[0]] * tab->w[qq[1]] * tab->w[qq[2]];
    const double ps = tab->pw[qq[0]][tab->ex[m][0]] * tab->pw[qq[1]][tab->ex[m][1]] * tab->pw[qq[2]][tab->ex[m][2]];
    b += Wq * ps * tab->D[ii][ai[c]];
  }
  bref[t] = -b * g.s[c] * g.detJ;
}

// One thread per (neighbour offset o, element e): the Np x Np block of row element e, column
// element e + d(o); zero where the neighbour lies outside the mesh.
template <typename T, int N>
__global__ void k_kw_assemble(Grid g, const double* __restrict__ bref, const double* __restrict__ cinv,
                              T* __restrict__ Kst) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP, K = N - 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 27LL * g.ne) return;
  const int o = (int)(t / g.ne), e = (int)(t - (long long)o * g.ne);
  const int d[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
  const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
  const int en[3] = {ex + d[0], ey + d[1], ez + d[2]};
  const bool inside = en[0] >= 0 && en[0] < g.nx && en[1] >= 0 && en[1] < g.ny && en[2] >= 0 && en[2] < g.nz;
  double acc[NP][NP];
  for (int m = 0; m < NP; ++m)
    for (int mp = 0; mp < NP; ++mp) acc[m][mp] = 0.0;
  if (inside) {
    // shared nodes: along an axis with offset 0 every local index, with offset +1 (-1) the last
    // (first) local index of e, which is the first (last) of the neighbour
    int lo[3], hi[3];
    for (int x = 0; x < 3; ++x) {
      lo[x] = d[x] > 0 ? K : 0;
      hi[x] = d[x] < 0 ? 0 : K;
    }
    for (int a2 = lo[2]; a2 <= hi[2]; ++a2)
      for (int a1 = lo[1]; a1 <= hi[1]; ++a1)
        for (int a0 = lo[0]; a0 <= hi[0]; ++a0) {
          const int node = (K * ex + a0) + g.NX * ((K * ey + a1) + g.NY * (K * ez + a2));
          const double ci = cinv[node];
          if (ci == 0.0) continue;
          const int qa = a0 + N * (a1 + N * a2);
          const int qp = (a0 - K * d[0]) + N * ((a1 - K * d[1]) + N * (a2 - K * d[2]));
          for (int c = 0; c < 3; ++c)
            for (int m = 0; m < NP; ++m) {
              const double bm = bref[(m * N3 + qa) * 3 + c] * ci;
              for (int mp = 0; mp < NP; ++mp) acc[m][mp] += bm * bref[(mp * N3 + qp) * 3 + c];
            }
        }
  }
  for (int m = 0; m < NP; ++m)
    for (int mp = 0; mp < NP; ++mp) Kst[((size_t)(o * NP + m) * NP + mp) * g.ne + e] = T(acc[m][mp]);
}

// y[e][m] = epilogue( sum over neighbours e' and modes m' of K[o][m][m'][e] p[e'][m'] ), one
// thread per (m, e); neighbours in the order dz, dy, dx ascending.
template <typename T, int N, int MODE>
__global__ void k_kw_apply(Grid g, const T* __restrict__ Kst, const T* __restrict__ p, Epi<T> E) {
  pdl_entry();
  constexpr int NP = Cfg<N>::NP;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)NP * g.ne) return;
  const int m = (int)(t / g.ne), e = (int)(t - (long long)m * g.ne);
  const size_t i = (size_t)e * NP + m;
  const EpiOps<T> eo = epi_pre<MODE>(E, i, 0);
  const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
  const size_t ne = (size_t)g.ne;
  T acc = T(0);
  for (int dz = -1; dz <= 1; ++dz) {
    if (ez + dz < 0 || ez + dz >= g.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      if (ey + dy < 0 || ey + dy >= g.ny) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (ex + dx < 0 || ex + dx >= g.nx) continue;
        const int o = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
        const int e2 = e + dx + g.nx * (dy + g.ny * dz);
        const T* kr = Kst + (size_t)(o * NP + m) * NP * ne + e;
        const T* pp = p + (size_t)e2 * NP;
#pragma unroll
        for (int mp = 0; mp < NP; ++mp) acc += kr[mp * ne] * pp[mp];
      }
    }
  }
  epi_post<MODE>(E, i, eo, acc);
}

// Jacobi diagonal of K_w from the reference table: diag[e][m] = sum over the element's nodes n and
// components c of B_e[m][(n, c)]^2 C^-1(n); dinv = 1 / diag (0 where the diagonal vanishes).
template <typename T, int N>
__global__ void k_kw_dinv(Grid g, const double* __restrict__ bref, const double* __restrict__ cinv,
                          T* __restrict__ dinv) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP, K = N - 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)NP * g.ne) return;
  const int e = (int)(t / NP), m = (int)(t - (long long)e * NP);
  const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
  double acc = 0.0;
  for (int q = 0; q < N3; ++q) {
    const int a0 = q % N, a1 = (q / N) % N, a2 = q / (N * N);
    const double ci = cinv[(K * ex + a0) + g.NX * ((K * ey + a1) + g.NY * (K * ez + a2))];
    if (ci == 0.0) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double b = bref[(m * N3 + q) * 3 + c];
      acc += b * b * ci;
    }
  }
  dinv[t] = acc > 0.0 ? T(1.0 / acc) : T(0);   // a zero diagonal (single-element mesh, constant mode) is skipped
}

inline unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

size_t kw_stencil_entries(const Grid& g, int k) {
  const size_t np = (size_t)k * (k + 1) * (k + 2) / 6;
  return 27 * np * np * (size_t)g.ne;
}

size_t kw_bref_entries(int k) {
  const size_t n = k + 1, np = (size_t)k * (k + 1) * (k + 2) / 6;
  return np * n * n * n * 3;
}

cudaError_t launch_kw_bref(const Grid& g, int k, const RefTables* dtab, double* bref, cudaStream_t st) {
  switch (k) {
    case 2: wb_launch(k_kw_bref<3>, nb256((long long)kw_bref_entries(2)), 256, 0, st, g, dtab, bref); break;
    case 3: wb_launch(k_kw_bref<4>, nb256((long long)kw_bref_entries(3)), 256, 0, st, g, dtab, bref); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kw_assemble(const Grid& g, int k, const double* bref, const double* cinv, T* Kst, cudaStream_t st) {
  const unsigned blocks = nb256(27LL * g.ne);
  switch (k) {
    case 2: wb_launch(k_kw_assemble<T, 3>, blocks, 256, 0, st, g, bref, cinv, Kst); break;
    case 3: wb_launch(k_kw_assemble<T, 4>, blocks, 256, 0, st, g, bref, cinv, Kst); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kw_apply(const Grid& g, int k, const T* Kst, const T* p, const Epi<T>& e, cudaStream_t st) {
  return epi_dispatch(e.mode, [&](auto md) -> cudaError_t {
    constexpr int MODE = decltype(md)::value;
    switch (k) {
      case 2: wb_launch(k_kw_apply<T, 3, MODE>, nb256(4LL * g.ne), 256, 0, st, g, Kst, p, e); break;
      case 3: wb_launch(k_kw_apply<T, 4, MODE>, nb256(10LL * g.ne), 256, 0, st, g, Kst, p, e); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  });
}

template <typename T>
cudaError_t launch_kw_dinv(const Grid& g, int k, const double* bref, const double* cinv, T* dinv, cudaStream_t st) {
  switch (k) {
    case 2: wb_launch(k_kw_dinv<T, 3>, nb256(4LL * g.ne), 256, 0, st, g, bref, cinv, dinv); break;
    case 3: wb_launch(k_kw_dinv<T, 4>, nb256(10LL * g.ne), 256, 0, st, g, bref, cinv, dinv); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_kw_dinv<double>(const Grid&, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_kw_assemble<double>(const Grid&, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_kw_assemble<float>(const Grid&, int, const double*, const double*, float*, cudaStream_t);
template cudaError_t launch_kw_apply<double>(const Grid&, int, const double*, const double*, const Epi<double>&,
                                             cudaStream_t);
template cudaError_t launch_kw_apply<float>(const Grid&, int, const float*, const float*, const Epi<float>&,
                                            cudaStream_t);
