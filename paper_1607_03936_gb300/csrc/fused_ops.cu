// Two-pass element operators with fused epilogues and fused grid transfers (see fused.h).
//
// Element pass: one thread per element point, EPB elements per block; the element's
// velocity tile is gathered into shared memory, the gradient is formed by 1-D
// derivative sums along each axis (sum factorisation, n FMAs per entry), the
// quadrature-weighted stress 2 mu W eps(u) - W p I is stored back, and the transposed
// derivative sums give the element's contribution to each of its nodes (Sec. 1.2:
// a(u,v) = int 2 mu eps(u):eps(v), b(v,q) = -int q div v).
// Node pass: each node adds the contributions of its elements in the order
// (ez, ey, ex) ascending, so results are bitwise reproducible.
#include <algorithm>
#include <type_traits>

#include "elem_common.cuh"
#include "epi.cuh"
#include "fused.h"
#include "kernels.h"

namespace {

using namespace wb;

// One batch of EPB elements (eb); every thread of the block reaches every barrier.
template <typename T, int N, int OPS>
__device__ inline void elem_batch(const Grid& g, const OpTab<T, N>& st, int eb, const T* __restrict__ u,
                                  const T* __restrict__ us, const T* __restrict__ p, const T* __restrict__ coef,
                                  int coef_nodal, T* __restrict__ Ye, const Epi<T>& pe) {
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP, EPB = Cfg<N>::EPB, K = N - 1;
  constexpr bool DA = OPS & OP_A, DBT = OPS & OP_BT, DB = OPS & OP_B;
  constexpr bool SCAT = DA || DBT, GRAD = DA || DB;
  constexpr int NS = DA ? 6 : 1;
  __shared__ T su[GRAD ? EPB : 1][3][N3];
  __shared__ T sS[SCAT ? EPB : 1][NS][N3];
  __shared__ T sdiv[DB ? EPB : 1][N3];

  const int tid = threadIdx.x;
  const int le = tid / N3, q = tid - le * N3;
  const int i = q % N, j = (q / N) % N, l = q / (N * N);
  const int e = eb * EPB + le;
  const bool act = e < g.ne;
  int node = 0;
  bool interior = false;
  if (act) {
    const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
    const int ix = K * ex + i, iy = K * ey + j, iz = K * ez + l;
    node = ix + g.NX * (iy + g.NY * iz);
    interior = !on_boundary(g, ix, iy, iz);
  }
  T mu = 0, pq = 0;
  if (act) {
    if (GRAD) {
      const T sc = (us != nullptr && interior) ? us[node] : T(1);
#pragma unroll
      for (int c = 0; c < 3; ++c) su[GRAD ? le : 0][c][q] = interior ? u[(size_t)c * g.nn + node] * sc : T(0);
    }
    if (DA) mu = coef_nodal ? coef[node] : coef[(size_t)e * N3 + q];
  }
  __syncthreads();
  if (act && DBT) {
#pragma unroll
    for (int m = 0; m < NP; ++m) pq += st.Psi[q][m] * p[(size_t)e * NP + m];
  }
  if (act) {
    const T Wq = st.W3[q];
    if (DA) {
      T G[3][3];
      T rx[N], ry[N], rz[N];   // this point's derivative rows, held in registers
#pragma unroll
      for (int a = 0; a < N; ++a) {
        rx[a] = st.Ds[0][i][a];
        ry[a] = st.Ds[1][j][a];
        rz[a] = st.Ds[2][l][a];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T a0 = 0, a1 = 0, a2 = 0;
        const T* uc = su[GRAD ? le : 0][c];
#pragma unroll
        for (int a = 0; a < N; ++a) {
          a0 += rx[a] * uc[a + N * (j + N * l)];
          a1 += ry[a] * uc[i + N * (a + N * l)];
          a2 += rz[a] * uc[i + N * (j + N * a)];
        }
        G[c][0] = a0;
        G[c][1] = a1;
        G[c][2] = a2;
      }
      if (DB) sdiv[DB ? le : 0][q] = Wq * (G[0][0] + G[1][1] + G[2][2]);
      const T f = Wq * T(2) * mu, hf = Wq * mu;
      const T t = DBT ? Wq * pq : T(0);
      T* S = &sS[SCAT ? le : 0][0][0];
      S[0 * N3 + q] = f * G[0][0] - t;
      S[(NS > 1 ? 1 : 0) * N3 + q] = f * G[1][1] - t;
      S[(NS > 2 ? 2 : 0) * N3 + q] = f * G[2][2] - t;
      S[(NS > 3 ? 3 : 0) * N3 + q] = hf * (G[0][1] + G[1][0]);
      S[(NS > 4 ? 4 : 0) * N3 + q] = hf * (G[0][2] + G[2][0]);
      S[(NS > 5 ? 5 : 0) * N3 + q] = hf * (G[1][2] + G[2][1]);
    } else {
      if (DB) {
        T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int a = 0; a < N; ++a) {
          a0 += st.Ds[0][i][a] * su[GRAD ? le : 0][0][a + N * (j + N * l)];
          a1 += st.Ds[1][j][a] * su[GRAD ? le : 0][1][i + N * (a + N * l)];
          a2 += st.Ds[2][l][a] * su[GRAD ? le : 0][2][i + N * (j + N * a)];
        }
        sdiv[DB ? le : 0][q] = Wq * (a0 + a1 + a2);
      }
      if (DBT) sS[SCAT ? le : 0][0][q] = -Wq * pq;
    }
  }
  __syncthreads();
  if (DB) {
    // B u per mode m: -sum_q Psi[q][m] sdiv[q], split over the element's threads in RC chunks of
    // ceil(N3 / RC) points (partials in shared memory), then RC-term sums: short dependent chains.
    constexpr int RC = (N3 / NP) < 8 ? (N3 / NP) : 8;
    constexpr int CH = (N3 + RC - 1) / RC;
    __shared__ T spart[DB ? EPB : 1][NP][RC];
    if (act && q < NP * RC) {
      const int m = q % NP, ch = q / NP;
      T acc = 0;
#pragma unroll
      for (int t = 0; t < CH; ++t) {
        const int qq = ch * CH + t;
        if (qq < N3) acc += st.Psi[qq][m] * sdiv[DB ? le : 0][qq];
      }
      spart[DB ? le : 0][m][ch] = acc;
    }
    __syncthreads();
    if (act && q < NP) {
      T acc = 0;
#pragma unroll
      for (int ch = 0; ch < RC; ++ch) acc += spart[DB ? le : 0][q][ch];
      epi_apply(pe, (size_t)e * NP + q, 0, -acc);
    }
  }
  if (!act) return;
  if (SCAT) {
    const T* S = &sS[SCAT ? le : 0][0][0];
    T* out = Ye + (size_t)e * 3 * N3 + q;
    T cx[N], cy[N], cz[N];   // this point's derivative columns (transposed apply)
#pragma unroll
    for (int a = 0; a < N; ++a) {
      cx[a] = st.Ds[0][a][i];
      cy[a] = st.Ds[1][a][j];
      cz[a] = st.Ds[2][a][l];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T acc = 0;
      if (DA) {
        const int i0 = sym_index(c, 0), i1 = sym_index(c, 1), i2 = sym_index(c, 2);
#pragma unroll
        for (int a = 0; a < N; ++a) {
          acc += cx[a] * S[i0 * N3 + a + N * (j + N * l)];
          acc += cy[a] * S[i1 * N3 + i + N * (a + N * l)];
          acc += cz[a] * S[i2 * N3 + i + N * (j + N * a)];
        }
      } else {
#pragma unroll
        for (int a = 0; a < N; ++a) {
          const int qa = c == 0 ? a + N * (j + N * l) : (c == 1 ? i + N * (a + N * l) : i + N * (j + N * a));
          const int qc = c == 0 ? i : (c == 1 ? j : l);
          acc += st.Ds[c][a][qc] * S[qa];
        }
      }
      out[c * N3] = acc;
    }
  }
}

// Grid-stride over element batches: the block copies the operator tables once and reuses them.
template <typename T, int N, int OPS>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_elem(Grid g, const OpTab<T, N>* __restrict__ otab, const T* __restrict__ u, const T* __restrict__ us,
       const T* __restrict__ p, const T* __restrict__ coef, int coef_nodal, T* __restrict__ Ye, Epi<T> pe) {
  pdl_entry();
  __shared__ OpTab<T, N> st;
  copy_tab(st, otab);
  const int nbatch = (g.ne + Cfg<N>::EPB - 1) / Cfg<N>::EPB;
  for (int eb = blockIdx.x; eb < nbatch; eb += gridDim.x) {
    __syncthreads();
    elem_batch<T, N, OPS>(g, st, eb, u, us, p, coef, coef_nodal, Ye, pe);
  }
}

template <typename T, int N>
__device__ inline void poisson_batch(const Grid& g, const OpTab<T, N>& st, int eb, const T* __restrict__ u,
                                     const T* __restrict__ coef, T* __restrict__ Ye) {
  constexpr int N3 = Cfg<N>::N3, EPB = Cfg<N>::EPB, K = N - 1;
  __shared__ T su[EPB][N3];
  __shared__ T sF[EPB][3][N3];
  const int tid = threadIdx.x;
  const int le = tid / N3, q = tid - le * N3;
  const int i = q % N, j = (q / N) % N, l = q / (N * N);
  const int e = eb * EPB + le;
  const bool act = e < g.ne;
  if (act) {
    const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
    su[le][q] = u[(K * ex + i) + g.NX * ((K * ey + j) + g.NY * (K * ez + l))];
  }
  __syncthreads();
  T cx[N], cy[N], cz[N];
  if (act) {
    T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      a0 += st.Ds[0][i][a] * su[le][a + N * (j + N * l)];
      a1 += st.Ds[1][j][a] * su[le][i + N * (a + N * l)];
      a2 += st.Ds[2][l][a] * su[le][i + N * (j + N * a)];
      cx[a] = st.Ds[0][a][i];
      cy[a] = st.Ds[1][a][j];
      cz[a] = st.Ds[2][a][l];
    }
    const T f = st.W3[q] * coef[(size_t)e * N3 + q];
    sF[le][0][q] = f * a0;
    sF[le][1][q] = f * a1;
    sF[le][2][q] = f * a2;
  }
  __syncthreads();
  if (!act) return;
  T acc = 0;
#pragma unroll
  for (int a = 0; a < N; ++a) {
    acc += cx[a] * sF[le][0][a + N * (j + N * l)];
    acc += cy[a] * sF[le][1][i + N * (a + N * l)];
    acc += cz[a] * sF[le][2][i + N * (j + N * a)];
  }
  Ye[(size_t)e * N3 + q] = acc;
}

template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_elem_poisson(Grid g, const OpTab<T, N>* __restrict__ otab, const T* __restrict__ u, const T* __restrict__ coef,
               T* __restrict__ Ye) {
  pdl_entry();
  __shared__ OpTab<T, N> st;
  copy_tab(st, otab);
  const int nbatch = (g.ne + Cfg<N>::EPB - 1) / Cfg<N>::EPB;
  for (int eb = blockIdx.x; eb < nbatch; eb += gridDim.x) {
    __syncthreads();
    poisson_batch<T, N>(g, st, eb, u, coef, Ye);
  }
}

// Node pass: thread per node, sum over the elements containing it in (ez, ey, ex) order; launch
// shape of node_pass_geometry, epilogue operands loaded before the contributions.
template <typename T, int N, int NC, int MODE>
__global__ void k_gather(Grid g, int mask_boundary, const T* __restrict__ Ye, Epi<T> E) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, K = N - 1;
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= g.NX) return;
  for (int iz = blockIdx.z; iz < g.NZ; iz += gridDim.z)
    for (int iy = blockIdx.y; iy < g.NY; iy += gridDim.y) {
      const int n = ix + g.NX * (iy + g.NY * iz);
      EpiOps<T> eo[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) eo[c] = epi_pre<MODE>(E, (size_t)c * g.nn + n, n);
      T v[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c] = T(0);
      if (!(mask_boundary && on_boundary(g, ix, iy, iz))) {
        for_elements_of_node(g, K, ix, iy, iz, [&](int e, int, int, int, int a0, int a1, int a2) {
          const T* src = Ye + (size_t)e * NC * N3 + (a0 + N * (a1 + N * a2));
#pragma unroll
          for (int c = 0; c < NC; ++c) v[c] += src[c * N3];
        });
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) epi_post<MODE>(E, (size_t)c * g.nn + n, eo[c], v[c]);
    }
}

// Fine node value = sum over the N^3 coarse nodes of its coarse element of the tensor weights.
template <typename T, int N>
__global__ void k_prolong3d(Grid gc, const OpTab<T, N>* __restrict__ otab, int ncomp, const T* __restrict__ in_c,
                            T* __restrict__ out_f, int add) {
  pdl_entry();
  constexpr int K = N - 1;
  __shared__ T P1[2][N][N];
  for (int t = threadIdx.x; t < 2 * N * N; t += blockDim.x) (&P1[0][0][0])[t] = (&otab->P1[0][0][0])[t];
  __syncthreads();
  const int NXf = 2 * K * gc.nx + 1, NYf = 2 * K * gc.ny + 1, NZf = 2 * K * gc.nz + 1;
  const long long nf = (long long)NXf * NYf * NZf;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nf) return;
  const int idx[3] = {(int)(t % NXf), (int)((t / NXf) % NYf), (int)(t / ((long long)NXf * NYf))};
  const int nfe[3] = {2 * gc.nx, 2 * gc.ny, 2 * gc.nz};
  int base[3], sa[3][2];
  for (int d = 0; d < 3; ++d) {
    int ef = idx[d] / K;
    if (ef > nfe[d] - 1) ef = nfe[d] - 1;
    sa[d][0] = ef % 2;
    sa[d][1] = idx[d] - K * ef;
    base[d] = K * (ef / 2);
  }
  const T* wx = P1[sa[0][0]][sa[0][1]];
  const T* wy = P1[sa[1][0]][sa[1][1]];
  const T* wz = P1[sa[2][0]][sa[2][1]];
  for (int c = 0; c < ncomp; ++c) {
    const T* src = in_c + (size_t)c * gc.nn;
    T acc = 0;
#pragma unroll
    for (int bz = 0; bz < N; ++bz) {
#pragma unroll
      for (int by = 0; by < N; ++by) {
        const T wzy = wz[bz] * wy[by];
        const T* row = src + (size_t)base[0] + (size_t)gc.NX * ((base[1] + by) + (size_t)gc.NY * (base[2] + bz));
        T r = 0;
#pragma unroll
        for (int bx = 0; bx < N; ++bx) r += wx[bx] * row[bx];
        acc += wzy * r;
      }
    }
    T* dst = out_f + (size_t)c * nf + t;
    *dst = add ? *dst + acc : acc;
  }
}

// One axis of P^T for all components (grid.y = component); the last pass may zero boundary nodes.
template <typename T, int N>
__global__ void k_rpass(const OpTab<T, N>* __restrict__ otab, int axis, int d0, int d1, int d2, int nc_el,
                        long long in_stride, long long out_stride, const T* __restrict__ in, T* __restrict__ out,
                        int mask_last) {
  pdl_entry();
  constexpr int K = N - 1;
  __shared__ T P1[2][N][N];
  for (int t = threadIdx.x; t < 2 * N * N; t += blockDim.x) (&P1[0][0][0])[t] = (&otab->P1[0][0][0])[t];
  __syncthreads();
  const int nfine = 2 * K * nc_el + 1, ncoarse = K * nc_el + 1;
  int od[3] = {d0, d1, d2};
  od[axis] = ncoarse;
  const long long tot = (long long)od[0] * od[1] * od[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  int o[3];
  o[0] = (int)(t % od[0]);
  o[1] = (int)((t / od[0]) % od[1]);
  o[2] = (int)(t / ((long long)od[0] * od[1]));
  const T* src = in + blockIdx.y * in_stride;
  T* dst = out + blockIdx.y * out_stride;
  if (mask_last && (o[0] == 0 || o[1] == 0 || o[2] == 0 || o[0] == od[0] - 1 || o[1] == od[1] - 1 ||
                    o[2] == od[2] - 1)) {
    dst[t] = T(0);
    return;
  }
  const int id[3] = {d0, d1, d2};
  const int i_c = o[axis];
  const int nf_el = 2 * nc_el;
  int lo = 2 * i_c - 2 * K, hi = 2 * i_c + 2 * K;
  if (lo < 0) lo = 0;
  if (hi > nfine - 1) hi = nfine - 1;
  const long long stride = axis == 0 ? 1 : (axis == 1 ? id[0] : (long long)id[0] * id[1]);
  int c3[3] = {o[0], o[1], o[2]};
  c3[axis] = 0;
  const long long base = (long long)c3[0] + (long long)id[0] * (c3[1] + (long long)id[1] * c3[2]);
  T acc = 0;
  for (int i_f = lo; i_f <= hi; ++i_f) {
    int ef = i_f / K;
    if (ef > nf_el - 1) ef = nf_el - 1;
    const int a = i_f - K * ef, ec = ef / 2, s = ef % 2;
    const int b = i_c - K * ec;
    if (b < 0 || b > K) continue;
    acc += P1[s][a][b] * src[base + i_f * stride];
  }
  dst[t] = acc;
}

// Q2 restriction out_c = P^T in_f in one pass.  Along each axis coarse node i contributes the
// fine nodes of the coarse elements that contain it with the interpolation weights P1[s][a][b]
// (child s, fine local node a, coarse local node b): an odd i (b = 1) takes fine nodes 2i - 1,
// 2i, 2i + 1; an even i (b = 0 of its right element, b = 2 of its left one) takes 2i - 3,
// 2i - 1 (left element), 2i, 2i + 1, 2i + 3 (right element), where they exist; the other fine
// nodes of those elements have zero weight.  The x sum runs innermost.
// Taps of coarse node i along one axis in five fixed slots (ascending fine index; ok = used).
template <typename T>
struct Q2Taps {
  int off[5];
  T w[5];
  bool ok[5];
};

template <typename T>
__device__ inline Q2Taps<T> q2_taps(int i, int nf, const T (*P1)[3][3]) {
  Q2Taps<T> t;
  const bool odd = i & 1;
  t.off[0] = odd ? 2 * i - 1 : 2 * i - 3;
  t.w[0] = odd ? P1[0][1][1] : P1[0][1][2];
  t.ok[0] = odd || i > 0;
  t.off[1] = odd ? 2 * i : 2 * i - 1;
  t.w[1] = odd ? P1[1][0][1] : P1[1][1][2];
  t.ok[1] = odd || i > 0;
  t.off[2] = odd ? 2 * i + 1 : 2 * i;
  t.w[2] = odd ? P1[1][1][1] : P1[0][0][0];
  t.ok[2] = true;
  t.off[3] = 2 * i + 1;
  t.w[3] = P1[0][1][0];
  t.ok[3] = !odd && 2 * i + 1 < nf;
  t.off[4] = 2 * i + 3;
  t.w[4] = P1[1][1][0];
  t.ok[4] = !odd && 2 * i + 1 < nf;
  return t;
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_restrict_q2(Grid gc, const OpTab<T, 3>* __restrict__ otab, int ncomp, const T* __restrict__ in,
                              T* __restrict__ out, int mask) {
  pdl_entry();
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= gc.NX) return;
  const int NXf = 2 * gc.NX - 1, NYf = 2 * gc.NY - 1, NZf = 2 * gc.NZ - 1;
  const size_t nf = (size_t)NXf * NYf * NZf;
  const T(*P1)[3][3] = otab->P1;
  const Q2Taps<T> tx = q2_taps<T>(ix, NXf, P1);
  for (int iz = blockIdx.z; iz < gc.NZ; iz += gridDim.z)
    for (int iy = blockIdx.y; iy < gc.NY; iy += gridDim.y) {
      const size_t n = (size_t)ix + (size_t)gc.NX * (iy + (size_t)gc.NY * iz);
      const bool zero = mask && on_boundary(gc, ix, iy, iz);
      const Q2Taps<T> ty = q2_taps<T>(iy, NYf, P1), tz = q2_taps<T>(iz, NZf, P1);
      for (int c = 0; c < ncomp; ++c) {
        T acc = T(0);
        if (!zero) {
          const T* src = in + (size_t)c * nf;
#pragma unroll
          for (int a = 0; a < 5; ++a) {
            if (!tz.ok[a]) continue;
#pragma unroll
            for (int b = 0; b < 5; ++b) {
              if (!ty.ok[b]) continue;
              const T* row = src + (size_t)NXf * (ty.off[b] + (size_t)NYf * tz.off[a]);
              T r = T(0);
#pragma unroll
              for (int t = 0; t < 5; ++t)
                if (tx.ok[t]) r += tx.w[t] * row[tx.off[t]];
              acc += tz.w[a] * ty.w[b] * r;
            }
          }
        }
        out[(size_t)c * gc.nn + n] = acc;
      }
    }
}

// Q2 transfers on large grids, tiled through shared memory: the tensor-product weights are applied
// one axis at a time on a tile, so each fine value is read from memory about once instead of once
// per coarse node (restriction, 125 taps) or per fine node (prolongation, 27 taps).
constexpr int TR_C = 8;                 // restriction: coarse nodes per tile edge
constexpr int TR_F = 2 * TR_C + 5;      // fine nodes per tile edge (taps reach 3 beyond each end)
constexpr int TP_F = 16;                // prolongation: fine nodes per tile edge
constexpr int TP_C = TP_F / 2 + 1;      // coarse nodes per tile edge
constexpr int TT_THREADS = 256;

// Asynchronous copy of one entry into shared memory; src_bytes = 0 writes zeros (the source is not
// read).
template <typename T>
__device__ __forceinline__ void cp_async_entry(T* dst, const T* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(sizeof(T)),
               "r"(valid ? (int)sizeof(T) : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T>
constexpr size_t restrict_tiled_smem() {
  return sizeof(T) * ((size_t)TR_F * TR_F * TR_F + (size_t)TR_F * TR_F * TR_C + (size_t)TR_F * TR_C * TR_C +
                      3 * TR_C * 5) +
         sizeof(int) * 3 * TR_C * 5;
}
template <typename T>
constexpr size_t prolong_tiled_smem() {
  return sizeof(T) * ((size_t)TP_C * TP_C * TP_C + (size_t)TP_F * TP_C * TP_C + (size_t)TP_F * TP_F * TP_C +
                      (size_t)TP_F * TP_F * TP_F + 18);
}

// out_c = P^T in_f: the taps of k_restrict_q2 along x, then y, then z, on a TR_C^3 coarse tile.
// The taps of the tile's coarse nodes per axis are formed once (an absent tap has weight 0 and
// reads an entry of the tile: adding the exact zero leaves the sums unchanged).
template <typename T>
__global__ void __launch_bounds__(TT_THREADS) k_restrict_q2_tiled(Grid gc, const OpTab<T, 3>* __restrict__ otab,
                                                                  int ncomp, const T* __restrict__ in,
                                                                  T* __restrict__ out, int mask) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char tr_smem[];
  T* F = reinterpret_cast<T*>(tr_smem);        // [TR_F z][TR_F y][TR_F x]
  T* T1 = F + TR_F * TR_F * TR_F;              // [TR_F z][TR_F y][TR_C x]
  T* T2 = T1 + TR_F * TR_F * TR_C;             // [TR_F z][TR_C y][TR_C x]
  T* tw = T2 + TR_F * TR_C * TR_C;             // [axis][coarse node][tap]: weight
  int* to = reinterpret_cast<int*>(tw + 3 * TR_C * 5);   // tile-local fine index of the tap
  const int NXf = 2 * gc.NX - 1, NYf = 2 * gc.NY - 1, NZf = 2 * gc.NZ - 1;
  const size_t nf = (size_t)NXf * NYf * NZf;
  const int c = blockIdx.z % ncomp;   // one component per block: grid.z = tiles along z x ncomp
  const int cx0 = blockIdx.x * TR_C, cy0 = blockIdx.y * TR_C, cz0 = (blockIdx.z / ncomp) * TR_C;
  const int fx0 = 2 * cx0 - 3, fy0 = 2 * cy0 - 3, fz0 = 2 * cz0 - 3;
  const T* src = in + (size_t)c * nf;
  for (int t = threadIdx.x; t < TR_F * TR_F * TR_F; t += TT_THREADS) {
    const int gx = fx0 + t % TR_F, gy = fy0 + (t / TR_F) % TR_F, gz = fz0 + t / (TR_F * TR_F);
    const bool ok = gx >= 0 && gx < NXf && gy >= 0 && gy < NYf && gz >= 0 && gz < NZf;
    cp_async_entry(F + t, ok ? src + (size_t)gx + (size_t)NXf * (gy + (size_t)NYf * gz) : src, ok);
  }
  if (threadIdx.x < 3 * TR_C) {
    const int axis = threadIdx.x / TR_C, kk = threadIdx.x % TR_C;
    const int c0 = axis == 0 ? cx0 : (axis == 1 ? cy0 : cz0), f0 = 2 * c0 - 3;
    const int nfa = axis == 0 ? NXf : (axis == 1 ? NYf : NZf);
    const Q2Taps<T> tp = q2_taps<T>(c0 + kk, nfa, otab->P1);
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      tw[threadIdx.x * 5 + t] = tp.ok[t] ? tp.w[t] : T(0);
      to[threadIdx.x * 5 + t] = tp.ok[t] ? tp.off[t] - f0 : 0;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  {
    // a thread's coarse x node (t mod 8) is the same in every step: its taps stay in registers
    const int kx = threadIdx.x & (TR_C - 1);
    T w[5];
    int o[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      w[k] = tw[kx * 5 + k];
      o[k] = to[kx * 5 + k];
    }
    for (int t = threadIdx.x; t < TR_F * TR_F * TR_C; t += TT_THREADS) {
      const T* fr = F + (t >> 3) * TR_F;
      T r = T(0);
#pragma unroll
      for (int k = 0; k < 5; ++k) r += w[k] * fr[o[k]];
      T1[t] = r;
    }
  }
  __syncthreads();
  {
    // likewise the coarse y node ((t / 8) mod 8)
    const int kx = threadIdx.x & (TR_C - 1), ky = (threadIdx.x >> 3) & (TR_C - 1);
    T w[5];
    int o[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      w[k] = tw[(TR_C + ky) * 5 + k];
      o[k] = to[(TR_C + ky) * 5 + k] * TR_C + kx;
    }
    for (int t = threadIdx.x; t < TR_F * TR_C * TR_C; t += TT_THREADS) {
      const T* tz = T1 + (t >> 6) * TR_F * TR_C;
      T r = T(0);
#pragma unroll
      for (int k = 0; k < 5; ++k) r += w[k] * tz[o[k]];
      T2[t] = r;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < TR_C * TR_C * TR_C; t += TT_THREADS) {
    const int kx = t & (TR_C - 1), ky = (t >> 3) & (TR_C - 1), kz = t >> 6;
    const int ix = cx0 + kx, iy = cy0 + ky, iz = cz0 + kz;
    if (ix >= gc.NX || iy >= gc.NY || iz >= gc.NZ) continue;
    T r = T(0);
    if (!(mask && on_boundary(gc, ix, iy, iz))) {
      const T* w = tw + (2 * TR_C + kz) * 5;
      const int* o = to + (2 * TR_C + kz) * 5;
#pragma unroll
      for (int k = 0; k < 5; ++k) r += w[k] * T2[(o[k] * TR_C + ky) * TR_C + kx];
    }
    out[(size_t)c * gc.nn + (size_t)ix + (size_t)gc.NX * (iy + (size_t)gc.NY * iz)] = r;
  }
}
static_assert(TR_C == 8 && TT_THREADS % 64 == 0, "the pass index arithmetic assumes 8 coarse nodes per tile edge");

// out_f (+)= P in_c: the nodal interpolation weights of k_prolong3d along z, then y, then x, on a
// TP_F^3 fine tile (its coarse nodes: a TP_C^3 block).  The target tile is fetched asynchronously
// with the coarse block, so the final pass reads it from shared memory.
template <typename T>
__global__ void __launch_bounds__(TT_THREADS) k_prolong_q2_tiled(Grid gc, const OpTab<T, 3>* __restrict__ otab,
                                                                 int ncomp, const T* __restrict__ in_c,
                                                                 T* __restrict__ out_f, int add) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char tp_smem[];
  T* C = reinterpret_cast<T*>(tp_smem);       // [TP_C z][TP_C y][TP_C x]
  T* Z1 = C + TP_C * TP_C * TP_C;             // [TP_F z][TP_C y][TP_C x]
  T* Y1 = Z1 + TP_F * TP_C * TP_C;            // [TP_F z][TP_F y][TP_C x]
  T* O = Y1 + TP_F * TP_F * TP_C;             // [TP_F z][TP_F y][TP_F x]: the target tile
  T* P1 = O + TP_F * TP_F * TP_F;             // [2][3][3]
  const int NXf = 4 * gc.nx + 1, NYf = 4 * gc.ny + 1, NZf = 4 * gc.nz + 1;
  const size_t nf = (size_t)NXf * NYf * NZf;
  const int c = blockIdx.z % ncomp;   // one component per block: grid.z = tiles along z x ncomp
  const int fx0 = blockIdx.x * TP_F, fy0 = blockIdx.y * TP_F, fz0 = (blockIdx.z / ncomp) * TP_F;
  const int nfe[3] = {2 * gc.nx, 2 * gc.ny, 2 * gc.nz};
  // fine node f along an axis: its fine element ef (the last one for the end node), child s of
  // the coarse element ef / 2, local node a; coarse nodes 2 (ef / 2) + b, b = 0, 1, 2
  auto split = [&](int f, int d, int& s, int& a, int& cb) {
    int ef = f / 2;
    if (ef > nfe[d] - 1) ef = nfe[d] - 1;
    s = ef % 2;
    a = f - 2 * ef;
    cb = 2 * (ef / 2);
  };
  // the tile's first coarse node per axis: that of its first fine node (a tile holding only the
  // end node starts two coarse nodes before it); every fine node of the tile then reads coarse
  // nodes c0 .. c0 + TP_C - 1
  int c0x, c0y, c0z, s_, a_;
  split(fx0, 0, s_, a_, c0x);
  split(fy0, 1, s_, a_, c0y);
  split(fz0, 2, s_, a_, c0z);
  const T* src = in_c + (size_t)c * gc.nn;
  T* dst = out_f + (size_t)c * nf;
  for (int t = threadIdx.x; t < TP_C * TP_C * TP_C; t += TT_THREADS) {
    const int x = t % TP_C, y = (t / TP_C) % TP_C, z = t / (TP_C * TP_C);
    const int gx = c0x + x, gy = c0y + y, gz = c0z + z;
    const bool ok = gx < gc.NX && gy < gc.NY && gz < gc.NZ;
    cp_async_entry(C + t, ok ? src + (size_t)gx + (size_t)gc.NX * (gy + (size_t)gc.NY * gz) : src, ok);
  }
  if (add) {
    for (int t = threadIdx.x; t < TP_F * TP_F * TP_F; t += TT_THREADS) {
      const int gx = fx0 + (t & (TP_F - 1)), gy = fy0 + ((t >> 4) & (TP_F - 1)), gz = fz0 + (t >> 8);
      const bool ok = gx < NXf && gy < NYf && gz < NZf;
      cp_async_entry(O + t, ok ? dst + (size_t)gx + (size_t)NXf * (gy + (size_t)NYf * gz) : dst, ok);
    }
  }
  for (int t = threadIdx.x; t < 18; t += TT_THREADS) P1[t] = (&otab->P1[0][0][0])[t];
  cp_async_wait_all();
  __syncthreads();
  for (int t = threadIdx.x; t < TP_F * TP_C * TP_C; t += TT_THREADS) {
    const int x = t % TP_C, y = (t / TP_C) % TP_C, fz = t / (TP_C * TP_C);
    int s, a, cb;
    split(min(fz0 + fz, NZf - 1), 2, s, a, cb);
    T r = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) r += P1[(s * 3 + a) * 3 + b] * C[((cb + b - c0z) * TP_C + y) * TP_C + x];
    Z1[t] = r;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < TP_F * TP_F * TP_C; t += TT_THREADS) {
    const int x = t % TP_C, fy = (t / TP_C) % TP_F, fz = t / (TP_C * TP_F);
    int s, a, cb;
    split(min(fy0 + fy, NYf - 1), 1, s, a, cb);
    T r = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) r += P1[(s * 3 + a) * 3 + b] * Z1[(fz * TP_C + (cb + b - c0y)) * TP_C + x];
    Y1[t] = r;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < TP_F * TP_F * TP_F; t += TT_THREADS) {
    const int fx = t & (TP_F - 1), fy = (t >> 4) & (TP_F - 1), fz = t >> 8;
    const int gx = fx0 + fx, gy = fy0 + fy, gz = fz0 + fz;
    if (gx >= NXf || gy >= NYf || gz >= NZf) continue;
    int s, a, cb;
    split(gx, 0, s, a, cb);
    T r = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) r += P1[(s * 3 + a) * 3 + b] * Y1[(fz * TP_F + fy) * TP_C + (cb + b - c0x)];
    dst[(size_t)gx + (size_t)NXf * (gy + (size_t)NYf * gz)] = add ? O[t] + r : r;
  }
}
static_assert(TP_F == 16, "the pass index arithmetic assumes 16 fine nodes per tile edge");

// Pressure transfers of the two-space Poisson cycle (|J| cancels between M_d^-1 and the masses):
//   element pass of r_c = M_cd M_d^-1 r_d: Ye[e][q] = W_q sum_m psi_m(q) (Minv r_e)_m
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_d2c_elem(Grid g, const OpTab<T, N>* __restrict__ otab, const T* __restrict__ rd, T* __restrict__ Ye) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP, EPB = Cfg<N>::EPB;
  __shared__ OpTab<T, N> st;
  __shared__ T sv[EPB][NP];
  copy_tab(st, otab);
  const int le = threadIdx.x / N3, q = threadIdx.x - le * N3;
  const int e = blockIdx.x * EPB + le;
  const bool act = e < g.ne;
  __syncthreads();
  if (act && q < NP) {
    T v = 0;
#pragma unroll
    for (int mp = 0; mp < NP; ++mp) v += st.Minv[q][mp] * rd[(size_t)e * NP + mp];
    sv[le][q] = v;
  }
  __syncthreads();
  if (!act) return;
  T acc = 0;
#pragma unroll
  for (int m = 0; m < NP; ++m) acc += st.Psi[q][m] * sv[le][m];
  Ye[(size_t)e * N3 + q] = st.Wref[q] * acc;
}

//   e_d[e][m] (+)= sum_m' Minv[m][m'] sum_q W_q psi_m'(q) e_c(node(e, q))
template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_c2d_elem(Grid g, const OpTab<T, N>* __restrict__ otab, const T* __restrict__ ec, T* __restrict__ ed, int add) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP, EPB = Cfg<N>::EPB, K = N - 1;
  __shared__ OpTab<T, N> st;
  __shared__ T sw[EPB][N3];
  __shared__ T sg[EPB][NP];
  copy_tab(st, otab);
  const int le = threadIdx.x / N3, q = threadIdx.x - le * N3;
  const int i = q % N, j = (q / N) % N, l = q / (N * N);
  const int e = blockIdx.x * EPB + le;
  const bool act = e < g.ne;
  __syncthreads();
  if (act) {
    const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
    sw[le][q] = st.Wref[q] * ec[(K * ex + i) + g.NX * ((K * ey + j) + g.NY * (K * ez + l))];
  }
  __syncthreads();
  if (act && q < NP) {
    T acc = 0;
#pragma unroll
    for (int qq = 0; qq < N3; ++qq) acc += st.Psi[qq][q] * sw[le][qq];
    sg[le][q] = acc;
  }
  __syncthreads();
  if (act && q < NP) {
    T v = 0;
#pragma unroll
    for (int mp = 0; mp < NP; ++mp) v += st.Minv[q][mp] * sg[le][mp];
    T* dst = ed + (size_t)e * NP + q;
    *dst = add ? *dst + v : v;
  }
}

inline unsigned nb(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Element-pass grid: one block per batch up to 12 blocks per SM (152 SMs); beyond that each
// block loops over batches, so its shared operator tables are loaded once per several batches.
inline unsigned elem_blocks(int ne, int epb) {
  const long long nbatch = (ne + epb - 1) / epb;
  return (unsigned)(nbatch < 152 * 12 ? nbatch : 152 * 12);
}

template <typename T, int N>
cudaError_t run_elem(const Grid& g, const void* otab_v, int ops, const T* u, const T* us, const T* p, const T* coef,
                     int cn, T* Ye, const Epi<T>& pe, cudaStream_t st) {
  constexpr int EPB = Cfg<N>::EPB, TH = Cfg<N>::THREADS;
  const OpTab<T, N>* tab = static_cast<const OpTab<T, N>*>(otab_v);
  const unsigned blocks = elem_blocks(g.ne, EPB);
  switch (ops) {
    case OP_A: wb_launch(k_elem<T, N, OP_A>, blocks, TH, 0, st, g, tab, u, us, p, coef, cn, Ye, pe); break;
    case OP_BT: wb_launch(k_elem<T, N, OP_BT>, blocks, TH, 0, st, g, tab, u, us, p, coef, cn, Ye, pe); break;
    case OP_B: wb_launch(k_elem<T, N, OP_B>, blocks, TH, 0, st, g, tab, u, us, p, coef, cn, Ye, pe); break;
    case OP_A | OP_BT | OP_B:
      wb_launch(k_elem<T, N, OP_A | OP_BT | OP_B>, blocks, TH, 0, st, g, tab, u, us, p, coef, cn, Ye, pe);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

#define WB_FUSED_DISPATCH(k, CALL) \
  switch (k) {                     \
    case 1: { constexpr int N = 2; return CALL; } \
    case 2: { constexpr int N = 3; return CALL; } \
    case 3: { constexpr int N = 4; return CALL; } \
    case 4: { constexpr int N = 5; return CALL; } \
    default: return cudaErrorInvalidValue; \
  }

#define WB_TAB(T) static_cast<const OpTab<T, N>*>(otab)

// At k = 2 on grids flagged `rowk` the element passes take the row-segment kernels: the scalar
// ones (Poisson, pressure transfers; q2_ops.cu) in both precisions, the vector Stokes ones with
// a thread per element in single precision (q2_ops.cu) and a warp per element point in double
// precision (q2_fp64.cu).  Their scratch layout is the row one, which the matching launch_gather
// reads (ncomp 1: scalar producers, ncomp 3: Stokes producers).
template <typename T>
bool row_path_scalar(const Grid& g, int k) {
  return k == 2 && g.rowk;
}
template <typename T>
bool row_path_vector(const Grid& g, int k) {
  return k == 2 && g.rowk;
}

// Below the row-segment size, FP64 k = 2 levels of at least 2048 elements take the flat
// warp-per-point passes (q2_fp64.cu, element-major scratch) unless the option asks for the
// per-point kernels; smaller levels keep the per-point kernels (more blocks than SMs).
template <typename T>
bool flat_path(const Grid& g, int k) {
  return std::is_same<T, double>::value && k == 2 && !g.rowk && g.kern != 1 && g.ne >= 2048;
}

template <typename T>
bool fused_path(const Grid& g, int k) {
  return std::is_same<T, float>::value && k == 2 && q2_fused_eligible(g);
}

template <typename T>
size_t elem_scratch_size(const Grid& g, int k) {
  const size_t n = (size_t)(k + 1);
  const size_t elem = 3 * (size_t)g.ne * n * n * n;
  if (fused_path<T>(g, k)) return std::max({elem, q2_row_scratch(g, 3), q2_fused_scratch(g)});
  if (row_path_vector<T>(g, k)) return std::max(elem, q2_row_scratch(g, 3));
  if (row_path_scalar<T>(g, k)) return std::max(elem, q2_row_scratch(g, 1));
  return elem;
}

template <typename T>
cudaError_t launch_elem_stokes(const Grid& g, int k, const void* otab, int ops, const T* u, const T* us, const T* p,
                               const T* coef, int cn, T* Ye, const Epi<T>& pe, cudaStream_t st) {
  if (row_path_vector<T>(g, k)) {
    if (us != nullptr) return cudaErrorInvalidValue;   // input scaling is not part of the row kernels
    if constexpr (std::is_same<T, float>::value) return launch_q2_elem(g, ops, u, p, coef, cn, Ye, pe, st);
    else return launch_q2_elem64(g, ops, u, p, coef, cn, Ye, pe, st);
  }
  if constexpr (std::is_same<T, double>::value) {
    if (flat_path<T>(g, k) && ops == OP_A && us == nullptr) return launch_q2_elem64_flat(g, u, coef, cn, Ye, st);
  }
  WB_FUSED_DISPATCH(k, (run_elem<T, N>(g, otab, ops, u, us, p, coef, cn, Ye, pe, st)));
}

template <typename T>
cudaError_t launch_apply_vec_epi(const Grid& g, int k, const void* otab, int ops, const T* u, const T* p,
                                 const T* coef, int cn, T* Ye, int mask, const Epi<T>& e, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (fused_path<T>(g, k)) return launch_q2_fused(g, ops, u, p, coef, cn, Ye, mask, e, st);
  }
  const cudaError_t err = launch_elem_stokes<T>(g, k, otab, ops, u, nullptr, p, coef, cn, Ye, Epi<T>(), st);
  if (err != cudaSuccess) return err;
  return launch_gather<T>(g, k, 3, mask, Ye, e, st);
}

template <typename T>
cudaError_t launch_elem_poisson(const Grid& g, int k, const void* otab, const T* u, const T* coef, T* Ye,
                                cudaStream_t st);

template <typename T>
cudaError_t launch_apply_poisson_epi(const Grid& g, int k, const void* otab, const T* u, const T* coef, T* Ye,
                                     const Epi<T>& e, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (fused_path<T>(g, k)) return launch_q2_fused(g, Q2_FUSED_POISSON, u, nullptr, coef, 0, Ye, 0, e, st);
  }
  const cudaError_t err = launch_elem_poisson<T>(g, k, otab, u, coef, Ye, st);
  if (err != cudaSuccess) return err;
  return launch_gather<T>(g, k, 1, 0, Ye, e, st);
}

template <typename T>
cudaError_t launch_elem_poisson(const Grid& g, int k, const void* otab, const T* u, const T* coef, T* Ye,
                                cudaStream_t st) {
  if (row_path_scalar<T>(g, k)) {
    if constexpr (std::is_same<T, double>::value) return launch_q2_poisson64(g, u, coef, Ye, st);
    else return launch_q2_poisson<T>(g, u, coef, Ye, st);
  }
  if constexpr (std::is_same<T, double>::value) {
    if (flat_path<T>(g, k)) return launch_q2_poisson64_flat(g, u, coef, Ye, st);
  }
  WB_FUSED_DISPATCH(k, ((wb_launch(k_elem_poisson<T, N>, elem_blocks(g.ne, Cfg<N>::EPB), Cfg<N>::THREADS, 0, st, g, WB_TAB(T), u, coef, Ye)),
                        cudaGetLastError()));
}

template <typename T>
cudaError_t launch_gather_elem(const Grid& g, int k, int ncomp, int mask, const T* Ye, const Epi<T>& e,
                               cudaStream_t st);

template <typename T>
cudaError_t launch_disc_to_cont_fused(const Grid& g, int k, const void* otab, const T* rd, T* rc, T* Ye,
                                      cudaStream_t st) {
  if (row_path_scalar<T>(g, k)) return launch_q2_d2c<T>(g, rd, rc, Ye, st);
  cudaError_t e = cudaSuccess;
  switch (k) {
    case 2: { constexpr int N = 3; wb_launch(k_d2c_elem<T, N>, (unsigned)((g.ne + Cfg<N>::EPB - 1) / Cfg<N>::EPB), Cfg<N>::THREADS, 0, st, g, WB_TAB(T), rd, Ye); break; }
    case 3: { constexpr int N = 4; wb_launch(k_d2c_elem<T, N>, (unsigned)((g.ne + Cfg<N>::EPB - 1) / Cfg<N>::EPB), Cfg<N>::THREADS, 0, st, g, WB_TAB(T), rd, Ye); break; }
    case 4: { constexpr int N = 5; wb_launch(k_d2c_elem<T, N>, (unsigned)((g.ne + Cfg<N>::EPB - 1) / Cfg<N>::EPB), Cfg<N>::THREADS, 0, st, g, WB_TAB(T), rd, Ye); break; }
    default: return cudaErrorInvalidValue;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  Epi<T> ep;
  ep.mode = EPI_STORE;
  ep.y = rc;
  return launch_gather_elem<T>(g, k, 1, 0, Ye, ep, st);
}

template <typename T>
cudaError_t launch_cont_to_disc_fused(const Grid& g, int k, const void* otab, const T* ec, T* ed, int add,
                                      cudaStream_t st) {
  if (row_path_scalar<T>(g, k)) return launch_q2_c2d<T>(g, ec, ed, add, st);
  WB_FUSED_DISPATCH(k, ((wb_launch(k_c2d_elem<T, N>, (unsigned)((g.ne + Cfg<N>::EPB - 1) / Cfg<N>::EPB), Cfg<N>::THREADS, 0, st, g, WB_TAB(T), ec, ed, add)),
                        cudaGetLastError()));
}

// Node pass over the element-major scratch [ne][ncomp][n^3].
template <typename T>
cudaError_t launch_gather_elem(const Grid& g, int k, int ncomp, int mask, const T* Ye, const Epi<T>& e,
                               cudaStream_t st) {
  dim3 grid;
  int bs;
  node_pass_geometry(g, grid, bs);
  return epi_dispatch(e.mode, [&](auto m) -> cudaError_t {
    constexpr int MODE = decltype(m)::value;
    if (ncomp == 3) {
      WB_FUSED_DISPATCH(k, ((wb_launch(k_gather<T, N, 3, MODE>, grid, bs, 0, st, g, mask, Ye, e)),
                            cudaGetLastError()));
    }
    if (ncomp == 1) {
      WB_FUSED_DISPATCH(k, ((wb_launch(k_gather<T, N, 1, MODE>, grid, bs, 0, st, g, mask, Ye, e)),
                            cudaGetLastError()));
    }
    return cudaErrorInvalidValue;
  });
}

template <typename T>
cudaError_t launch_gather(const Grid& g, int k, int ncomp, int mask, const T* Ye, const Epi<T>& e, cudaStream_t st) {
  if (ncomp == 3 ? row_path_vector<T>(g, k) : row_path_scalar<T>(g, k))
    return launch_q2_gather<T>(g, ncomp, mask, Ye, e, st);
  return launch_gather_elem<T>(g, k, ncomp, mask, Ye, e, st);
}

// The tiled Q2 transfers on grids of at least this many coarse nodes, under the automatic kernel
// choice (the forced choices keep the per-node kernels).
constexpr long long TILED_MIN_NODES = 100000;
bool tiled_transfers(const Grid& gc, int k) { return k == 2 && gc.kern == 0 && gc.nn >= TILED_MIN_NODES; }

cudaError_t transfer_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_restrict_q2_tiled<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)restrict_tiled_smem<float>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_restrict_q2_tiled<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)restrict_tiled_smem<double>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_prolong_q2_tiled<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)prolong_tiled_smem<float>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_prolong_q2_tiled<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)prolong_tiled_smem<double>());
  return e;
}

template <typename T>
cudaError_t launch_prolong_fused(const Grid& gc, int k, const void* otab, int ncomp, const T* in_c, T* out_f, int add,
                                 cudaStream_t st) {
  if (tiled_transfers(gc, k)) {
    const dim3 grid((unsigned)((4 * gc.nx + TP_F) / TP_F), (unsigned)((4 * gc.ny + TP_F) / TP_F),
                    (unsigned)((4 * gc.nz + TP_F) / TP_F * ncomp));
    wb_launch(k_prolong_q2_tiled<T>, grid, TT_THREADS, prolong_tiled_smem<T>(), st, gc,
              static_cast<const OpTab<T, 3>*>(otab), ncomp, in_c, out_f, add);
    return cudaGetLastError();
  }
  const long long nf = (long long)(2 * k * gc.nx + 1) * (2 * k * gc.ny + 1) * (2 * k * gc.nz + 1);
  WB_FUSED_DISPATCH(k, ((wb_launch(k_prolong3d<T, N>, nb(nf, 128), 128, 0, st, gc, WB_TAB(T), ncomp, in_c,
                                                                                            out_f, add)),
                        cudaGetLastError()));
}

namespace {
template <typename T, int N>
cudaError_t run_restrict(const Grid& gc, const void* otab, int ncomp, const T* in_f, T* out_c, int mask, T* w1, T* w2,
                         cudaStream_t st) {
  constexpr int K = N - 1;
  const OpTab<T, N>* tab = static_cast<const OpTab<T, N>*>(otab);
  const int ncx = gc.NX, ncy = gc.NY, ncz = gc.NZ;
  const int nfx = 2 * K * gc.nx + 1, nfy = 2 * K * gc.ny + 1, nfz = 2 * K * gc.nz + 1;
  const long long nf = (long long)nfx * nfy * nfz, n1 = (long long)ncx * nfy * nfz, n2 = (long long)ncx * ncy * nfz;
  const long long nc = (long long)ncx * ncy * ncz;
  const int bs = 256;
  wb_launch(k_rpass<T, N>, dim3(nb(n1, bs), ncomp), bs, 0, st, tab, 0, nfx, nfy, nfz, gc.nx, nf, n1, in_f, w1, 0);
  wb_launch(k_rpass<T, N>, dim3(nb(n2, bs), ncomp), bs, 0, st, tab, 1, ncx, nfy, nfz, gc.ny, n1, n2, w1, w2, 0);
  wb_launch(k_rpass<T, N>, dim3(nb(nc, bs), ncomp), bs, 0, st, tab, 2, ncx, ncy, nfz, gc.nz, n2, nc, w2, out_c,
                                                                           mask);
  return cudaGetLastError();
}
}  // namespace

template <typename T>
cudaError_t launch_restrict_batched(const Grid& gc, int k, const void* otab, int ncomp, const T* in_f, T* out_c,
                                    int mask, T* w1, T* w2, cudaStream_t st) {
  // One pass (one thread per coarse node) pays off on large coarse grids; small ones keep three
  // short separable passes, which have more threads per node (the element-kernel option forces
  // either: per element -> one pass, per point -> three passes).
  if (tiled_transfers(gc, k)) {
    const dim3 grid((unsigned)((gc.NX + TR_C - 1) / TR_C), (unsigned)((gc.NY + TR_C - 1) / TR_C),
                    (unsigned)((gc.NZ + TR_C - 1) / TR_C * ncomp));
    wb_launch(k_restrict_q2_tiled<T>, grid, TT_THREADS, restrict_tiled_smem<T>(), st, gc,
              static_cast<const OpTab<T, 3>*>(otab), ncomp, in_f, out_c, mask);
    return cudaGetLastError();
  }
  const bool one_pass = gc.kern == 2 || (gc.kern == 0 && gc.nn >= TILED_MIN_NODES);
  if (k == 2 && one_pass) {
    dim3 grid;
    int bs;
    node_pass_geometry(gc, grid, bs);
    wb_launch(k_restrict_q2<T>, grid, bs, 0, st, gc, static_cast<const OpTab<T, 3>*>(otab), ncomp, in_f,
                                                              out_c, mask);
    return cudaGetLastError();
  }
  WB_FUSED_DISPATCH(k, (run_restrict<T, N>(gc, otab, ncomp, in_f, out_c, mask, w1, w2, st)));
}

template <typename T>
size_t optab_bytes(int k) {
  switch (k) {
    case 1: return sizeof(OpTab<T, 2>);
    case 2: return sizeof(OpTab<T, 3>);
    case 3: return sizeof(OpTab<T, 4>);
    case 4: return sizeof(OpTab<T, 5>);
    default: return 0;
  }
}

template <typename T>
void build_optab_host(const RefTables& t, const Grid& g, int k, void* out) {
  switch (k) {
    case 1: make_optab<T, 2>(t, g, static_cast<OpTab<T, 2>*>(out)); break;
    case 2: make_optab<T, 3>(t, g, static_cast<OpTab<T, 3>*>(out)); break;
    case 3: make_optab<T, 4>(t, g, static_cast<OpTab<T, 4>*>(out)); break;
    case 4: make_optab<T, 5>(t, g, static_cast<OpTab<T, 5>*>(out)); break;
    default: break;
  }
}

#define WB_FUSED_INST(T)                                                                                              \
  template cudaError_t launch_elem_stokes<T>(const Grid&, int, const void*, int, const T*, const T*, const T*,        \
                                             const T*, int, T*, const Epi<T>&, cudaStream_t);                         \
  template cudaError_t launch_elem_poisson<T>(const Grid&, int, const void*, const T*, const T*, T*, cudaStream_t);  \
  template cudaError_t launch_apply_poisson_epi<T>(const Grid&, int, const void*, const T*, const T*, T*,          \
                                                   const Epi<T>&, cudaStream_t);                                     \
  template cudaError_t launch_apply_vec_epi<T>(const Grid&, int, const void*, int, const T*, const T*, const T*, int, \
                                               T*, int, const Epi<T>&, cudaStream_t);                                \
  template cudaError_t launch_gather<T>(const Grid&, int, int, int, const T*, const Epi<T>&, cudaStream_t);           \
  template cudaError_t launch_gather_elem<T>(const Grid&, int, int, int, const T*, const Epi<T>&, cudaStream_t);      \
  template cudaError_t launch_prolong_fused<T>(const Grid&, int, const void*, int, const T*, T*, int, cudaStream_t);  \
  template cudaError_t launch_restrict_batched<T>(const Grid&, int, const void*, int, const T*, T*, int, T*, T*,      \
                                                  cudaStream_t);                                                      \
  template cudaError_t launch_disc_to_cont_fused<T>(const Grid&, int, const void*, const T*, T*, T*, cudaStream_t);   \
  template cudaError_t launch_cont_to_disc_fused<T>(const Grid&, int, const void*, const T*, T*, int, cudaStream_t);  \
  template size_t optab_bytes<T>(int);                                                                                \
  template size_t elem_scratch_size<T>(const Grid&, int);                                                                                \
  template void build_optab_host<T>(const RefTables&, const Grid&, int, void*);
WB_FUSED_INST(double)
WB_FUSED_INST(float)
