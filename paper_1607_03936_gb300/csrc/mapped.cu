// Stokes operators on mapped (non-affine) hexahedra: the element pass of A, B, B^T and the fused K,
// and the point weights W_q det J_q, for an isoparametric Q_k geometry given by the physical
// coordinates of every node (Sec. 1.2 forms on the mapped element).
//
// One thread per element point, EPB elements per block (the per-point layout of fused_ops.cu).  The
// element's nodal coordinates and velocities are staged in shared memory; each thread forms, by the
// same 1-D derivative sums along the three reference axes (sum factorisation),
//   J[d][r] = dx_d / dxi_r   and   gh[c][r] = du_c / dxi_r,
// inverts J by its adjugate, takes the physical gradient G[c][d] = sum_r gh[c][r] Jinv[r][d], the
// weighted stress S = W det J (2 mu eps(u) - p I) and its pull-back T[c][r] = sum_d S[c][d] Jinv[r][d]
// (nine values per point, in shared memory); the transposed reference derivative sums of T give the
// element's contribution to each of its nodes:
//   y_c(i,j,l) = sum_a D[a][i] T[c][0](a,j,l) + D[a][j] T[c][1](i,a,l) + D[a][l] T[c][2](i,j,a).
// The geometry is recomputed per apply from the coordinates (3 values per node, read like a
// velocity), not stored per point (10 values per point): the pass stays one nodal read heavier than
// the brick's instead of carrying a metric array three to four times the size of the velocity.
// The node pass (the brick's element-major gather, in fixed element order) sums the contributions.
#include <type_traits>

#include "elem_common.cuh"
#include "epi.cuh"
#include "fused.h"
#include "kernels.h"

namespace {

using namespace wb;

constexpr int OPM_MASS = 16;   // this file only: the point weights W_q det J_q, one component

template <typename T>
struct Jac {
  T inv[3][3];   // inv[r][d] = dxi_r / dx_d
  T det;
};

// Reference derivative of the staged nodal field f (N^3 values) at point (i, j, l) along each axis.
template <typename T, int N>
__device__ __forceinline__ void ref_grad(const OpTab<T, N>& st, const T* f, int i, int j, int l, T (&g)[3]) {
  T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
  for (int a = 0; a < N; ++a) {
    a0 += st.Ds[0][i][a] * f[a + N * (j + N * l)];
    a1 += st.Ds[1][j][a] * f[i + N * (a + N * l)];
    a2 += st.Ds[2][l][a] * f[i + N * (j + N * a)];
  }
  g[0] = a0;
  g[1] = a1;
  g[2] = a2;
}

// Inverse of M (M[d][r] = dx_d / dxi_r) by the adjugate; det M returned beside it.
template <typename T>
__device__ __forceinline__ Jac<T> invert(const T (&M)[3][3]) {
  Jac<T> J;
  const T c00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
  const T c01 = M[0][2] * M[2][1] - M[0][1] * M[2][2];
  const T c02 = M[0][1] * M[1][2] - M[0][2] * M[1][1];
  const T c10 = M[1][2] * M[2][0] - M[1][0] * M[2][2];
  const T c11 = M[0][0] * M[2][2] - M[0][2] * M[2][0];
  const T c12 = M[0][2] * M[1][0] - M[0][0] * M[1][2];
  const T c20 = M[1][0] * M[2][1] - M[1][1] * M[2][0];
  const T c21 = M[0][1] * M[2][0] - M[0][0] * M[2][1];
  const T c22 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
  J.det = M[0][0] * c00 + M[0][1] * c10 + M[0][2] * c20;
  const T id = T(1) / J.det;
  J.inv[0][0] = c00 * id; J.inv[0][1] = c01 * id; J.inv[0][2] = c02 * id;
  J.inv[1][0] = c10 * id; J.inv[1][1] = c11 * id; J.inv[1][2] = c12 * id;
  J.inv[2][0] = c20 * id; J.inv[2][1] = c21 * id; J.inv[2][2] = c22 * id;
  return J;
}

// Grid-stride over batches of EPB elements.  X: coordinates [3][nn]; u: velocity [3][nn] (Dirichlet
// nodes read as zero); p: pressure [ne][Np]; coef: viscosity (nodal or per point).  Ye: element-major
// outputs [ne][3][N^3] (A, B^T), or [ne][N^3] point weights (OPM_MASS).  pe: epilogue of the
// pressure output (B).  bad: set to 1 where det J <= 0 (the outputs there are not meaningful).
template <typename T, int N, int OPS>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_mapped_elem(Grid g, const OpTab<T, N>* __restrict__ otab, const T* __restrict__ X, const T* __restrict__ u,
              const T* __restrict__ p, const T* __restrict__ coef, int coef_nodal, T* __restrict__ Ye, Epi<T> pe,
              int* __restrict__ bad) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP, EPB = Cfg<N>::EPB, K = N - 1;
  constexpr bool DA = OPS & OP_A, DBT = OPS & OP_BT, DB = OPS & OP_B, MASS = OPS & OPM_MASS;
  constexpr bool GRAD = DA || DB, SCAT = DA || DBT;
  __shared__ OpTab<T, N> st;
  __shared__ T sX[EPB][3][N3];
  __shared__ T su[GRAD ? EPB : 1][3][N3];
  __shared__ T sT[SCAT ? EPB : 1][9][N3];
  __shared__ T sdiv[DB ? EPB : 1][N3];
  copy_tab(st, otab);
  const int tid = threadIdx.x;
  const int le = tid / N3, q = tid - le * N3;
  const int i = q % N, j = (q / N) % N, l = q / (N * N);
  const int nbatch = (g.ne + EPB - 1) / EPB;
  for (int eb = blockIdx.x; eb < nbatch; eb += gridDim.x) {
    __syncthreads();
    const int e = eb * EPB + le;
    const bool act = e < g.ne;
    int node = 0;
    if (act) {
      const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
      const int ix = K * ex + i, iy = K * ey + j, iz = K * ez + l;
      node = ix + g.NX * (iy + g.NY * iz);
      const bool interior = !on_boundary(g, ix, iy, iz);
#pragma unroll
      for (int d = 0; d < 3; ++d) sX[le][d][q] = X[(size_t)d * g.nn + node];
      if (GRAD) {
#pragma unroll
        for (int c = 0; c < 3; ++c) su[GRAD ? le : 0][c][q] = interior ? u[(size_t)c * g.nn + node] : T(0);
      }
    }
    __syncthreads();
    if (act) {
      T M[3][3];
#pragma unroll
      for (int d = 0; d < 3; ++d) ref_grad<T, N>(st, sX[le][d], i, j, l, M[d]);
      const Jac<T> J = invert(M);
      if (!(J.det > T(0))) *bad = 1;
      const T wdet = st.Wref[q] * J.det;
      if (MASS) Ye[(size_t)e * N3 + q] = wdet;
      T G[3][3];
      if (GRAD) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T gh[3];
          ref_grad<T, N>(st, su[GRAD ? le : 0][c], i, j, l, gh);
#pragma unroll
          for (int d = 0; d < 3; ++d) G[c][d] = gh[0] * J.inv[0][d] + gh[1] * J.inv[1][d] + gh[2] * J.inv[2][d];
        }
      }
      if (DB) sdiv[DB ? le : 0][q] = wdet * (G[0][0] + G[1][1] + G[2][2]);
      if (SCAT) {
        T S[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) S[c][d] = T(0);
        if (DA) {
          const T mu = coef_nodal ? coef[node] : coef[(size_t)e * N3 + q];
          const T f = T(2) * wdet * mu, hf = wdet * mu;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            S[c][c] = f * G[c][c];
#pragma unroll
            for (int d = c + 1; d < 3; ++d) {
              S[c][d] = hf * (G[c][d] + G[d][c]);
              S[d][c] = S[c][d];
            }
          }
        }
        if (DBT) {
          T pq = 0;
#pragma unroll
          for (int m = 0; m < NP; ++m) pq += st.Psi[q][m] * p[(size_t)e * NP + m];
          const T t = wdet * pq;
#pragma unroll
          for (int c = 0; c < 3; ++c) S[c][c] -= t;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int r = 0; r < 3; ++r)
            sT[SCAT ? le : 0][3 * c + r][q] = S[c][0] * J.inv[r][0] + S[c][1] * J.inv[r][1] + S[c][2] * J.inv[r][2];
      }
    }
    if (!(SCAT || DB)) continue;
    __syncthreads();
    if (DB && act && q < NP) {
      T acc = 0;
      for (int qq = 0; qq < N3; ++qq) acc += st.Psi[qq][q] * sdiv[DB ? le : 0][qq];
      epi_apply(pe, (size_t)e * NP + q, 0, -acc);
    }
    if (SCAT && act) {
      const T(*Tq)[N3] = sT[SCAT ? le : 0];
      T* out = Ye + (size_t)e * 3 * N3 + q;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T acc = 0;
#pragma unroll
        for (int a = 0; a < N; ++a) {
          acc += st.Ds[0][a][i] * Tq[3 * c + 0][a + N * (j + N * l)];
          acc += st.Ds[1][a][j] * Tq[3 * c + 1][i + N * (a + N * l)];
          acc += st.Ds[2][a][l] * Tq[3 * c + 2][i + N * (j + N * a)];
        }
        out[c * N3] = acc;
      }
    }
  }
}

template <typename T, int N>
cudaError_t run_mapped(const Grid& g, const void* reftab, const T* X, int ops, const T* u, const T* p, const T* coef,
                       int cn, T* Ye, const Epi<T>& pe, int* bad, cudaStream_t st) {
  constexpr int EPB = Cfg<N>::EPB, TH = Cfg<N>::THREADS;
  const OpTab<T, N>* tab = static_cast<const OpTab<T, N>*>(reftab);
  const long long nb = ((long long)g.ne + EPB - 1) / EPB;
  const unsigned blocks = (unsigned)(nb < 152LL * 16 ? nb : 152LL * 16);
  switch (ops) {
    case OP_A: wb_launch(k_mapped_elem<T, N, OP_A>, blocks, TH, 0, st, g, tab, X, u, p, coef, cn, Ye, pe, bad); break;
    case OP_BT: wb_launch(k_mapped_elem<T, N, OP_BT>, blocks, TH, 0, st, g, tab, X, u, p, coef, cn, Ye, pe, bad); break;
    case OP_B: wb_launch(k_mapped_elem<T, N, OP_B>, blocks, TH, 0, st, g, tab, X, u, p, coef, cn, Ye, pe, bad); break;
    case OP_A | OP_BT | OP_B:
      wb_launch(k_mapped_elem<T, N, OP_A | OP_BT | OP_B>, blocks, TH, 0, st, g, tab, X, u, p, coef, cn, Ye, pe, bad);
      break;
    case OPM_MASS:
      wb_launch(k_mapped_elem<T, N, OPM_MASS>, blocks, TH, 0, st, g, tab, X, u, p, coef, cn, Ye, pe, bad);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_mapped_k(const Grid& g, int k, const void* reftab, const T* X, int ops, const T* u, const T* p,
                         const T* coef, int cn, T* Ye, const Epi<T>& pe, int* bad, cudaStream_t st) {
  switch (k) {
    case 2: return run_mapped<T, 3>(g, reftab, X, ops, u, p, coef, cn, Ye, pe, bad, st);
    case 3: return run_mapped<T, 4>(g, reftab, X, ops, u, p, coef, cn, Ye, pe, bad, st);
    case 4: return run_mapped<T, 5>(g, reftab, X, ops, u, p, coef, cn, Ye, pe, bad, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_mapped_stokes(const Grid& g, int k, const void* reftab, const T* X, int ops, const T* u,
                                 const T* p, const T* coef, int cn, T* Ye, const Epi<T>& yu, const Epi<T>& yp,
                                 int* bad, cudaStream_t st) {
  if (ops != OP_A && ops != OP_B && ops != OP_BT && ops != (OP_A | OP_BT | OP_B)) return cudaErrorInvalidValue;
  const cudaError_t e = run_mapped_k<T>(g, k, reftab, X, ops, u, p, coef, cn, Ye, yp, bad, st);
  if (e != cudaSuccess || ops == OP_B) return e;
  return launch_gather_elem<T>(g, k, 3, 1, Ye, yu, st);
}

template <typename T>
cudaError_t launch_mapped_mass(const Grid& g, int k, const void* reftab, const T* X, T* Ye, T* lm, int* bad,
                               cudaStream_t st) {
  const cudaError_t e = run_mapped_k<T>(g, k, reftab, X, OPM_MASS, nullptr, nullptr, nullptr, 0, Ye, Epi<T>(), bad, st);
  if (e != cudaSuccess) return e;
  Epi<T> ep;
  ep.mode = EPI_STORE;
  ep.y = lm;
  return launch_gather_elem<T>(g, k, 1, 0, Ye, ep, st);
}

#define WB_MAPPED_INST(T)                                                                                          \
  template cudaError_t launch_mapped_stokes<T>(const Grid&, int, const void*, const T*, int, const T*, const T*,  \
                                               const T*, int, T*, const Epi<T>&, const Epi<T>&, int*,             \
                                               cudaStream_t);                                                     \
  template cudaError_t launch_mapped_mass<T>(const Grid&, int, const void*, const T*, T*, T*, int*, cudaStream_t);
WB_MAPPED_INST(double)
WB_MAPPED_INST(float)
