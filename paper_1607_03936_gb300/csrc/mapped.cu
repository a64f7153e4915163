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

// Elements per block: in FP64 at k = 2, 32, so the 27 x 32 threads fill 27 warps (four elements
// would leave a quarter of the last warp idle; the FP64 pass is bound by the FP64 pipe, 2469 against
// 2767 us for the A apply at 64^3); otherwise the per-point layout's count (FP32 k = 2: 4 x 27
// threads, measured faster there; k = 3: 2 x 64; k = 4: 125).
template <typename T, int N>
struct MCfg {
  static constexpr int N3 = N * N * N;
  static constexpr int EPB = (N == 3 && sizeof(T) == 8) ? 32 : Cfg<N>::EPB;
  static constexpr int THREADS = EPB * N3;
};

// Dynamic shared memory of one block: the operator tables, then the staged coordinates, velocities,
// pulled-back stresses and weighted divergences of its elements.
template <typename T, int N, int OPS>
constexpr size_t mapped_smem() {
  constexpr bool GRAD = (OPS & OP_A) || (OPS & OP_B), SCAT = (OPS & OP_A) || (OPS & OP_BT), DB = OPS & OP_B;
  constexpr size_t tab = (sizeof(OpTab<T, N>) + 15) / 16 * 16;
  return tab + sizeof(T) * MCfg<T, N>::EPB * MCfg<T, N>::N3 * (3 + (GRAD ? 3 : 0) + (SCAT ? 9 : 0) + (DB ? 1 : 0));
}

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
__global__ void __launch_bounds__(MCfg<T, N>::THREADS)
k_mapped_elem(Grid g, const OpTab<T, N>* __restrict__ otab, const T* __restrict__ X, const T* __restrict__ u,
              const T* __restrict__ p, const T* __restrict__ coef, int coef_nodal, T* __restrict__ Ye, Epi<T> pe,
              int* __restrict__ bad) {
  pdl_entry();
  constexpr int N3 = MCfg<T, N>::N3, NP = Cfg<N>::NP, EPB = MCfg<T, N>::EPB, K = N - 1;
  constexpr bool DA = OPS & OP_A, DBT = OPS & OP_BT, DB = OPS & OP_B, MASS = OPS & OPM_MASS;
  constexpr bool GRAD = DA || DB, SCAT = DA || DBT;
  extern __shared__ __align__(16) unsigned char msm[];
  OpTab<T, N>& st = *reinterpret_cast<OpTab<T, N>*>(msm);
  T* base = reinterpret_cast<T*>(msm + (sizeof(OpTab<T, N>) + 15) / 16 * 16);
  T(*sX)[3][N3] = reinterpret_cast<T(*)[3][N3]>(base);
  base += (size_t)EPB * 3 * N3;
  T(*su)[3][N3] = reinterpret_cast<T(*)[3][N3]>(base);
  base += GRAD ? (size_t)EPB * 3 * N3 : 0;
  T(*sT)[9][N3] = reinterpret_cast<T(*)[9][N3]>(base);
  base += SCAT ? (size_t)EPB * 9 * N3 : 0;
  T(*sdiv)[N3] = reinterpret_cast<T(*)[N3]>(base);
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

template <typename T, int N, int OPS>
cudaError_t launch_one(const Grid& g, const OpTab<T, N>* tab, const T* X, const T* u, const T* p, const T* coef,
                       int cn, T* Ye, const Epi<T>& pe, int* bad, cudaStream_t st) {
  constexpr int EPB = MCfg<T, N>::EPB, TH = MCfg<T, N>::THREADS;
  const long long nb = ((long long)g.ne + EPB - 1) / EPB;
  const long long cap = 152LL * 16 * Cfg<N>::EPB / EPB;   // about 16 blocks' worth of elements per SM
  const unsigned blocks = (unsigned)(nb < cap ? nb : cap);
  wb_launch(k_mapped_elem<T, N, OPS>, blocks, TH, mapped_smem<T, N, OPS>(), st, g, tab, X, u, p, coef, cn, Ye, pe,
            bad);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t run_mapped(const Grid& g, const void* reftab, const T* X, int ops, const T* u, const T* p, const T* coef,
                       int cn, T* Ye, const Epi<T>& pe, int* bad, cudaStream_t st) {
  const OpTab<T, N>* tab = static_cast<const OpTab<T, N>*>(reftab);
  switch (ops) {
    case OP_A: return launch_one<T, N, OP_A>(g, tab, X, u, p, coef, cn, Ye, pe, bad, st);
    case OP_BT: return launch_one<T, N, OP_BT>(g, tab, X, u, p, coef, cn, Ye, pe, bad, st);
    case OP_B: return launch_one<T, N, OP_B>(g, tab, X, u, p, coef, cn, Ye, pe, bad, st);
    case OP_A | OP_BT | OP_B: return launch_one<T, N, OP_A | OP_BT | OP_B>(g, tab, X, u, p, coef, cn, Ye, pe, bad, st);
    case OPM_MASS: return launch_one<T, N, OPM_MASS>(g, tab, X, u, p, coef, cn, Ye, pe, bad, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int N, int OPS>
cudaError_t smem_attr() {
  return cudaFuncSetAttribute(k_mapped_elem<T, N, OPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)mapped_smem<T, N, OPS>());
}

template <typename T, int N>
cudaError_t smem_attrs() {
  cudaError_t e = smem_attr<T, N, OP_A>();
  if (e == cudaSuccess) e = smem_attr<T, N, OP_BT>();
  if (e == cudaSuccess) e = smem_attr<T, N, OP_B>();
  if (e == cudaSuccess) e = smem_attr<T, N, OP_A | OP_BT | OP_B>();
  if (e == cudaSuccess) e = smem_attr<T, N, OPM_MASS>();
  return e;
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

cudaError_t mapped_prepare() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = smem_attrs<double, 3>();
  if (e == cudaSuccess) e = smem_attrs<double, 4>();
  if (e == cudaSuccess) e = smem_attrs<double, 5>();
  if (e == cudaSuccess) e = smem_attrs<float, 3>();
  if (e == cudaSuccess) e = smem_attrs<float, 4>();
  if (e == cudaSuccess) e = smem_attrs<float, 5>();
  done = e == cudaSuccess;
  return e;
}

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
