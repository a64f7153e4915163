// Solver context, multigrid hierarchies, w-BFBT, block preconditioner and FGMRES
// behind the C ABI of include/wbfbt.h.
//
//  w-BFBT (Eq. wbfbt):   S~^-1 = (B C^-1 B^T)^-1 (B C^-1 A D^-1 B^T) (B D^-1 B^T)^-1,
//                        C = M~_u(w_l), D = M~_u(w_r), w = a(e) sqrt(mu) (Eq. bdramp)
//  block preconditioner (Eq. precond-stokes): y_p = s S~^-1 r_p, y_u = A~^-1 (r_u - B^T y_p)
//  inner inverses (Sec. 6): geometric V-cycles with Chebyshev(3)-Jacobi smoothing, nested
//                        Q_k transfers, re-discretised coarse operators, FP64 dense coarsest
//                        solve; the pressure-Poisson cycle smooths on P_{k-1}^disc and
//                        corrects with a continuous Q_k Poisson V-cycle.
//  Krylov (Sec. 1.3):    right-preconditioned FGMRES(m), FP64, CGS2, Givens on the host.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <algorithm>
#include <type_traits>
#include <vector>

#include "fused.h"
#include "kernels.h"
#include "unet.h"
#include "vec_ops.h"
#include "wbfbt.h"

namespace {

struct WbErr {
  int code;
};

#define CK(...)                                           \
  do {                                                    \
    cudaError_t _e = (__VA_ARGS__);                       \
    if (_e != cudaSuccess) throw WbErr{WBFBT_ERR_CUDA};   \
  } while (0)

constexpr double CHEB_LO = 0.1, CHEB_HI = 1.1;
constexpr int POWER_ITERS = 10;
constexpr unsigned long long START_SEED = 0x5EED;
constexpr int MAX_DENSE = 12000;   // coarsest dense matrices are n x n FP64 (three copies during setup)

// Device allocations owned by a context, freed together.
struct Pool {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  template <typename T>
  T* get(size_t n) {
    void* p = nullptr;
    size_t b = (n ? n : 1) * sizeof(T);
    if (cudaMalloc(&p, b) != cudaSuccess) throw WbErr{WBFBT_ERR_CUDA};
    ptrs.push_back(p);
    bytes += b;
    return static_cast<T*>(p);
  }
  // Allocate on first use only, so a second setup pass over the same structures allocates nothing.
  template <typename T>
  T* ensure(T*& p, size_t n) {
    if (!p) p = get<T>(n);
    return p;
  }
  ~Pool() {
    for (void* p : ptrs) cudaFree(p);
  }
};

template <typename T>
struct Level {
  Grid g;
  int k = 2;                       // element order of this level (1 on the p-coarsened levels)
  const RefTables* dtab = nullptr; // reference tables of that order (device)
  const T* coef = nullptr;     // level 0 of A: nodal viscosity; otherwise per element point
  int coef_nodal = 0;
  double* coef64 = nullptr;    // FP64 copy used by the setup (per point; nodal on A level 0)
  T* dinv = nullptr;
  double lam = 0.0;
  T *b = nullptr, *x = nullptr, *r = nullptr, *d = nullptr, *tmp = nullptr;
  T *w1 = nullptr, *w2 = nullptr;  // transfer workspaces towards the next coarser level
  bool coarsest = false;
  int* map = nullptr;              // node -> dense index (coarsest)
  int nfree_nodes = 0, ndense = 0;
  double *Ainv = nullptr, *bf = nullptr, *xf = nullptr;
  // setup scratch kept for re-setup without allocation
  double *pts64 = nullptr, *d64 = nullptr, *Md = nullptr;
  T *coefT = nullptr, *pv = nullptr, *pw = nullptr;
  void* optab = nullptr;           // this level's operator tables in precision T (device)
};

template <typename T>
struct Hier {
  bool vec = true;
  int ncomp = 3;
  std::vector<Level<T>> lv;
};

template <typename T>
struct Precond {
  T *mu = nullptr, *cinv = nullptr, *dinvw = nullptr;   // fine nodal viscosity, C^-1, D^-1
  Hier<T> HA, HL[2];
  T* dKw[2] = {nullptr, nullptr};
  double lamKw[2] = {0, 0};
  T *pb = nullptr, *px = nullptr, *pr = nullptr, *pd = nullptr, *ptmp = nullptr, *vtmp = nullptr;
  T *sr = nullptr, *sy = nullptr, *sz = nullptr, *sy2 = nullptr, *sv1 = nullptr, *sv2 = nullptr;
  T *urhs = nullptr, *utmp = nullptr;                   // Schur / block workspaces
  T *ares = nullptr, *acor = nullptr;                   // A~^-1 residual and correction (ainv_cycles > 1)
  T *vin = nullptr, *vout = nullptr;                    // mixed-precision Krylov <-> preconditioner
  T* Ye = nullptr;                                      // element-pass outputs [ne][3][n^3] (finest level)
  T* Kst[2] = {nullptr, nullptr};                       // assembled K_w stencils (k <= 3), w_l and w_r
  T* kwin = nullptr;                                    // copy of a K_w input its epilogue overwrites
  T* Mp = nullptr;                                      // lumped M_p(1/mu)^-1 blocks [ne][Np][Np] (schur = MASS)
  T* wdof = nullptr;                                    // diag(A)^-1 per DOF [3][nn] (weights = DIAG_A): C = D = diag(A)
  double *c0[2] = {nullptr, nullptr}, *dK64[2] = {nullptr, nullptr};
};

}  // namespace

struct wbfbt_ctx {
  ~wbfbt_ctx() {
    if (st) cudaStreamSynchronize(st);
    if (pgraph) cudaGraphExecDestroy(pgraph);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (st) cudaStreamDestroy(st);
  }
  cudaStream_t st = nullptr;    // internal stream: every kernel of the context runs here
  cudaStream_t ust = nullptr;   // the caller's stream, fenced against st at every entry point
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t pgraph = nullptr;   // captured preconditioner application (FGMRES hot loop)
  bool graph_dirty = true;
  long long graph_kernels = 0;
  int k = 2, N = 3, N3 = 27, NP = 4;
  Grid g;
  wbfbt_opts opt;
  int nlev = 1;
  RefTables htab;
  RefTables* dtab = nullptr;
  RefTables htab1;                // order-1 tables for the p-coarsened viscous multigrid (pmg)
  RefTables* dtab1 = nullptr;
  Pool pool;
  // FP64 fine data
  double *mu64 = nullptr, *lm = nullptr, *C = nullptr, *D = nullptr, *cinv64 = nullptr, *dinv64 = nullptr;
  float* mu32 = nullptr;
  double* part = nullptr;   // reduction partials
  double* kwbref = nullptr; // reference divergence matrix for the K_w assembly (k <= 3)
  double* Mp64 = nullptr;   // lumped M_p(1/mu)^-1 blocks in FP64 (schur = MASS)
  double* wpts = nullptr;   // w-BFBT weights per element point (weights = GRAD), or mu per point (DIAG_A)
  double* adinv64 = nullptr;// diag(A)^-1 per DOF, 0 on Dirichlet DOFs (weights = DIAG_A)
  double* dsc = nullptr;    // device scalars (64)
  int* dflag = nullptr;
  Precond<double> P64;
  Precond<float> P32;
  bool mixed = false;
  // FGMRES
  long long ntot = 0;
  int m = 50;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *x = nullptr, *r = nullptr, *F = nullptr, *hdev = nullptr;
  double *stage_f = nullptr, *stage_u = nullptr, *stage_p = nullptr;
  double* Ye64 = nullptr;   // element-pass scratch for the FP64 applies
  float* Ye32 = nullptr;    // element-pass scratch for the FP32 applies
  void* ot64 = nullptr;     // fine-level operator tables, FP64
  void* ot32 = nullptr;     // fine-level operator tables, FP32
  // mapped geometry (wbfbt_set_geometry): the Krylov operator, the entry-point applies and the
  // load vector take the isoparametric map of these nodal coordinates
  bool mapped = false;
  double* X64 = nullptr;    // coordinates [3][nn]
  float* X32 = nullptr;
  void* rt64 = nullptr;     // reference-element operator tables (unscaled derivatives, weights)
  void* rt32 = nullptr;
  double* lm_map = nullptr; // mapped lumped mass per node
  struct DenseJob {
    double* M;
    int n;
    int pin;
  };
  std::vector<DenseJob> dense_jobs;   // coarsest matrices awaiting inversion in the current setup
  double* gj_work = nullptr;          // 4 x 32 x 32 pivot-block workspace
  // learned correction
  wbfbt_net* net = nullptr;
  wbfbt_net* own_net = nullptr;   // created by wbfbt_load_learned, destroyed with the context
  int net_mask = 0;
  double net_accept = 1.0;
  float *lx = nullptr, *ly = nullptr, *lq = nullptr, *llogmu = nullptr;
  long long learned_acc = 0, learned_rej = 0;
};

namespace {

template <typename T>
Precond<T>& prec(wbfbt_ctx* c);
template <>
Precond<double>& prec<double>(wbfbt_ctx* c) { return c->P64; }
template <>
Precond<float>& prec<float>(wbfbt_ctx* c) { return c->P32; }

template <typename T>
const void* fine_tab(wbfbt_ctx* c) {
  return std::is_same<T, double>::value ? c->ot64 : c->ot32;
}

// Device copy of the operator tables of grid g in precision T (built once; tables depend only on g).
template <typename T>
void* make_device_optab(wbfbt_ctx* c, const Grid& g, int k) {
  const size_t nb = optab_bytes<T>(k);
  std::vector<unsigned char> h(nb);
  build_optab_host<T>(k == 1 ? c->htab1 : c->htab, g, k, h.data());
  unsigned char* d = c->pool.get<unsigned char>(nb);
  CK(cudaMemcpy(d, h.data(), nb, cudaMemcpyHostToDevice));
  return d;
}

double read_scalar(wbfbt_ctx* c, const double* dptr) {
  double v = 0.0;
  CK(cudaMemcpyAsync(&v, dptr, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return v;
}

template <typename T>
double norm(wbfbt_ctx* c, const T* v, long long n) {
  CK(launch_dot<T, T>(v, v, n, 1, c->part, c->dsc, 1, c->st));
  return read_scalar(c, c->dsc);
}

// ------------------------------------------------------------------ operators in precision T
//
// Every operator below takes an epilogue: the value M u is never stored on its own but handed to
// a fused update (store, Chebyshev step, residual update, Jacobi scaling) in the node pass.

template <typename T>
Epi<T> epi_store(T* y) {
  Epi<T> e;
  e.mode = EPI_STORE;
  e.y = y;
  return e;
}

template <typename T>
Epi<T> epi_scale(T* y, const T* sc) {
  Epi<T> e;
  e.mode = EPI_SCALE;
  e.y = y;
  e.sc = sc;
  return e;
}

// y[i] = dinv[i] v per entry (a per-DOF diagonal scaling)
template <typename T>
Epi<T> epi_dinv(T* y, const T* dinv) {
  Epi<T> e;
  e.mode = EPI_DINV;
  e.y = y;
  e.dinv = dinv;
  return e;
}

// Level operator (A for the vector hierarchy, L_c for the scalar ones) with epilogue.
template <typename T>
void level_apply(wbfbt_ctx* c, const Hier<T>& H, const Level<T>& L, const T* u, const Epi<T>& e) {
  T* Ye = prec<T>(c).Ye;
  if (H.vec) {
    CK(launch_apply_vec_epi<T>(L.g, L.k, L.optab, OP_A, u, nullptr, L.coef, L.coef_nodal, Ye, 1, e, c->st));
    return;
  }
  CK(launch_apply_poisson_epi<T>(L.g, L.k, L.optab, u, L.coef, Ye, e, c->st));
}

// epilogue(B^T p) on the fine velocity nodes (Dirichlet nodes 0): element pass + node pass, or the
// single-kernel form on large FP32 levels.  (A node-by-node variant summing the pressure side per
// node was measured slower in the solve.)
template <typename T>
void apply_BT_epi(wbfbt_ctx* c, const T* p, const Epi<T>& e) {
  CK(launch_apply_vec_epi<T>(c->g, c->k, fine_tab<T>(c), OP_BT, nullptr, p, nullptr, 0, prec<T>(c).Ye, 1, e,
                             c->st));
}

// K_w p = B C_w^-1 B^T p with epilogue on the pressure output (which: 0 -> C (w_l), 1 -> D (w_r)).
template <typename T>
void op_Kw(wbfbt_ctx* c, int which, const T* p, const Epi<T>& e) {
  Precond<T>& P = prec<T>(c);
  if (P.Kst[which]) {   // assembled stencil (k <= 3)
    // one kernel reads p at neighbouring elements while the epilogue writes its outputs: an
    // output that is also the input (a Chebyshev direction or iterate) is read from a copy
    const T* src = p;
    if (e.y == p || e.r == p || e.d == p || e.x == p) {
      CK((launch_cast<T, T>((long long)c->g.ne * c->NP, p, P.kwin, c->st)));
      src = P.kwin;
    }
    CK(launch_kw_apply<T>(c->g, c->k, P.Kst[which], src, e, c->st));
    return;
  }
  const T* winv = which == 0 ? P.cinv : P.dinvw;
  apply_BT_epi<T>(c, p, P.wdof ? epi_dinv<T>(P.vtmp, P.wdof) : epi_scale<T>(P.vtmp, winv));
  CK(launch_elem_stokes<T>(c->g, c->k, fine_tab<T>(c), OP_B, P.vtmp, nullptr, nullptr, nullptr, 0, nullptr, e, c->st));
}

// Chebyshev-Jacobi (Saad, Alg. 12.1) over [0.1, 1.1] lambda_hat; M(src, epi) applies the operator
// to src and feeds the result to the epilogue.
template <typename T, class Op>
void chebyshev(wbfbt_ctx* c, Op M, long long n, const T* dinv, double lam, const T* b, T* x, bool zero_guess,
               bool want_res, T* r, T* d) {
  const double lmin = CHEB_LO * lam, lmax = CHEB_HI * lam;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const int steps = c->opt.cheb_degree;
  Epi<T> e;
  e.r = r;
  e.d = d;
  e.x = x;
  e.b = b;
  e.dinv = dinv;
  e.inv_theta = T(1.0 / theta);
  if (zero_guess) {
    CK(launch_cheb_init0<T>(n, b, dinv, T(1.0 / theta), r, d, x, c->st));
  } else {
    e.mode = EPI_CHEB_INIT1;
    M(x, e);
  }
  for (int s = 0; s < steps; ++s) {
    if (s == steps - 1 && !want_res) break;
    if (s == steps - 1) {
      e.mode = EPI_SUB;
      M(d, e);
      break;
    }
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    e.mode = EPI_CHEB_STEP;
    e.a = T(rho_new * rho);
    e.bc = T(2.0 * rho_new / delta);
    M(d, e);
    rho = rho_new;
  }
}

template <typename T>
void vcycle(wbfbt_ctx* c, Hier<T>& H, int l, const T* b, T* x) {
  Level<T>& L = H.lv[l];
  if (L.coarsest) {
    CK(launch_coarse_solve<T>(L.g.nn, H.ncomp, L.map, L.nfree_nodes, L.ndense, L.Ainv, H.vec ? 0 : 1, b, x, L.bf,
                              L.xf, c->st));
    return;
  }
  const long long n = (long long)H.ncomp * L.g.nn;
  auto M = [&](const T* u, const Epi<T>& e) { level_apply<T>(c, H, L, u, e); };
  chebyshev<T>(c, M, n, L.dinv, L.lam, b, x, true, true, L.r, L.d);
  Level<T>& Lc = H.lv[l + 1];
  // Lc.g refined with Lc.k has the node grid of level l: for the p-step (Q_k on N^3 -> Q1 on N^3,
  // k = 2) that is the Q1 grid on (2N)^3, whose nodes are exactly the Q2 nodes, and trilinear
  // interpolation from the N^3 vertices to them is the Q1 -> Q2 embedding
  // (k >= 3: the p-step has its own transfer kernels)
  const bool pstep = Lc.k != L.k && L.k > 2;
  if (pstep)
    CK(launch_p_restrict<T>(Lc.g, L.k, L.dtab, H.ncomp, L.r, Lc.b, H.vec ? 1 : 0, c->st));
  else
    CK(launch_restrict_batched<T>(Lc.g, Lc.k, Lc.optab, H.ncomp, L.r, Lc.b, H.vec ? 1 : 0, L.w1, L.w2, c->st));
  vcycle<T>(c, H, l + 1, Lc.b, Lc.x);
  if (pstep)
    CK(launch_p_prolong<T>(Lc.g, L.k, L.dtab, H.ncomp, Lc.x, x, 1, c->st));
  else
    CK(launch_prolong_fused<T>(Lc.g, Lc.k, Lc.optab, H.ncomp, Lc.x, x, 1, c->st));
  chebyshev<T>(c, M, n, L.dinv, L.lam, b, x, false, false, L.r, L.d);
}

// Two-space pressure-Poisson V-cycle for K_w (Sec. 6): disc smoothing, Q_k correction, disc smoothing.
template <typename T>
void kinv(wbfbt_ctx* c, int which, const T* bd, T* xd) {
  Precond<T>& P = prec<T>(c);
  const long long n = (long long)c->g.ne * c->NP;
  auto M = [&](const T* p, const Epi<T>& e) { op_Kw<T>(c, which, p, e); };
  chebyshev<T>(c, M, n, P.dKw[which], P.lamKw[which], bd, xd, true, true, P.pr, P.pd);
  Level<T>& L0 = P.HL[which].lv[0];
  CK(launch_disc_to_cont_fused<T>(c->g, c->k, fine_tab<T>(c), P.pr, L0.b, P.Ye, c->st));
  vcycle<T>(c, P.HL[which], 0, L0.b, L0.x);
  CK(launch_cont_to_disc_fused<T>(c->g, c->k, fine_tab<T>(c), L0.x, xd, 1, c->st));
  chebyshev<T>(c, M, n, P.dKw[which], P.lamKw[which], bd, xd, false, false, P.pr, P.pd);
}

// ------------------------------------------------------------------ learned correction

__global__ void k_elem_logmu(Grid g, int K, const double* __restrict__ mu, float* __restrict__ out) {
  pdl_entry();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ne) return;
  const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
  const int n = K + 1;
  double s = 0.0;
  for (int l = 0; l < n; ++l)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) s += log10(mu[(K * ex + i) + g.NX * ((K * ey + j) + g.NY * (K * ez + l))]);
  out[e] = (float)(s / (n * n * n) / 4.0);
}

// q = diag(K_w)^-1/2 r   (dK holds diag(K_w)^-1)
template <typename T>
__global__ void k_learn_q(long long n, const T* __restrict__ dK, const T* __restrict__ r, float* __restrict__ q) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = (float)(sqrt((double)dK[i]) * (double)r[i]);
}

// x[e] = (logmu[e], q[e][0..np) / s),  s = ||q|| / sqrt(count)
__global__ void k_learn_pack(int ne, int np, const float* __restrict__ logmu, const float* __restrict__ q,
                             const double* __restrict__ qnorm, long long count, float* __restrict__ x) {
  pdl_entry();
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ne * (np + 1)) return;
  const int e = (int)(t / (np + 1)), c = (int)(t % (np + 1));
  const double s = qnorm[0] / sqrt((double)count);
  x[t] = c == 0 ? logmu[e] : (s > 0.0 ? (float)(q[(size_t)e * np + c - 1] / s) : 0.f);
}

// z = s diag(K_w)^-1/2 y
template <typename T>
__global__ void k_learn_unpack(long long n, const T* __restrict__ dK, const float* __restrict__ y,
                               const double* __restrict__ qnorm, long long count, T* __restrict__ z) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = qnorm[0] / sqrt((double)count);
  z[i] = T(s * sqrt((double)dK[i]) * (double)y[i]);
}

// target y = z / (s diag(K_w)^-1/2)  (0 where the diagonal entry is skipped)
template <typename T>
__global__ void k_learn_target(long long n, const T* __restrict__ dK, const T* __restrict__ z,
                               const double* __restrict__ qnorm, long long count, float* __restrict__ y) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = qnorm[0] / sqrt((double)count);
  const double sc = s * sqrt((double)dK[i]);
  y[i] = sc > 0.0 ? (float)((double)z[i] / sc) : 0.f;
}

inline unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }

// features of residual r into c->lx, ||q|| into dsc[16]
template <typename T>
void learned_features(wbfbt_ctx* c, int which, const T* r, float* x) {
  Precond<T>& P = prec<T>(c);
  const long long n = (long long)c->g.ne * c->NP;
  wb_launch(k_learn_q<T>, nb256(n), 256, 0, c->st, n, P.dKw[which], r, c->lq);
  CK(launch_dot<float, float>(c->lq, c->lq, n, 1, c->part, c->dsc + 16, 1, c->st));
  wb_launch(k_learn_pack, nb256((long long)c->g.ne * (c->NP + 1)), 256, 0, c->st,
      c->g.ne, c->NP, c->llogmu, c->lq, c->dsc + 16, n, x);
  CK(cudaGetLastError());
}

// Learned pressure-Poisson correction with the V-cycle as fallback (kept only if it reduces ||r||).
template <typename T>
void kinv_learned(wbfbt_ctx* c, int which, const T* bd, T* xd) {
  Precond<T>& P = prec<T>(c);
  const long long n = (long long)c->g.ne * c->NP;
  learned_features<T>(c, which, bd, c->lx);
  if (unet_forward_into(c->net, c->lx, c->ly, c->st) != WBFBT_OK) throw WbErr{WBFBT_ERR_CUDA};
  wb_launch(k_learn_unpack<T>, nb256(n), 256, 0, c->st, n, P.dKw[which], c->ly, c->dsc + 16, n, xd);
  CK(cudaGetLastError());
  Epi<T> e;
  e.mode = EPI_BMINUS;
  e.y = P.ptmp;
  e.b = bd;
  op_Kw<T>(c, which, xd, e);
  CK(launch_dot<T, T>(P.ptmp, P.ptmp, n, 1, c->part, c->dsc + 17, 1, c->st));
  CK(launch_dot<T, T>(bd, bd, n, 1, c->part, c->dsc + 18, 1, c->st));
  double nr[2];
  CK(cudaMemcpyAsync(nr, c->dsc + 17, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  // nr holds squared norms: keep z if ||r - K_w z|| < accept ||r||
  if (std::isfinite(nr[0]) && nr[0] < c->net_accept * c->net_accept * nr[1]) {
    ++c->learned_acc;
  } else {
    ++c->learned_rej;
    kinv<T>(c, which, bd, xd);
  }
}

// K~_w^-1: the learned step when a net is attached for this operator, else kinv_cycles
// V-cycles (default 1, Sec. 6); further cycles correct the residual of the current iterate,
// x += V(b - K_w x), so many cycles approach the exact inverse.
template <typename T>
void kinv_any(wbfbt_ctx* c, int which, const T* bd, T* xd) {
  if (c->net && ((c->net_mask >> which) & 1)) {
    kinv_learned<T>(c, which, bd, xd);
    return;
  }
  kinv<T>(c, which, bd, xd);
  Precond<T>& P = prec<T>(c);
  for (int cyc = 1; cyc < c->opt.kinv_cycles; ++cyc) {
    Epi<T> e;
    e.mode = EPI_BMINUS;
    e.y = P.pb;
    e.b = bd;
    op_Kw<T>(c, which, xd, e);                       // pb = b - K_w x
    kinv<T>(c, which, P.pb, P.px);
    CK(launch_axpby<T>((long long)c->g.ne * c->NP, T(1), xd, T(1), P.px, xd, c->st));
  }
}

template <typename T>
void project(wbfbt_ctx* c, const T* src, T* dst) {
  CK(launch_project_pressure<T>(c->g.ne, c->NP, src, dst, c->part, c->dsc + 1, c->st));
}

// y = S~^-1 r (Eq. wbfbt), r and y pressure vectors; with schur = MASS / MASS_DIAG the
// inverse-viscosity pressure mass (Eq. lumping, or its diagonal) instead.
template <typename T>
void schur_inv(wbfbt_ctx* c, const T* r, T* y) {
  Precond<T>& P = prec<T>(c);
  project<T>(c, r, P.sr);
  if (c->opt.schur != WBFBT_SCHUR_WBFBT) {
    CK(launch_block_apply<T>(c->g.ne, c->NP, P.Mp, P.sr, P.sy, c->st));
    project<T>(c, P.sy, y);
    return;
  }
  kinv_any<T>(c, 1, P.sr, P.sy);
  // middle factor B C^-1 A D^-1 B^T y, each diagonal scaling fused into the preceding node pass
  apply_BT_epi<T>(c, P.sy, P.wdof ? epi_dinv<T>(P.sv1, P.wdof) : epi_scale<T>(P.sv1, P.dinvw));
  CK(launch_apply_vec_epi<T>(c->g, c->k, fine_tab<T>(c), OP_A, P.sv1, nullptr, P.mu, 1, P.Ye, 1,
                             P.wdof ? epi_dinv<T>(P.sv2, P.wdof) : epi_scale<T>(P.sv2, P.cinv), c->st));
  CK(launch_elem_stokes<T>(c->g, c->k, fine_tab<T>(c), OP_B, P.sv2, nullptr, nullptr, nullptr, 0, nullptr,
                           epi_store<T>(P.sz), c->st));
  kinv_any<T>(c, 0, P.sz, P.sy2);
  project<T>(c, P.sy2, y);
}

// y = [A~ B^T; 0 s S~]^-1 x (Eq. precond-stokes)
template <typename T>
void precond(wbfbt_ctx* c, const T* x, T* y) {
  Precond<T>& P = prec<T>(c);
  const long long nu = 3LL * c->g.nn;
  const T* xu = x;
  const T* xp = x + nu;
  T* yu = y;
  T* yp = y + nu;
  schur_inv<T>(c, xp, yp);
  if (c->opt.schur_sign < 0) CK(launch_scale<T>((long long)c->g.ne * c->NP, T(-1), yp, yp, c->st));
  // r_u - B^T y_p
  Epi<T> e;
  e.mode = EPI_BMINUS;
  e.y = P.urhs;
  e.b = xu;
  apply_BT_epi<T>(c, yp, e);
  vcycle<T>(c, P.HA, 0, P.urhs, yu);
  // further V-cycles on the residual of the current iterate: y_u += V(b - A y_u)
  Level<T>& L0 = P.HA.lv[0];
  for (int cyc = 1; cyc < c->opt.ainv_cycles && !L0.coarsest; ++cyc) {
    Epi<T> er;
    er.mode = EPI_BMINUS;
    er.y = P.ares;
    er.b = P.urhs;
    level_apply<T>(c, P.HA, L0, yu, er);
    vcycle<T>(c, P.HA, 0, P.ares, P.acor);
    CK(launch_axpby<T>(nu, T(1), yu, T(1), P.acor, yu, c->st));
  }
}

// ------------------------------------------------------------------ setup

// lambda_hat of D^-1 M by 10 power iterations; the normalisation divides by a norm kept in device
// memory, so the only host round trip is the final read.
template <typename T, class Op>
double power_lambda(wbfbt_ctx* c, Op M, long long n, const T* dinv, T* v, T* w, const Grid* mask_grid) {
  double* nrm = c->dsc + 8;
  CK(launch_splitmix_start<T>(n, START_SEED, v, c->st));
  if (mask_grid) CK(launch_mask_boundary<T>(*mask_grid, 3, v, c->st));
  CK(launch_dot<T, T>(v, v, n, 1, c->part, nrm, 1, c->st));
  CK(launch_scale_by_inv<T>(n, nrm, v, v, c->st));
  for (int it = 0; it < POWER_ITERS; ++it) {
    Epi<T> e;
    e.mode = EPI_DINV;
    e.y = w;
    e.dinv = dinv;
    M(v, e);
    CK(launch_dot<T, T>(w, w, n, 1, c->part, nrm, 1, c->st));
    if (it < POWER_ITERS - 1) CK(launch_scale_by_inv<T>(n, nrm, w, v, c->st));
  }
  const double lam = read_scalar(c, nrm);
  if (!(lam > 0.0) || !std::isfinite(lam)) throw WbErr{WBFBT_ERR_SETUP};
  return lam;
}

// Element-kernel family of a grid (the row kernels need enough elements to fill the GPU: one
// thread per element gives a 16^3 level only 4096 threads).
constexpr int ROW_MIN_ELEMS = 20000;
Grid with_kernels(const wbfbt_ctx* c, Grid g) {
  const int mode = c->opt.elem_kernels;
  g.rowk = mode == WBFBT_ELEM_ROW || (mode == WBFBT_ELEM_AUTO && g.ne >= ROW_MIN_ELEMS);
  g.kern = mode;
  return g;
}

Grid coarser(const Grid& g, int k) {
  return make_grid(g.nx / 2, g.ny / 2, g.nz / 2, k, g.h[0] * g.nx, g.h[1] * g.ny, g.h[2] * g.nz);
}

template <typename T>
void build_hier(wbfbt_ctx* c, Hier<T>& H, bool vec, const double* coef0_64, int coef0_nodal) {
  H.vec = vec;
  H.ncomp = vec ? 3 : 1;
  // p-coarsened viscous multigrid (Sec. 6, Fig. 5: p- before h-coarsening): Q_k on the fine mesh,
  // then Q1 on the same mesh and on its h-coarsenings; otherwise fixed-order Q_k h-levels
  const bool pmg = vec && c->opt.pmg && c->k > 1;
  const int nl = c->nlev + (pmg ? 1 : 0);
  H.lv.resize(nl);
  Grid g = c->g;
  int kl = c->k;
  const double* prev_pts = nullptr;   // FP64 per-point coefficient of the previous level
  for (int l = 0; l < nl; ++l) {
    Level<T>& L = H.lv[l];
    L.g = g;
    L.k = kl;
    L.dtab = kl == 1 ? c->dtab1 : c->dtab;
    L.coarsest = (l == nl - 1);
    const size_t npts = (size_t)g.ne * (kl + 1) * (kl + 1) * (kl + 1);
    const size_t nv = (size_t)H.ncomp * g.nn;
    if (l == 0) {
      L.coef64 = const_cast<double*>(coef0_64);
      L.coef_nodal = coef0_nodal;
      if (coef0_nodal) {
        c->pool.ensure(L.pts64, npts);   // per-point FP64 copy for coarsening
        CK(launch_nodal_to_points<double>(g, c->k, coef0_64, L.pts64, c->st));
        prev_pts = L.pts64;
      } else {
        prev_pts = coef0_64;
      }
    } else {
      c->pool.ensure(L.pts64, npts);
      const Level<T>& Lf = H.lv[l - 1];
      if (Lf.k != L.k)   // the p-step: Q_k points -> Q1 points on the same elements
        CK(launch_pcoarsen_coef(Lf.g, Lf.k, Lf.dtab, prev_pts, L.pts64, c->st));
      else
        CK(launch_coarsen_coef<double>(Lf.g, L.k, L.dtab, prev_pts, L.pts64, c->st));
      L.coef64 = L.pts64;
      L.coef_nodal = 0;
      prev_pts = L.pts64;
    }
    // coefficient in T
    if (std::is_same<T, double>::value) {
      L.coef = reinterpret_cast<const T*>(L.coef64);
    } else {
      size_t nc = L.coef_nodal ? (size_t)g.nn : npts;
      c->pool.ensure(L.coefT, nc);
      CK((launch_cast<double, T>((long long)nc, L.coef64, L.coefT, c->st)));
      L.coef = L.coefT;
    }
    c->pool.ensure(L.b, nv);
    c->pool.ensure(L.x, nv);
    if (!L.optab) L.optab = make_device_optab<T>(c, g, kl);
    if (!L.coarsest) {
      c->pool.ensure(L.r, nv);
      c->pool.ensure(L.d, nv);
      c->pool.ensure(L.tmp, nv);
      c->pool.ensure(L.dinv, nv);
      c->pool.ensure(L.d64, nv);
      if (vec)
        CK(launch_dinv_A<double>(g, L.k, L.dtab, L.coef64, L.coef_nodal, L.d64, c->st));
      else
        CK(launch_dinv_L<double>(g, L.k, L.dtab, L.coef64, L.d64, c->st));
      CK((launch_cast<double, T>((long long)nv, L.d64, L.dinv, c->st)));
      // the next level: Q1 on this mesh after the fine level of a p-coarsened hierarchy, else the
      // h-coarsening of this mesh at this level's order
      const int kc = (pmg && l == 0) ? 1 : kl;
      Grid gc = (pmg && l == 0) ? make_grid(g.nx, g.ny, g.nz, 1, g.h[0] * g.nx, g.h[1] * g.ny, g.h[2] * g.nz)
                                : coarser(g, kc);
      gc = with_kernels(c, gc);
      size_t ws = transfer_work_size(gc, kc);
      c->pool.ensure(L.w1, ws * H.ncomp);   // restriction passes run all components at once
      c->pool.ensure(L.w2, ws * H.ncomp);
      c->pool.ensure(L.pv, nv);
      c->pool.ensure(L.pw, nv);
      auto M = [&](const T* u, const Epi<T>& e) { level_apply<T>(c, H, L, u, e); };
      L.lam = power_lambda<T>(c, M, (long long)nv, L.dinv, L.pv, L.pw, vec ? &L.g : nullptr);
      g = gc;
      kl = kc;
    } else {
      // coarsest: dense FP64 matrix over the free DOFs, explicit inverse
      std::vector<int> hmap(g.nn);
      int nfree = 0;
      for (int n = 0; n < g.nn; ++n) {
        int ix = n % g.NX, iy = (n / g.NX) % g.NY, iz = n / (g.NX * g.NY);
        hmap[n] = (vec && on_boundary(g, ix, iy, iz)) ? -1 : nfree++;
      }
      const int nd = H.ncomp * nfree;
      if (nd > MAX_DENSE) throw WbErr{WBFBT_ERR_INVALID};
      L.nfree_nodes = nfree;
      L.ndense = nd;
      if (!L.map) {
        c->pool.ensure(L.map, g.nn);
        CK(cudaMemcpyAsync(L.map, hmap.data(), sizeof(int) * g.nn, cudaMemcpyHostToDevice, c->st));
        CK(cudaStreamSynchronize(c->st));   // hmap is a stack-local host buffer
      }
      c->pool.ensure(L.Md, (size_t)nd * nd);
      c->pool.ensure(L.bf, nd);
      c->pool.ensure(L.xf, nd);
      CK(cudaMemsetAsync(L.Md, 0, sizeof(double) * (size_t)nd * nd, c->st));
      if (vec)
        CK(launch_assemble_dense_A(g, L.k, L.dtab, L.coef64, L.coef_nodal, L.map, nfree, L.Md, nd, c->st));
      else
        CK(launch_assemble_dense_L_mapped(g, L.k, L.dtab, L.coef64, L.map, L.Md, nd, c->st));
      L.Ainv = L.Md;   // inverted in place by run_dense_jobs once every hierarchy is assembled
      c->dense_jobs.push_back({L.Md, nd, vec ? 0 : 1});
    }
  }
}

// Invert every coarsest matrix assembled in this setup, all in one blocked Gauss-Jordan sweep.
void run_dense_jobs(wbfbt_ctx* c) {
  const int cnt = (int)c->dense_jobs.size();
  if (cnt == 0) return;
  if (cnt > 4) throw WbErr{WBFBT_ERR_INVALID};
  double* M[4];
  int n[4], pin[4];
  for (int z = 0; z < cnt; ++z) {
    M[z] = c->dense_jobs[z].M;
    n[z] = c->dense_jobs[z].n;
    pin[z] = c->dense_jobs[z].pin;
  }
  c->pool.ensure(c->gj_work, (size_t)4 * 32 * 32);
  CK(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st));
  CK(launch_dense_inverse_batch(cnt, M, n, pin, c->gj_work, c->dflag, c->st));
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->dense_jobs.clear();
  if (flag) throw WbErr{WBFBT_ERR_SETUP};
}

template <typename T>
void build_precond(wbfbt_ctx* c) {
  Precond<T>& P = prec<T>(c);
  c->dense_jobs.clear();
  const Grid& g = c->g;
  const size_t nn = g.nn, nu = 3 * nn, np = (size_t)g.ne * c->NP, npts = (size_t)g.ne * c->N3;
  if (std::is_same<T, double>::value) {
    P.mu = reinterpret_cast<T*>(c->mu64);
    P.cinv = reinterpret_cast<T*>(c->cinv64);
    P.dinvw = reinterpret_cast<T*>(c->dinv64);
  } else {
    P.mu = reinterpret_cast<T*>(c->mu32);
    c->pool.ensure(P.cinv, nn);
    c->pool.ensure(P.dinvw, nn);
    CK((launch_cast<double, T>((long long)nn, c->cinv64, P.cinv, c->st)));
    CK((launch_cast<double, T>((long long)nn, c->dinv64, P.dinvw, c->st)));
  }
  const bool diag_a = c->opt.weights == WBFBT_WEIGHTS_DIAG_A;
  if (diag_a) {   // diag(A)-BFBT: C = D = diag(A) per DOF (Sec. 1.3)
    if (std::is_same<T, double>::value) {
      P.wdof = reinterpret_cast<T*>(c->adinv64);
    } else {
      c->pool.ensure(P.wdof, nu);
      CK((launch_cast<double, T>((long long)nu, c->adinv64, P.wdof, c->st)));
    }
  }
  for (T** q : {&P.pb, &P.px, &P.pr, &P.pd, &P.ptmp, &P.sr, &P.sy, &P.sz, &P.sy2}) c->pool.ensure(*q, np);
  for (T** q : {&P.vtmp, &P.sv1, &P.sv2, &P.urhs, &P.utmp}) c->pool.ensure(*q, nu);
  if (c->opt.ainv_cycles > 1)
    for (T** q : {&P.ares, &P.acor}) c->pool.ensure(*q, nu);
  c->pool.ensure(P.vin, c->ntot);
  c->pool.ensure(P.vout, c->ntot);
  {
    // element-pass scratch: the largest any level's element pass writes
    size_t ye = 0;
    Grid gl = g;
    for (int l = 0; l < c->nlev; ++l) {
      ye = std::max(ye, elem_scratch_size<T>(gl, c->k));
      if (l + 1 < c->nlev) gl = with_kernels(c, coarser(gl, c->k));
    }
    c->pool.ensure(P.Ye, ye);
  }
  // A hierarchy: viscosity per node on the fine level
  build_hier<T>(c, P.HA, true, c->mu64, 1);
  // Poisson hierarchies: c = 1 / (a(e) sqrt(mu)) per point
  const double amp[2] = {c->opt.a_l, c->opt.a_r};
  for (int wi = 0; wi < 2; ++wi) {
    c->pool.ensure(P.c0[wi], npts);
    if (c->opt.weights == WBFBT_WEIGHTS_GRAD)
      CK(launch_poisson_coef_pts<double>(g, c->k, c->wpts, amp[wi], P.c0[wi], c->st));
    else if (diag_a)   // the Poisson surrogate of B diag(A)^-1 B^T: coefficient 1/mu (weight mu)
      CK(launch_poisson_coef_pts<double>(g, c->k, c->wpts, 1.0, P.c0[wi], c->st));
    else
      CK(launch_poisson_coef0<double>(g, c->k, c->mu64, amp[wi], P.c0[wi], c->st));
    build_hier<T>(c, P.HL[wi], false, P.c0[wi], 0);
    // disc level: Jacobi diagonal of K_w and lambda_hat
    c->pool.ensure(P.dK64[wi], np);
    if (diag_a)
      CK(launch_dinv_Kw<double>(g, c->k, c->dtab, c->adinv64, 1, P.dK64[wi], c->st));
    else if (c->kwbref)
      CK(launch_kw_dinv<double>(g, c->k, c->kwbref, wi == 0 ? c->cinv64 : c->dinv64, P.dK64[wi], c->st));
    else
      CK(launch_dinv_Kw<double>(g, c->k, c->dtab, wi == 0 ? c->cinv64 : c->dinv64, 0, P.dK64[wi], c->st));
    c->pool.ensure(P.dKw[wi], np);
    CK((launch_cast<double, T>((long long)np, P.dK64[wi], P.dKw[wi], c->st)));
    // FP64 preconditioners apply K_w as an assembled stencil (one memory-bound pass instead of
    // three FP64-bound element/node passes: 3x faster at 32^3 Q2); single precision keeps the
    // matrix-free row kernels, which move fewer bytes (the stencil is 27 Np^2 words per element)
    if (c->kwbref && std::is_same<T, double>::value && !diag_a) {
      c->pool.ensure(P.Kst[wi], kw_stencil_entries(g, c->k));
      c->pool.ensure(P.kwin, np);
      CK(launch_kw_assemble<T>(g, c->k, c->kwbref, wi == 0 ? c->cinv64 : c->dinv64, P.Kst[wi], c->st));
    }
    auto M = [&](const T* p, const Epi<T>& e) { op_Kw<T>(c, wi, p, e); };
    P.lamKw[wi] = power_lambda<T>(c, M, (long long)np, P.dKw[wi], P.px, P.pd, nullptr);
  }
  if (c->opt.schur != WBFBT_SCHUR_WBFBT) {
    const size_t nb = (size_t)g.ne * c->NP * c->NP;
    c->pool.ensure(c->Mp64, nb);
    CK(launch_mass_lumped_inv(g, c->k, c->dtab, c->mu64, c->opt.schur == WBFBT_SCHUR_MASS_DIAG ? 1 : 0,
                              c->Mp64, c->st));
    if (std::is_same<T, double>::value) {
      P.Mp = reinterpret_cast<T*>(c->Mp64);
    } else {
      c->pool.ensure(P.Mp, nb);
      CK((launch_cast<double, T>((long long)nb, c->Mp64, P.Mp, c->st)));
    }
  }
  run_dense_jobs(c);
}

__global__ void k_inv_masked(Grid g, const double* __restrict__ w, double* __restrict__ inv) {
  pdl_entry();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int ix = n % g.NX, iy = (n / g.NX) % g.NY, iz = n / (g.NX * g.NY);
  inv[n] = on_boundary(g, ix, iy, iz) ? 0.0 : 1.0 / w[n];
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int n_levels(int nx, int ny, int nz, int min_n) {
  int L = 1;
  while (nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0 && std::min(nx, std::min(ny, nz)) > min_n) {
    nx /= 2; ny /= 2; nz /= 2;
    ++L;
  }
  return L;
}

template <class F>
int guarded(F f) {
  try {
    f();
    return WBFBT_OK;
  } catch (const WbErr& e) {
    return e.code;
  } catch (...) {
    return WBFBT_ERR_CUDA;
  }
}

// Runs f on the context's internal stream, ordered after all prior work on the caller's stream,
// and makes the caller's stream wait for it.
template <class F>
int guarded_ctx(wbfbt_ctx* c, F f) {
  if (cudaEventRecord(c->ev_in, c->ust) != cudaSuccess || cudaStreamWaitEvent(c->st, c->ev_in, 0) != cudaSuccess)
    return WBFBT_ERR_CUDA;
  int r = guarded(f);
  if (cudaEventRecord(c->ev_out, c->st) != cudaSuccess || cudaStreamWaitEvent(c->ust, c->ev_out, 0) != cudaSuccess)
    return r != WBFBT_OK ? r : WBFBT_ERR_CUDA;
  return r;
}

// ------------------------------------------------------------------ FGMRES

void apply_K64(wbfbt_ctx* c, const double* x, double* y) {
  const long long nu = 3LL * c->g.nn;
  if (c->mapped) {
    CK(launch_mapped_stokes<double>(c->g, c->k, c->rt64, c->X64, OP_A | OP_BT | OP_B, x, x + nu, c->mu64, 1, c->Ye64,
                                    epi_store<double>(y), epi_store<double>(y + nu), c->dflag, c->st));
    return;
  }
  CK(launch_elem_stokes<double>(c->g, c->k, c->ot64, OP_A | OP_BT | OP_B, x, nullptr, x + nu, c->mu64, 1, c->Ye64,
                                epi_store<double>(y + nu), c->st));
  CK(launch_gather<double>(c->g, c->k, 3, 1, c->Ye64, epi_store<double>(y), c->st));
}

template <typename T>
void precond_graphed(wbfbt_ctx* c, const double* v, double* z) {
  Precond<T>& P = prec<T>(c);
  if (c->pgraph == nullptr || c->graph_dirty) {
    if (c->pgraph) {
      cudaGraphExecDestroy(c->pgraph);
      c->pgraph = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const long long n0 = wb_launch_counter().load();
    CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    try {
      precond<T>(c, P.vin, P.vout);
    } catch (...) {
      cudaStreamEndCapture(c->st, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    CK(cudaStreamEndCapture(c->st, &graph));
    const cudaError_t e = cudaGraphInstantiate(&c->pgraph, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    c->graph_kernels = wb_launch_counter().load() - n0;
    wb_launch_counter().fetch_sub(c->graph_kernels);   // captured, not run
    c->graph_dirty = false;
  }
  CK((launch_cast<double, T>(c->ntot, v, P.vin, c->st)));
  CK(cudaGraphLaunch(c->pgraph, c->st));
  wb_launch_counter().fetch_add(c->graph_kernels);
  CK((launch_cast<T, double>(c->ntot, P.vout, z, c->st)));
}

// w = K z inside the Arnoldi process.  FP64 by default (the exact Arnoldi relation).  With the
// mixed-precision option arnoldi_precision = WBFBT_F32 the fused K apply runs in FP32 on the
// preconditioner's FP32 output (z_j is exactly that vector widened), so the FP64 element pass
// leaves the iteration; the true residual F - K x at every restart and at exit stays FP64, and
// the solve ends only when that residual meets the tolerance.
void apply_K_arnoldi(wbfbt_ctx* c, const double* z, double* w) {
  if (!(c->mixed && c->opt.arnoldi_precision == WBFBT_F32)) {
    apply_K64(c, z, w);
    return;
  }
  Precond<float>& P = c->P32;
  const long long nu = 3LL * c->g.nn;
  if (c->mapped) {
    CK(launch_mapped_stokes<float>(c->g, c->k, c->rt32, c->X32, OP_A | OP_BT | OP_B, P.vout, P.vout + nu, c->mu32, 1,
                                   c->Ye32, epi_store<float>(P.vin), epi_store<float>(P.vin + nu), c->dflag, c->st));
  } else {
    CK(launch_elem_stokes<float>(c->g, c->k, c->ot32, OP_A | OP_BT | OP_B, P.vout, nullptr, P.vout + nu, c->mu32, 1,
                                 c->Ye32, epi_store<float>(P.vin + nu), c->st));
    CK(launch_gather<float>(c->g, c->k, 3, 1, c->Ye32, epi_store<float>(P.vin), c->st));
  }
  CK((launch_cast<float, double>(c->ntot, P.vin, w, c->st)));
}

void precond_any(wbfbt_ctx* c, const double* v, double* z) {
  if (c->opt.use_graphs && c->net == nullptr) {
    if (c->mixed)
      precond_graphed<float>(c, v, z);
    else
      precond_graphed<double>(c, v, z);
  } else if (!c->mixed) {
    precond<double>(c, v, z);
  } else {
    CK((launch_cast<double, float>(c->ntot, v, c->P32.vin, c->st)));
    precond<float>(c, c->P32.vin, c->P32.vout);
    CK((launch_cast<float, double>(c->ntot, c->P32.vout, z, c->st)));
  }
}

// Right-preconditioned FGMRES(m) on vectors of length n <= ntot (Sec. 1.3): x0 = 0, CGS2
// orthogonalisation and the Hessenberg/Givens recurrence in FP64, the true residual F - K x
// recomputed in FP64 at every restart and at exit.  arn(z, w): w = K z inside the Arnoldi
// process; tru(x, w): w = K x for the true residual; pc(v, z): z = P^-1 v.
template <class Arn, class Tru, class Pc>
int fgmres_core(wbfbt_ctx* c, long long n, const double* F, double* x, double* r, Arn arn, Tru tru, Pc pc,
                double rtol, int maxit, int* iters, double* relres) {
  const int m = c->m;
  CK(cudaMemsetAsync(x, 0, sizeof(double) * n, c->st));
  CK(cudaMemcpyAsync(r, F, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
  const double beta0 = norm<double>(c, r, n);
  if (!std::isfinite(beta0)) return WBFBT_ERR_NONFINITE;
  if (beta0 == 0.0) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return WBFBT_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m), hcol(2 * (m + 1) + 1);
  int its = 0;
  double rel = 1.0;
  bool done = false;
  int status = WBFBT_OK;
  while (!done) {
    const double beta = norm<double>(c, r, n);
    CK(launch_scale<double>(n, 1.0 / beta, r, c->V, c->st));
    std::fill(gv.begin(), gv.end(), 0.0);
    std::fill(H.begin(), H.end(), 0.0);
    gv[0] = beta;
    int jdone = 0;
    bool converged = false;
    for (int j = 0; j < m; ++j) {
      double* vj = c->V + (size_t)j * n;
      double* zj = c->Z + (size_t)j * n;
      pc(vj, zj);
      arn(zj, c->w);
      // CGS2: h = V^T w, w -= V h, twice.  (A second pass only when the first shrank w below
      // 1/sqrt(2) of its norm was measured slower: with a good preconditioner K z_j is close to
      // v_j, the first projection removes most of w, and the test asked for the second pass
      // almost every step, at the cost of an extra host synchronisation.)
      double* h1 = c->hdev;
      double* h2 = c->hdev + (m + 1);
      double* hn = c->hdev + 2 * (m + 1);
      CK(launch_mdot(c->V, n, j + 1, c->w, n, c->part, h1, c->st));
      CK(launch_gemv_sub(c->V, n, j + 1, h1, c->w, n, c->st));
      CK(launch_mdot(c->V, n, j + 1, c->w, n, c->part, h2, c->st));
      CK(launch_gemv_sub(c->V, n, j + 1, h2, c->w, n, c->st));
      CK(launch_dot<double, double>(c->w, c->w, n, 1, c->part, hn, 1, c->st));
      CK(cudaMemcpyAsync(hcol.data(), c->hdev, sizeof(double) * (2 * (m + 1) + 1), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      const double hnrm = hcol[2 * (m + 1)];
      for (int i = 0; i <= j; ++i) {
        const double hv = hcol[i] + hcol[(m + 1) + i];
        if (!std::isfinite(hv)) return WBFBT_ERR_NONFINITE;
        H[(size_t)i * m + j] = hv;
      }
      if (!std::isfinite(hnrm)) return WBFBT_ERR_NONFINITE;
      H[(size_t)(j + 1) * m + j] = hnrm;
      if (hnrm > 0.0) CK(launch_scale<double>(n, 1.0 / hnrm, c->w, c->V + (size_t)(j + 1) * n, c->st));
      for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
      }
      const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
      const double den = std::hypot(a, b);
      if (!(den > 0.0)) return WBFBT_ERR_BREAKDOWN;
      cs[j] = a / den;
      sn[j] = b / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++its;
      jdone = j + 1;
      if (std::fabs(gv[j + 1]) <= rtol * beta0 || its >= maxit || hnrm == 0.0) {
        converged = std::fabs(gv[j + 1]) <= rtol * beta0;
        break;
      }
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double s = gv[i];
      for (int k2 = i + 1; k2 < jdone; ++k2) s -= H[(size_t)i * m + k2] * y[k2];
      y[i] = s / H[(size_t)i * m + i];
    }
    CK(cudaMemcpyAsync(c->hdev, y.data(), sizeof(double) * jdone, cudaMemcpyHostToDevice, c->st));
    CK(launch_gemv_add(c->Z, n, jdone, c->hdev, x, n, c->st));
    tru(x, c->w);
    CK(launch_axpby<double>(n, 1.0, F, -1.0, c->w, r, c->st));
    rel = norm<double>(c, r, n) / beta0;
    if (!std::isfinite(rel)) return WBFBT_ERR_NONFINITE;
    if ((converged && rel <= rtol) || its >= maxit) done = true;
  }
  if (rel > rtol) status = WBFBT_ERR_MAXIT;
  if (iters) *iters = its;
  if (relres) *relres = rel;
  return status;
}

// The Stokes solve: K = [A B^T; B 0], P = the block preconditioner of Eq. precond-stokes.
int fgmres(wbfbt_ctx* c, double rtol, int maxit, int* iters, double* relres) {
  return fgmres_core(
      c, c->ntot, c->F, c->x, c->r, [&](const double* z, double* w) { apply_K_arnoldi(c, z, w); },
      [&](const double* xx, double* w) { apply_K64(c, xx, w); }, [&](const double* v, double* z) { precond_any(c, v, z); },
      rtol, maxit, iters, relres);
}

// One block of the preconditioner solved on its own (Table 3's "alone" counts): the viscous
// block A with its V-cycle, or K_w = B C_w^-1 B^T (which 0: w_l, 1: w_r) with its two-space
// V-cycle, both as right preconditioners of FGMRES.  The V-cycles run in the context's
// preconditioner precision T (FP64, or FP32 in a mixed context), the Krylov vectors in FP64; the
// operator is FP64 for A and in precision T for K_w.
template <typename T>
int block_solve(wbfbt_ctx* c, int block, long long n, double rtol, int maxit, int* iters, double* relres) {
  Precond<T>& P = prec<T>(c);
  T* tin = std::is_same<T, double>::value ? nullptr : P.vin;
  T* tout = std::is_same<T, double>::value ? nullptr : P.vout;
  // run f on T views of a (in) and b (out): direct for FP64, through casts for FP32
  auto via = [&](const double* a, double* b, auto f) {
    if (std::is_same<T, double>::value) {
      f(reinterpret_cast<const T*>(a), reinterpret_cast<T*>(b));
    } else {
      CK((launch_cast<double, T>(n, a, tin, c->st)));
      f(tin, tout);
      CK((launch_cast<T, double>(n, tout, b, c->st)));
    }
  };
  if (block == 0) {
    // the operator in FP64 in every context: an FP32 A caps the attainable residual of the
    // ill-conditioned viscous block near eps_32 kappa(A) (measured 3e-5 at 8^3, DR 1e4)
    auto op = [&](const double* z, double* w) {
      CK(launch_elem_stokes<double>(c->g, c->k, c->ot64, OP_A, z, nullptr, nullptr, c->mu64, 1, c->Ye64,
                                    Epi<double>(), c->st));
      CK(launch_gather<double>(c->g, c->k, 3, 1, c->Ye64, epi_store<double>(w), c->st));
    };
    auto pc = [&](const double* v, double* z) {
      via(v, z, [&](const T* vi, T* zo) { vcycle<T>(c, P.HA, 0, vi, zo); });
    };
    return fgmres_core(c, n, c->F, c->x, c->r, op, op, pc, rtol, maxit, iters, relres);
  }
  const int which = block - 1;
  auto op = [&](const double* z, double* w) {
    via(z, w, [&](const T* zi, T* wo) { op_Kw<T>(c, which, zi, epi_store<T>(wo)); });
  };
  auto pc = [&](const double* v, double* z) {
    via(v, z, [&](const T* vi, T* zo) {
      project<T>(c, vi, P.sr);
      kinv_any<T>(c, which, P.sr, P.sy);
      project<T>(c, P.sy, zo);
    });
  };
  return fgmres_core(c, n, c->F, c->x, c->r, op, op, pc, rtol, maxit, iters, relres);
}

}  // namespace

namespace {

__global__ void k_check_positive(long long n, const double* __restrict__ v, int* __restrict__ flag) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (!(v[i] > 0.0) || !isfinite(v[i]))) atomicExch(flag, 1);
}

// Everything that depends on the viscosity: weights, hierarchies, diagonals, eigenvalue
// estimates, coarsest inverses.  Allocates only on the first call for a context.
void run_setup(wbfbt_ctx* cp, const double* mu_nodes) {
  const Grid& g = cp->g;
  const size_t nn = g.nn;
  CK(cudaMemcpyAsync(cp->mu64, mu_nodes, sizeof(double) * nn, cudaMemcpyDefault, cp->st));
  CK(cudaMemsetAsync(cp->dflag, 0, sizeof(int), cp->st));
  wb_launch(k_check_positive, (unsigned)((nn + 255) / 256), 256, 0, cp->st, (long long)nn, cp->mu64, cp->dflag);
  CK(cudaGetLastError());
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, cp->dflag, sizeof(int), cudaMemcpyDeviceToHost, cp->st));
  CK(cudaStreamSynchronize(cp->st));
  if (bad) throw WbErr{WBFBT_ERR_INVALID};
  CK((launch_cast<double, float>((long long)nn, cp->mu64, cp->mu32, cp->st)));
  if (cp->opt.weights == WBFBT_WEIGHTS_GRAD) {
    // viscosity-gradient weights (remark in Sec. 4): per element point, then lumped per node
    cp->pool.ensure(cp->wpts, (size_t)g.ne * cp->N3);
    CK(launch_weight_points(g, cp->k, cp->dtab, cp->mu64, 1, cp->wpts, cp->st));
    CK(launch_lumped_weight_pts(g, cp->k, cp->dtab, cp->wpts, cp->opt.a_l, cp->C, cp->st));
    CK(launch_lumped_weight_pts(g, cp->k, cp->dtab, cp->wpts, cp->opt.a_r, cp->D, cp->st));
  } else {
    CK(launch_lumped_weight(g, cp->k, cp->dtab, cp->mu64, cp->opt.a_l, cp->C, cp->st));
    CK(launch_lumped_weight(g, cp->k, cp->dtab, cp->mu64, cp->opt.a_r, cp->D, cp->st));
  }
  if (cp->opt.weights == WBFBT_WEIGHTS_DIAG_A) {
    // diag(A)-BFBT: diag(A)^-1 per DOF in FP64, and mu per point for the Poisson surrogate
    cp->pool.ensure(cp->adinv64, 3 * nn);
    CK(launch_dinv_A<double>(g, cp->k, cp->dtab, cp->mu64, 1, cp->adinv64, cp->st));
    cp->pool.ensure(cp->wpts, (size_t)g.ne * cp->N3);
    CK(launch_nodal_to_points<double>(g, cp->k, cp->mu64, cp->wpts, cp->st));
  }
  wb_launch(k_inv_masked, (unsigned)((nn + 255) / 256), 256, 0, cp->st, g, cp->C, cp->cinv64);
  wb_launch(k_inv_masked, (unsigned)((nn + 255) / 256), 256, 0, cp->st, g, cp->D, cp->dinv64);
  CK(cudaGetLastError());
  if (cp->mixed)
    build_precond<float>(cp);
  else
    build_precond<double>(cp);
  cp->graph_dirty = true;   // Chebyshev coefficients are baked into the captured launches
  wb_launch(k_elem_logmu, (unsigned)((g.ne + 127) / 128), 128, 0, cp->st, g, cp->k, cp->mu64, cp->llogmu);
  CK(cudaGetLastError());
}

}  // namespace

namespace {

template <typename T>
void stokes_apply_t(wbfbt_ctx* c, int ops, const T* u, const T* p, T* yu, T* yp, const T* mu, T* Ye) {
  if (c->mapped) {
    const bool dbl = std::is_same<T, double>::value;
    CK(launch_mapped_stokes<T>(c->g, c->k, dbl ? c->rt64 : c->rt32,
                               dbl ? (const T*)(const void*)c->X64 : (const T*)(const void*)c->X32, ops, u, p, mu, 1,
                               Ye, epi_store<T>(yu), epi_store<T>(yp), c->dflag, c->st));
    return;
  }
  if (ops == OP_A || ops == OP_BT) {
    CK(launch_apply_vec_epi<T>(c->g, c->k, fine_tab<T>(c), ops, u, p, mu, 1, Ye, 1, epi_store<T>(yu), c->st));
    return;
  }
  const bool scat = (ops & OP_A) || (ops & OP_BT);
  CK(launch_elem_stokes<T>(c->g, c->k, fine_tab<T>(c), ops, u, nullptr, p, mu, 1, Ye, epi_store<T>(yp), c->st));
  if (scat) CK(launch_gather<T>(c->g, c->k, 3, 1, Ye, epi_store<T>(yu), c->st));
}

}  // namespace

// ================================================================== C ABI

extern "C" {

void wbfbt_default_opts(wbfbt_opts* o) {
  if (!o) return;
  o->a_l = 1.0;
  o->a_r = 0.0;
  o->restart = 50;
  o->cheb_degree = 3;
  o->mg_min_n = 4;
  o->precision = WBFBT_F64;
  o->schur_sign = -1;
  o->use_graphs = 1;
  o->elem_kernels = WBFBT_ELEM_AUTO;
  o->schur = WBFBT_SCHUR_WBFBT;
  o->arnoldi_precision = WBFBT_F64;
  o->weights = WBFBT_WEIGHTS_SQRT_MU;
  o->kinv_cycles = 1;
  o->ainv_cycles = 1;
  o->pmg = 0;
}

const char* wbfbt_status_string(int s) {
  switch (s) {
    case WBFBT_OK: return "ok";
    case WBFBT_ERR_INVALID: return "invalid argument";
    case WBFBT_ERR_CUDA: return "CUDA runtime error";
    case WBFBT_ERR_NONFINITE: return "non-finite value in a residual or Krylov coefficient";
    case WBFBT_ERR_BREAKDOWN: return "Krylov breakdown";
    case WBFBT_ERR_MAXIT: return "iteration limit reached before the tolerance";
    case WBFBT_ERR_SETUP: return "setup failed (coarse matrix not SPD or bad eigenvalue estimate)";
    default: return "unknown status";
  }
}

static bool mesh_ok(const wbfbt_mesh* m, int k) {
  return m && k >= 2 && k <= 4 && m->nx >= 1 && m->ny >= 1 && m->nz >= 1 && m->lx > 0 && m->ly > 0 && m->lz > 0 &&
         (long long)(k * m->nx + 1) * (k * m->ny + 1) * (k * m->nz + 1) < (1LL << 30);
}

int wbfbt_sinker_setup(const wbfbt_mesh* mesh, int k, const double* centres, int ns, double omega, double delta,
                       double dr, double beta, double* mu_out, double* f_out, void* stream) {
  if (!mesh_ok(mesh, k) || (!centres && ns > 0) || ns < 0 || ns > 128 || !mu_out || !(dr >= 1.0)) return WBFBT_ERR_INVALID;
  RefTables t;
  if (!build_ref_tables(k, &t)) return WBFBT_ERR_INVALID;
  Grid g = make_grid(mesh->nx, mesh->ny, mesh->nz, k, mesh->lx, mesh->ly, mesh->lz);
  cudaError_t e = launch_sinker(g, k, t, centres, ns, omega, delta, dr, beta, mu_out, f_out, (cudaStream_t)stream);
  return e == cudaSuccess ? WBFBT_OK : WBFBT_ERR_CUDA;
}

int wbfbt_sinker_setup_at(const wbfbt_mesh* mesh, int k, const double* X_nodes, const double* centres, int ns,
                          double omega, double delta, double dr, double beta, double* mu_out, double* f_out,
                          void* stream) {
  if (!mesh_ok(mesh, k) || !X_nodes || (!centres && ns > 0) || ns < 0 || ns > 128 || !mu_out || !(dr >= 1.0))
    return WBFBT_ERR_INVALID;
  if (!is_device_ptr(X_nodes) || !is_device_ptr(mu_out) || (f_out && !is_device_ptr(f_out))) return WBFBT_ERR_INVALID;
  RefTables t;
  if (!build_ref_tables(k, &t)) return WBFBT_ERR_INVALID;
  Grid g = make_grid(mesh->nx, mesh->ny, mesh->nz, k, mesh->lx, mesh->ly, mesh->lz);
  cudaError_t e = launch_sinker(g, k, t, centres, ns, omega, delta, dr, beta, mu_out, f_out, (cudaStream_t)stream,
                                X_nodes);
  return e == cudaSuccess ? WBFBT_OK : WBFBT_ERR_CUDA;
}

int wbfbt_node_coords(const wbfbt_mesh* mesh, int k, double* X_out, void* stream) {
  if (!mesh_ok(mesh, k) || !X_out || !is_device_ptr(X_out)) return WBFBT_ERR_INVALID;
  RefTables t;
  if (!build_ref_tables(k, &t)) return WBFBT_ERR_INVALID;
  Grid g = make_grid(mesh->nx, mesh->ny, mesh->nz, k, mesh->lx, mesh->ly, mesh->lz);
  cudaError_t e = launch_node_coords(g, k, t, X_out, (cudaStream_t)stream);
  return e == cudaSuccess ? WBFBT_OK : WBFBT_ERR_CUDA;
}

int wbfbt_create(const wbfbt_mesh* mesh, int k, const double* mu_nodes, const wbfbt_opts* opts, void* stream,
                 wbfbt_ctx** out) {
  if (!out || !mu_nodes || !mesh_ok(mesh, k)) return WBFBT_ERR_INVALID;
  *out = nullptr;
  auto c = std::make_unique<wbfbt_ctx>();
  wbfbt_default_opts(&c->opt);
  if (opts) c->opt = *opts;
  if (c->opt.restart < 1 || c->opt.restart > 1000 || c->opt.cheb_degree < 1 || c->opt.cheb_degree > 16 ||
      c->opt.a_l < 1.0 || (c->opt.a_r > 0 && c->opt.a_r < 1.0) ||
      (c->opt.precision != WBFBT_F64 && c->opt.precision != WBFBT_MIXED) || c->opt.mg_min_n < 1 ||
      c->opt.elem_kernels < WBFBT_ELEM_AUTO || c->opt.elem_kernels > WBFBT_ELEM_ROW ||
      c->opt.schur < WBFBT_SCHUR_WBFBT || c->opt.schur > WBFBT_SCHUR_MASS_DIAG ||
      (c->opt.arnoldi_precision != WBFBT_F64 && c->opt.arnoldi_precision != WBFBT_F32) ||
      (c->opt.arnoldi_precision == WBFBT_F32 && c->opt.precision != WBFBT_MIXED) ||
      c->opt.weights < WBFBT_WEIGHTS_SQRT_MU || c->opt.weights > WBFBT_WEIGHTS_DIAG_A ||
      c->opt.kinv_cycles < 1 || c->opt.kinv_cycles > 64 || (c->opt.pmg != 0 && c->opt.pmg != 1) ||
      c->opt.ainv_cycles < 1 || c->opt.ainv_cycles > 64)
    return WBFBT_ERR_INVALID;
  if (c->opt.schur_sign >= 0) c->opt.schur_sign = 1; else c->opt.schur_sign = -1;
  c->ust = (cudaStream_t)stream;
  if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return WBFBT_ERR_CUDA;
  c->k = k;
  c->N = k + 1;
  c->N3 = c->N * c->N * c->N;
  c->NP = k * (k + 1) * (k + 2) / 6;
  c->g = with_kernels(c.get(), make_grid(mesh->nx, mesh->ny, mesh->nz, k, mesh->lx, mesh->ly, mesh->lz));
  if (c->opt.a_r <= 0) {
    const int N = std::max(mesh->nx, std::max(mesh->ny, mesh->nz));
    c->opt.a_r = std::max(1.0, (N / 16.0) * std::pow(2.0, k - 2));
  }
  c->nlev = n_levels(mesh->nx, mesh->ny, mesh->nz, c->opt.mg_min_n);
  c->mixed = c->opt.precision == WBFBT_MIXED;
  c->m = c->opt.restart;
  if (!build_ref_tables(k, &c->htab)) return WBFBT_ERR_INVALID;
  if (c->opt.pmg && !build_ref_tables(1, &c->htab1)) return WBFBT_ERR_INVALID;
  wbfbt_ctx* cp = c.get();
  int status = guarded_ctx(cp, [&]() {
    const Grid& g = cp->g;
    const size_t nn = g.nn;
    cp->dtab = cp->pool.get<RefTables>(1);
    CK(cudaMemcpyAsync(cp->dtab, &cp->htab, sizeof(RefTables), cudaMemcpyHostToDevice, cp->st));
    if (cp->opt.pmg) {
      cp->dtab1 = cp->pool.get<RefTables>(1);
      CK(cudaMemcpyAsync(cp->dtab1, &cp->htab1, sizeof(RefTables), cudaMemcpyHostToDevice, cp->st));
    }
    if (k == 2) {
      CK(q2_elem64_prepare());
      CK(q2_fused_prepare());
      CK(transfer_prepare());
    }
    if (k <= 3) {
      cp->kwbref = cp->pool.get<double>(kw_bref_entries(k));
      CK(launch_kw_bref(g, k, cp->dtab, cp->kwbref, cp->st));
    }
    cp->part = cp->pool.get<double>((size_t)592 * (1001));
    cp->dsc = cp->pool.get<double>(64);
    cp->dflag = cp->pool.get<int>(4);
    cp->mu64 = cp->pool.get<double>(nn);
    cp->mu32 = cp->pool.get<float>(nn);
    cp->lm = cp->pool.get<double>(nn);
    cp->C = cp->pool.get<double>(nn);
    cp->D = cp->pool.get<double>(nn);
    cp->cinv64 = cp->pool.get<double>(nn);
    cp->dinv64 = cp->pool.get<double>(nn);
    cp->ntot = 3LL * nn + (long long)g.ne * cp->NP;
    cp->Ye64 = cp->pool.get<double>(elem_scratch_size<double>(g, k));
    cp->Ye32 = cp->pool.get<float>(elem_scratch_size<float>(g, k));
    cp->ot64 = make_device_optab<double>(cp, g, cp->k);
    cp->ot32 = make_device_optab<float>(cp, g, cp->k);
    cp->lx = cp->pool.get<float>((size_t)g.ne * (cp->NP + 1));
    cp->ly = cp->pool.get<float>((size_t)g.ne * cp->NP);
    cp->lq = cp->pool.get<float>((size_t)g.ne * cp->NP);
    cp->llogmu = cp->pool.get<float>((size_t)g.ne);
    CK(launch_lumped_mass(g, cp->k, cp->dtab, cp->lm, cp->st));
    run_setup(cp, mu_nodes);
    const long long n = cp->ntot;
    cp->V = cp->pool.get<double>((size_t)(cp->m + 1) * n);
    cp->Z = cp->pool.get<double>((size_t)cp->m * n);
    cp->w = cp->pool.get<double>(n);
    cp->x = cp->pool.get<double>(n);
    cp->r = cp->pool.get<double>(n);
    cp->F = cp->pool.get<double>(n);
    cp->hdev = cp->pool.get<double>(2 * (cp->m + 1) + 1);
    cp->stage_f = cp->pool.get<double>(3 * nn);
    cp->stage_u = cp->pool.get<double>(3 * nn);
    cp->stage_p = cp->pool.get<double>((size_t)g.ne * cp->NP);
    CK(cudaStreamSynchronize(cp->st));
  });
  if (status != WBFBT_OK) return status;
  *out = c.release();
  return WBFBT_OK;
}

int wbfbt_attach_net(wbfbt_ctx* c, wbfbt_net* net, int which_mask, double accept_ratio) {
  if (!c || !(accept_ratio > 0.0 && accept_ratio <= 1.0)) return WBFBT_ERR_INVALID;
  if (net) {
    if (unet_grid(net) != c->g.nx || c->g.nx != c->g.ny || c->g.nx != c->g.nz || unet_channels_in(net) != 1 + c->NP ||
        unet_channels_out(net) != c->NP || (which_mask & ~3))
      return WBFBT_ERR_INVALID;
  }
  c->net = net;
  c->net_mask = net ? which_mask : 0;
  c->net_accept = accept_ratio;
  return WBFBT_OK;
}

int wbfbt_learned_sample(wbfbt_ctx* c, int which, const double* r, float* x_out, float* y_out) {
  if (!c || !r || !x_out || !y_out || (which != 0 && which != 1)) return WBFBT_ERR_INVALID;
  return guarded_ctx(c, [&]() {
    const long long n = (long long)c->g.ne * c->NP;
    auto run = [&](auto tag) {
      using T = decltype(tag);
      Precond<T>& P = prec<T>(c);
      CK((launch_cast<double, T>(n, r, P.pb, c->st)));
      kinv<T>(c, which, P.pb, P.px);
      learned_features<T>(c, which, P.pb, x_out);
      wb_launch(k_learn_target<T>, nb256(n), 256, 0, c->st, n, P.dKw[which], P.px, c->dsc + 16, n, y_out);
      CK(cudaGetLastError());
    };
    if (c->mixed)
      run(float());
    else
      run(double());
  });
}

int wbfbt_learned_stats(const wbfbt_ctx* c, long long* accepted, long long* rejected) {
  if (!c) return WBFBT_ERR_INVALID;
  if (accepted) *accepted = c->learned_acc;
  if (rejected) *rejected = c->learned_rej;
  return WBFBT_OK;
}

int wbfbt_setup(wbfbt_ctx* c, const double* mu_nodes) {
  if (!c || !mu_nodes) return WBFBT_ERR_INVALID;
  return guarded_ctx(c, [&]() { run_setup(c, mu_nodes); });
}

void wbfbt_destroy(wbfbt_ctx* c) {
  if (!c) return;
  if (c->own_net) wbfbt_net_destroy(c->own_net);
  delete c;
}

// ---- learned correction: checkpoint loading and native training (the loop the Python driver
// runs, over the same entry points)

}  // extern "C"

namespace {

// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
struct SplitMix64 {
  unsigned long long s;
  unsigned long long next() {
    unsigned long long z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }   // [0, 1)
  double normal() {   // Box-Muller
    const double u1 = ((double)(next() >> 11) + 1.0) * (1.0 / 9007199254740992.0);   // (0, 1]
    const double u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

struct TrainCfg {
  int fields = 100, per_field = 20, epochs = 20, batch = 4;
  double lr = 1e-3, omega = 0.1, delta = 200.0;
  long long seed = 1000, init_seed = 7;
};

// Flat JSON object of numbers; known keys are read, others ignored.  False on a malformed value.
bool parse_train_cfg(const char* js, TrainCfg* c) {
  auto num = [&](const char* key, double* out) -> bool {
    char pat[64];
    std::snprintf(pat, sizeof(pat), "\"%s\"", key);
    const char* p = std::strstr(js, pat);
    if (!p) return true;
    p += std::strlen(pat);
    while (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r') ++p;
    if (*p != ':') return false;
    ++p;
    char* end = nullptr;
    const double v = std::strtod(p, &end);
    if (end == p || !std::isfinite(v)) return false;
    *out = v;
    return true;
  };
  double f = c->fields, pf = c->per_field, ep = c->epochs, b = c->batch, sd = (double)c->seed,
         is = (double)c->init_seed;
  if (!num("fields", &f) || !num("per_field", &pf) || !num("epochs", &ep) || !num("batch", &b) ||
      !num("lr", &c->lr) || !num("omega", &c->omega) || !num("delta", &c->delta) || !num("seed", &sd) ||
      !num("init_seed", &is))
    return false;
  c->fields = (int)f;
  c->per_field = (int)pf;
  c->epochs = (int)ep;
  c->batch = (int)b;
  c->seed = (long long)sd;
  c->init_seed = (long long)is;
  return c->fields >= 1 && c->per_field >= 1 && c->epochs >= 1 && c->batch >= 1 && c->lr > 0 && c->omega > 0 &&
         c->delta > 0 && c->fields * (long long)c->per_field >= c->batch;
}

bool learned_grid_ok(const wbfbt_ctx* c) {
  return c->g.nx == c->g.ny && c->g.nx == c->g.nz && c->g.nx % 4 == 0 && 1 + c->NP <= 16;
}

struct DevBufs {
  std::vector<void*> p;
  template <typename T>
  T* get(size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) return nullptr;
    p.push_back(q);
    return static_cast<T*>(q);
  }
  ~DevBufs() {
    for (void* q : p) cudaFree(q);
  }
};

}  // namespace

extern "C" {

int wbfbt_load_learned(wbfbt_ctx* c, const char* path) {
  if (!c || !path || !learned_grid_ok(c)) return WBFBT_ERR_INVALID;
  wbfbt_net* net = nullptr;
  int st = wbfbt_net_create(1 + c->NP, c->NP, c->g.nx, 1, c->ust, &net);
  if (st != WBFBT_OK) return st;
  if ((st = wbfbt_net_load(net, path)) != WBFBT_OK || (st = wbfbt_attach_net(c, net, 2, 1.0)) != WBFBT_OK) {
    wbfbt_net_destroy(net);
    return st;
  }
  if (c->own_net) wbfbt_net_destroy(c->own_net);
  c->own_net = net;
  return WBFBT_OK;
}

int wbfbt_train_learned(wbfbt_ctx* c, const char* cfg_json, const char* out_path) {
  if (!c || !out_path || !learned_grid_ok(c)) return WBFBT_ERR_INVALID;
  TrainCfg cfg;
  if (cfg_json && !parse_train_cfg(cfg_json, &cfg)) return WBFBT_ERR_INVALID;
  const int n = c->g.nx, np = c->NP, cin = 1 + np;
  const long long E = c->g.ne, nn = c->g.nn, P = (long long)cfg.fields * cfg.per_field;
  const cudaStream_t us = c->ust;
  DevBufs B;
  float* X = B.get<float>((size_t)P * E * cin);
  float* Y = B.get<float>((size_t)P * E * np);
  float* xb = B.get<float>((size_t)cfg.batch * E * cin);
  float* yb = B.get<float>((size_t)cfg.batch * E * np);
  double* r = B.get<double>((size_t)E * np);
  double* mu = B.get<double>((size_t)nn);
  double* mu0 = B.get<double>((size_t)nn);
  if (!X || !Y || !xb || !yb || !r || !mu || !mu0) return WBFBT_ERR_CUDA;
  if (cudaMemcpyAsync(mu0, c->mu64, sizeof(double) * nn, cudaMemcpyDeviceToDevice, c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess)
    return WBFBT_ERR_CUDA;
  const wbfbt_mesh mesh{c->g.nx, c->g.ny, c->g.nz, c->g.h[0] * c->g.nx, c->g.h[1] * c->g.ny, c->g.h[2] * c->g.nz};
  // training pairs: multi-sinker fields with 8-48 sinkers and DR log-uniform in [1e4, 1e8] (the
  // learned-correction workload), standard-normal mean-free residuals, the solver's own
  // K_r V-cycle corrections as targets
  std::vector<double> rh((size_t)E * np), ch(3 * 48);
  int st = WBFBT_OK;
  for (int f = 0; f < cfg.fields && st == WBFBT_OK; ++f) {
    const long long seed = cfg.seed + f;
    SplitMix64 pd{(unsigned long long)(seed * 7919 + 17)};
    const int ns = 8 + (int)(pd.uniform() * 41);
    const double dr = std::pow(10.0, 4.0 + 4.0 * pd.uniform());
    SplitMix64 pc{(unsigned long long)seed};
    for (int i = 0; i < 3 * ns; ++i) ch[i] = 0.1 + 0.8 * pc.uniform();   // host array, as the call takes it
    if ((st = wbfbt_sinker_setup(&mesh, c->k, ch.data(), ns, cfg.omega, cfg.delta, dr, 10.0, mu, nullptr, us)) !=
            WBFBT_OK ||
        (st = wbfbt_setup(c, mu)) != WBFBT_OK)
      break;
    for (int j = 0; j < cfg.per_field; ++j) {
      SplitMix64 pr{(unsigned long long)(1000003LL * seed + j)};
      double mean = 0.0;
      for (long long i = 0; i < E * np; ++i) rh[i] = pr.normal();
      for (long long e = 0; e < E; ++e) mean += rh[e * np];
      mean /= (double)E;
      for (long long e = 0; e < E; ++e) rh[e * np] -= mean;   // constant mode removed
      if (cudaMemcpyAsync(r, rh.data(), sizeof(double) * E * np, cudaMemcpyHostToDevice, us) != cudaSuccess) {
        st = WBFBT_ERR_CUDA;   // leave through the restore below
        break;
      }
      const long long pidx = (long long)f * cfg.per_field + j;
      if ((st = wbfbt_learned_sample(c, 1, r, X + pidx * E * cin, Y + pidx * E * np)) != WBFBT_OK) break;
    }
    if (st != WBFBT_OK) break;
  }
  const int st_restore = wbfbt_setup(c, mu0);   // the context's own viscosity again
  if (st != WBFBT_OK) return st;
  if (st_restore != WBFBT_OK) return st_restore;
  // the U-Net: He-normal initial weights (N(0, 2 / (27 cin)), zero biases), Adam with a cosine
  // learning-rate decay, shuffled mini-batches
  wbfbt_net* net = nullptr;
  if ((st = wbfbt_net_create(cin, np, n, cfg.batch, us, &net)) != WBFBT_OK) return st;
  std::unique_ptr<wbfbt_net, void (*)(wbfbt_net*)> hold(net, wbfbt_net_destroy);
  {
    const int chans[11][2] = {{cin, 16}, {16, 16}, {16, 32}, {32, 32}, {32, 64}, {64, 64},
                              {96, 32},  {32, 32}, {48, 16}, {16, 16}, {16, np}};
    std::vector<float> theta;
    SplitMix64 pi{(unsigned long long)cfg.init_seed};
    for (const auto& ch2 : chans) {
      const double sd = std::sqrt(2.0 / (27.0 * ch2[0]));
      for (long long i = 0; i < 27LL * ch2[0] * ch2[1]; ++i) theta.push_back((float)(pi.normal() * sd));
      for (int i = 0; i < ch2[1]; ++i) theta.push_back(0.f);
    }
    if ((long long)theta.size() != wbfbt_net_param_count(net)) return WBFBT_ERR_INVALID;
    if ((st = wbfbt_net_set_params(net, theta.data())) != WBFBT_OK) return st;
  }
  const long long nb = P / cfg.batch, steps = (long long)cfg.epochs * nb;
  std::vector<long long> perm(P);
  SplitMix64 po{(unsigned long long)(cfg.seed + 12345)};
  long long step = 0;
  for (int ep = 0; ep < cfg.epochs; ++ep) {
    for (long long i = 0; i < P; ++i) perm[i] = i;
    for (long long i = P - 1; i > 0; --i) std::swap(perm[i], perm[(long long)(po.uniform() * (i + 1))]);
    for (long long b = 0; b < nb; ++b, ++step) {
      for (int t = 0; t < cfg.batch; ++t) {
        const long long q = perm[b * cfg.batch + t];
        if (cudaMemcpyAsync(xb + (size_t)t * E * cin, X + (size_t)q * E * cin, sizeof(float) * E * cin,
                            cudaMemcpyDeviceToDevice, us) != cudaSuccess ||
            cudaMemcpyAsync(yb + (size_t)t * E * np, Y + (size_t)q * E * np, sizeof(float) * E * np,
                            cudaMemcpyDeviceToDevice, us) != cudaSuccess)
          return WBFBT_ERR_CUDA;
      }
      if ((st = wbfbt_net_loss_grad(net, xb, yb, cfg.batch, nullptr, nullptr)) != WBFBT_OK) return st;
      const double lr_t = cfg.lr * 0.5 * (1.0 + std::cos(3.141592653589793 * (double)step / (double)steps));
      if ((st = wbfbt_net_adam_step(net, (float)std::max(lr_t, 1e-5))) != WBFBT_OK) return st;
    }
  }
  return wbfbt_net_save(net, out_path);
}

int wbfbt_sizes(const wbfbt_ctx* c, long long* nn, long long* ne, int* np, int* nl) {
  if (!c) return WBFBT_ERR_INVALID;
  if (nn) *nn = c->g.nn;
  if (ne) *ne = c->g.ne;
  if (np) *np = c->NP;
  if (nl) *nl = c->nlev;
  return WBFBT_OK;
}

long long wbfbt_device_bytes(const wbfbt_ctx* c) { return c ? (long long)c->pool.bytes : 0; }

long long wbfbt_launch_count(void) { return wb_launch_counter().load(); }

static int stokes_apply(wbfbt_ctx* c, int ops, const void* u, const void* p, void* yu, void* yp, int dtype) {
  if (!c || (dtype != WBFBT_F64 && dtype != WBFBT_F32)) return WBFBT_ERR_INVALID;
  return guarded_ctx(c, [&]() {
    if (dtype == WBFBT_F64)
      stokes_apply_t<double>(c, ops, (const double*)u, (const double*)p, (double*)yu, (double*)yp, c->mu64, c->Ye64);
    else
      stokes_apply_t<float>(c, ops, (const float*)u, (const float*)p, (float*)yu, (float*)yp, c->mu32, c->Ye32);
  });
}

int wbfbt_apply_A(wbfbt_ctx* c, const void* u, void* y, int dtype) {
  if (!u || !y) return WBFBT_ERR_INVALID;
  return stokes_apply(c, OP_A, u, nullptr, y, nullptr, dtype);
}

int wbfbt_apply_B(wbfbt_ctx* c, const void* u, void* p, int dtype) {
  if (!u || !p) return WBFBT_ERR_INVALID;
  return stokes_apply(c, OP_B, u, nullptr, nullptr, p, dtype);
}

int wbfbt_apply_BT(wbfbt_ctx* c, const void* p, void* u, int dtype) {
  if (!u || !p) return WBFBT_ERR_INVALID;
  return stokes_apply(c, OP_BT, nullptr, p, u, nullptr, dtype);
}

int wbfbt_apply_K(wbfbt_ctx* c, const void* x, void* y, int dtype) {
  if (!c || !x || !y) return WBFBT_ERR_INVALID;
  const size_t es = dtype == WBFBT_F64 ? 8 : 4;
  const size_t nu = 3 * (size_t)c->g.nn;
  return stokes_apply(c, OP_A | OP_BT | OP_B, x, (const char*)x + nu * es, y, (char*)y + nu * es, dtype);
}

static bool prec_dtype_ok(wbfbt_ctx* c, int dtype) {
  return c && ((dtype == WBFBT_F64 && !c->mixed) || (dtype == WBFBT_F32 && c->mixed));
}

int wbfbt_apply_Kw(wbfbt_ctx* c, int which, const void* p, void* y, int dtype) {
  if (!prec_dtype_ok(c, dtype) || !p || !y || (which != 0 && which != 1)) return WBFBT_ERR_INVALID;
  return guarded_ctx(c, [&]() {
    if (dtype == WBFBT_F64) op_Kw<double>(c, which, (const double*)p, epi_store<double>((double*)y));
    else op_Kw<float>(c, which, (const float*)p, epi_store<float>((float*)y));
  });
}

int wbfbt_apply_Ainv(wbfbt_ctx* c, const void* r, void* y, int dtype) {
  if (!prec_dtype_ok(c, dtype) || !r || !y) return WBFBT_ERR_INVALID;
  return guarded_ctx(c, [&]() {
    if (dtype == WBFBT_F64) vcycle<double>(c, c->P64.HA, 0, (const double*)r, (double*)y);
    else vcycle<float>(c, c->P32.HA, 0, (const float*)r, (float*)y);
  });
}

int wbfbt_apply_Kinv(wbfbt_ctx* c, int which, const void* r, void* y, int dtype) {
  if (!prec_dtype_ok(c, dtype) || !r || !y || (which != 0 && which != 1)) return WBFBT_ERR_INVALID;
  return guarded_ctx(c, [&]() {
    if (dtype == WBFBT_F64) kinv<double>(c, which, (const double*)r, (double*)y);
    else kinv<float>(c, which, (const float*)r, (float*)y);
  });
}

int wbfbt_apply_schur_inv(wbfbt_ctx* c, const void* r, void* y, int dtype) {
  if (!prec_dtype_ok(c, dtype) || !r || !y) return WBFBT_ERR_INVALID;
  return guarded_ctx(c, [&]() {
    if (dtype == WBFBT_F64) schur_inv<double>(c, (const double*)r, (double*)y);
    else schur_inv<float>(c, (const float*)r, (float*)y);
  });
}

int wbfbt_apply_precond(wbfbt_ctx* c, const void* x, void* y, int dtype) {
  if (!prec_dtype_ok(c, dtype) || !x || !y) return WBFBT_ERR_INVALID;
  return guarded_ctx(c, [&]() {
    if (dtype == WBFBT_F64) precond<double>(c, (const double*)x, (double*)y);
    else precond<float>(c, (const float*)x, (float*)y);
  });
}

int wbfbt_set_geometry(wbfbt_ctx* c, const double* X_nodes) {
  if (!c) return WBFBT_ERR_INVALID;
  if (!X_nodes) {
    c->mapped = false;
    return WBFBT_OK;
  }
  const bool dev = is_device_ptr(X_nodes);
  int bad = 0;
  int g = guarded_ctx(c, [&]() {
    const size_t nn = c->g.nn;
    if (c->X64 == nullptr) {
      CK(mapped_prepare());
      c->X64 = c->pool.get<double>(3 * nn);
      c->X32 = c->pool.get<float>(3 * nn);
      c->lm_map = c->pool.get<double>(nn);
      Grid gr = c->g;   // the reference element: unit derivative scale, |J| = 1
      gr.s[0] = gr.s[1] = gr.s[2] = 1.0;
      gr.detJ = 1.0;
      c->rt64 = make_device_optab<double>(c, gr, c->k);
      c->rt32 = make_device_optab<float>(c, gr, c->k);
    }
    c->mapped = false;
    CK(cudaMemcpyAsync(c->X64, X_nodes, sizeof(double) * 3 * nn, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->st));
    CK((launch_cast<double, float>(3LL * (long long)nn, c->X64, c->X32, c->st)));
    CK(cudaMemsetAsync(c->dflag, 0, sizeof(int), c->st));
    CK(launch_mapped_mass<double>(c->g, c->k, c->rt64, c->X64, c->Ye64, c->lm_map, c->dflag, c->st));
    CK(cudaMemcpyAsync(&bad, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->mapped = bad == 0;
  });
  if (g != WBFBT_OK) return g;
  return bad ? WBFBT_ERR_INVALID : WBFBT_OK;
}

int wbfbt_solve(wbfbt_ctx* c, const double* f_nodes, double* u, double* p, double rtol, int maxit, int* iters,
                double* final_rel_res) {
  if (!c || !f_nodes || !u || !p || !(rtol > 0.0) || maxit < 1) return WBFBT_ERR_INVALID;
  const bool dev_f = is_device_ptr(f_nodes), dev_u = is_device_ptr(u), dev_p = is_device_ptr(p);
  if (dev_f != dev_u || dev_u != dev_p) return WBFBT_ERR_INVALID;
  int status = WBFBT_OK;
  int g = guarded_ctx(c, [&]() {
    const size_t nn = c->g.nn, nu = 3 * nn, np = (size_t)c->g.ne * c->NP;
    const double* fd = f_nodes;
    if (!dev_f) {
      CK(cudaMemcpyAsync(c->stage_f, f_nodes, sizeof(double) * nu, cudaMemcpyHostToDevice, c->st));
      fd = c->stage_f;
    }
    CK(cudaMemsetAsync(c->F + nu, 0, sizeof(double) * np, c->st));
    CK(launch_load_vector(c->g, c->mapped ? c->lm_map : c->lm, fd, c->F, c->st));
    status = fgmres(c, rtol, maxit, iters, final_rel_res);
    if (status != WBFBT_OK && status != WBFBT_ERR_MAXIT) return;
    double* ud = dev_u ? u : c->stage_u;
    double* pd = dev_p ? p : c->stage_p;
    CK(cudaMemcpyAsync(ud, c->x, sizeof(double) * nu, cudaMemcpyDeviceToDevice, c->st));
    project<double>(c, c->x + nu, pd);
    if (!dev_u) {
      CK(cudaMemcpyAsync(u, c->stage_u, sizeof(double) * nu, cudaMemcpyDeviceToHost, c->st));
      CK(cudaMemcpyAsync(p, c->stage_p, sizeof(double) * np, cudaMemcpyDeviceToHost, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
  });
  return g != WBFBT_OK ? g : status;
}

int wbfbt_solve_block(wbfbt_ctx* c, int block, const double* b, double* x, double rtol, int maxit, int* iters,
                      double* final_rel_res) {
  if (!c || !b || !x || block < WBFBT_BLOCK_A || block > WBFBT_BLOCK_KR || !(rtol > 0.0) || maxit < 1 || c->mapped)
    return WBFBT_ERR_INVALID;
  if (!is_device_ptr(b) || !is_device_ptr(x)) return WBFBT_ERR_INVALID;
  int status = WBFBT_OK;
  int g = guarded_ctx(c, [&]() {
    const long long n = block == WBFBT_BLOCK_A ? 3LL * c->g.nn : (long long)c->g.ne * c->NP;
    CK(cudaMemcpyAsync(c->F, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
    if (block == WBFBT_BLOCK_A)
      CK(launch_mask_boundary<double>(c->g, 3, c->F, c->st));
    else
      project<double>(c, c->F, c->F);
    status = c->mixed ? block_solve<float>(c, block, n, rtol, maxit, iters, final_rel_res)
                      : block_solve<double>(c, block, n, rtol, maxit, iters, final_rel_res);
    if (status != WBFBT_OK && status != WBFBT_ERR_MAXIT) return;
    if (block == WBFBT_BLOCK_A)
      CK(cudaMemcpyAsync(x, c->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
    else
      project<double>(c, c->x, x);
    CK(cudaStreamSynchronize(c->st));
  });
  return g != WBFBT_OK ? g : status;
}

}  // extern "C"
