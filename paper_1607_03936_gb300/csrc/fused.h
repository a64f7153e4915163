// Two-pass element operators with fused vector epilogues, and fused grid transfers.
//
// An operator apply y = M u runs as an element pass, which writes every element's
// local output (its contribution to each of its n^3 nodes) to a scratch array Ye,
// and a node pass, which sums the contributions of the (up to 8) elements around
// each node in a fixed order -- deterministic, with no atomics and no colouring --
// and hands the sum to an epilogue (store, Chebyshev step, residual update, ...).
// Element-local outputs (B u, per element and pressure mode) take the epilogue
// directly in the element pass.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

enum : int {
  EPI_STORE = 0,       // y = v
  EPI_CHEB_STEP = 1,   // r -= v; d = a d + bc dinv r; x += d
  EPI_SUB = 2,         // r -= v
  EPI_CHEB_INIT1 = 3,  // r = b - v; d = dinv r inv_theta; x += d
  EPI_SCALE = 4,       // y = v * sc[node]            (nodal scale shared by the components)
  EPI_DINV = 5,        // y = dinv * v
  EPI_BMINUS = 6,      // y = b - v
};

template <typename T>
struct Epi {
  int mode = EPI_STORE;
  T* y = nullptr;
  T* r = nullptr;
  T* d = nullptr;
  T* x = nullptr;
  const T* b = nullptr;
  const T* dinv = nullptr;
  const T* sc = nullptr;
  T a = 0, bc = 0, inv_theta = 0;
};

// Element pass of the Stokes family (ops: OP_A | OP_BT | OP_B as in kernels.h).  Velocity
// contributions go to Ye [ne][3][n^3]; the B output (if OP_B) goes through `pe` per (e, m).
// Per-level operator tables (derivatives scaled by 2/h, weights, pressure basis, inverse pressure
// mass, transfer weights) in precision T, built on the host once per level: size and builder.
template <typename T>
size_t optab_bytes(int k);
template <typename T>
void build_optab_host(const RefTables& t, const Grid& g, int k, void* out);

template <typename T>
cudaError_t launch_elem_stokes(const Grid& g, int k, const void* optab, int ops, const T* u, const T* us, const T* p,
                               const T* coef, int coef_nodal, T* Ye, const Epi<T>& pe, cudaStream_t st);

// Element pass of the scalar Q_k Poisson operator: Ye [ne][n^3].
template <typename T>
cudaError_t launch_elem_poisson(const Grid& g, int k, const void* optab, const T* u, const T* coef, T* Ye,
                                cudaStream_t st);

// Pressure transfers of the two-space Poisson cycle: r_c = M_cd M_d^-1 r_d (element pass into Ye
// [ne][n^3], then a node pass) and e_d (+)= M_d^-1 M_dc e_c (element pass).
template <typename T>
cudaError_t launch_disc_to_cont_fused(const Grid& g, int k, const void* optab, const T* rd, T* rc, T* Ye,
                                      cudaStream_t st);
template <typename T>
cudaError_t launch_cont_to_disc_fused(const Grid& g, int k, const void* optab, const T* ec, T* ed, int add,
                                      cudaStream_t st);

// Node pass: v = sum of element contributions (0 on boundary nodes when mask_boundary), then the
// epilogue on entry c * nn + node for each of ncomp components.
template <typename T>
cudaError_t launch_gather(const Grid& g, int k, int ncomp, int mask_boundary, const T* Ye, const Epi<T>& e,
                          cudaStream_t st);

// The same node pass over the element-major scratch [ne][ncomp][n^3] on any grid (launch_gather
// reads the row-segment layout on grids whose k = 2 element passes take the row kernels).
template <typename T>
cudaError_t launch_gather_elem(const Grid& g, int k, int ncomp, int mask_boundary, const T* Ye, const Epi<T>& e,
                               cudaStream_t st);

// ---- Mapped (non-affine) hexahedra (mapped.cu): isoparametric Q_k geometry from the nodal
// coordinates X [3][nn] (precision T); reftab: the operator tables of the reference element
// (derivatives unscaled, weights without |J|).  Ye: element-major scratch [ne][3][n^3].
// ops OP_A, OP_BT, OP_B or all three: yu = epilogue of the velocity output (Dirichlet rows 0),
// yp = epilogue of the B output per (e, m).  bad: set to 1 where det J <= 0.
template <typename T>
cudaError_t launch_mapped_stokes(const Grid& g, int k, const void* reftab, const T* X, int ops, const T* u,
                                 const T* p, const T* coef, int coef_nodal, T* Ye, const Epi<T>& yu, const Epi<T>& yp,
                                 int* bad, cudaStream_t st);
// Once per process, outside stream capture: shared-memory opt-in of the mapped element passes.
cudaError_t mapped_prepare();
// lm(node) = sum over the points at that node of W_q det J_q (the mapped lumped mass, no mask).
template <typename T>
cudaError_t launch_mapped_mass(const Grid& g, int k, const void* reftab, const T* X, T* Ye, T* lm, int* bad,
                               cudaStream_t st);

// Fused transfers between coarse grid gc and its refinement, ncomp components.
//   prolong : out_f (+)= P in_c in one pass (N^3 coarse values per fine node)
//   restrict: out_c = P^T in_f in three separable passes, all components per launch
//             (w1, w2: transfer_work_size(gc, k) * ncomp entries each)
// (optab: the coarse grid's table; only its transfer weights are used.)
template <typename T>
cudaError_t launch_prolong_fused(const Grid& gc, int k, const void* optab, int ncomp, const T* in_c, T* out_f, int add,
                                 cudaStream_t st);
// Once per process, outside stream capture: shared-memory opt-in of the tiled transfers.
cudaError_t transfer_prepare();
template <typename T>
cudaError_t launch_restrict_batched(const Grid& gc, int k, const void* optab, int ncomp, const T* in_f, T* out_c,
                                    int mask_dirichlet, T* w1, T* w2, cudaStream_t st);

// ---- Q2 row-segment path (q2_ops.cu, q2_fp64.cu): element rows split into segments of 32.
// A row segment is up to 32 consecutive elements along x (fixed ey, ez), owned by one warp (a
// lane per element) or, in the FP64 Stokes pass, by one block of 27 such warps; its
// partial node values, summed along x within the segment, are stored per x-line of nodes as
// [segment][ez][ey][l][j][component][X], X = 0 .. 64 padded to Q2_ROW_LD entries.
// n / d for 0 <= n < 2^31 as a multiply-high and a shift (Granlund & Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994): m = ceil(2^(31 + L) / d), L = ceil(log2 d).
struct FastDiv {
  unsigned d, m, s;
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f{d, 0u, 0u};
  if (d > 1) {
    unsigned L = 0;
    while ((1ull << L) < d) ++L;
    f.m = (unsigned)(((1ull << (31 + L)) + d - 1) / d);
    f.s = L - 1;
  }
  return f;
}
#ifdef __CUDACC__
__device__ inline unsigned fdiv(unsigned n, const FastDiv& f) { return f.d == 1 ? n : __umulhi(n, f.m) >> f.s; }
#endif

// Node-pass launch shape: x blocks of bs threads (a multiple of 32, at most 256), y rows and z
// planes; z planes (and y rows beyond 65535) are strided only when the grid would exceed about
// four waves of resident blocks (152 SMs, 64 warps and 32 blocks each).
inline void node_pass_geometry(const Grid& g, dim3& grid, int& bs) {
  bs = ((g.NX + 31) / 32) * 32;
  if (bs > 256) bs = 256;
  const long long nxb = (g.NX + bs - 1) / bs;
  const long long gy = g.NY < 65535 ? g.NY : 65535;
  const long long per_sm = std::min(32, 64 / (bs / 32));
  const long long cap = 4 * 152 * per_sm;
  long long gz = g.NZ;
  if (nxb * gy * gz > cap) gz = std::max(1LL, cap / (nxb * gy));
  if (gz > 65535) gz = 65535;
  grid = dim3((unsigned)nxb, (unsigned)gy, (unsigned)gz);
}

constexpr int Q2_SEG = 32;      // elements per row segment (one warp)
constexpr int Q2_ROW_LD = 66;   // stored nodes per x-line of a segment (65, padded to even)

// Row segments along x: segment index w = seg + nseg (ey + ny ez).
struct Rows {
  int nseg;             // segments along x
  int nrows;            // nseg * ny * nz
  FastDiv fseg, fny;    // segment index -> (seg, ey, ez)
};

inline Rows make_rows(const Grid& g) {
  Rows r;
  r.nseg = (g.nx + Q2_SEG - 1) / Q2_SEG;
  r.nrows = r.nseg * g.ny * g.nz;
  r.fseg = make_fastdiv(r.nseg);
  r.fny = make_fastdiv(g.ny);
  return r;
}
// Scratch entries the row-segment element pass writes for ncomp components.
size_t q2_row_scratch(const Grid& g, int ncomp);
// Scratch entries (precision T, order k) an element pass on grid g may write for 3 components.
template <typename T>
size_t elem_scratch_size(const Grid& g, int k);

cudaError_t launch_q2_elem(const Grid& g, int ops, const float* u, const float* p, const float* coef, int coef_nodal,
                           float* R, const Epi<float>& pe, cudaStream_t st);
// The FP64 Stokes element pass on the same segments and scratch layout (q2_fp64.cu): one warp
// per element point and one lane per element (81 + 81 FP64 registers per thread would not fit).
cudaError_t launch_q2_elem64(const Grid& g, int ops, const double* u, const double* p, const double* coef,
                             int coef_nodal, double* R, const Epi<double>& pe, cudaStream_t st);
// The FP64 scalar Poisson pass in the same layout (q2_fp64.cu, warp per element point).
cudaError_t launch_q2_poisson64(const Grid& g, const double* u, const double* coef, double* R, cudaStream_t st);
// Flat FP64 variants (q2_fp64.cu) for k = 2 levels below the row-segment size: 32 consecutive
// elements per block in linear order, element-major scratch (A: [E][3][27], Poisson [E][27]).
cudaError_t launch_q2_elem64_flat(const Grid& g, const double* u, const double* coef, int coef_nodal, double* Ye,
                                  cudaStream_t st);
cudaError_t launch_q2_poisson64_flat(const Grid& g, const double* u, const double* coef, double* Ye, cudaStream_t st);
// One-time launch set-up of the q2_fp64.cu passes (shared-memory opt-in, occupancy); call it
// outside any stream capture.
cudaError_t q2_elem64_prepare();
// Scalar row kernels (Poisson, node pass, pressure transfers) in FP32 and FP64.
template <typename T>
cudaError_t launch_q2_poisson(const Grid& g, const T* u, const T* coef, T* R, cudaStream_t st);
template <typename T>
cudaError_t launch_q2_gather(const Grid& g, int ncomp, int mask_boundary, const T* R, const Epi<T>& e,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_q2_d2c(const Grid& g, const T* rd, T* rc, T* R, cudaStream_t st);
template <typename T>
cudaError_t launch_q2_c2d(const Grid& g, const T* ec, T* ed, int add, cudaStream_t st);

// ---- Single-kernel FP32 Q2 A apply (q2_fused.cu) on large row-segment levels: tiles of 32 x 4
// element columns and zc element layers; the element kernel applies the epilogue to the nodes
// inside each tile's node box and stores the box-surface parts in a shell array [tile][3][ss],
// which a second kernel sums per surface node (1, 2, 4 or 8 tiles) before the epilogue.
struct Q2Tiles {
  int zc;                  // element layers per tile (each thread marches its column through them)
  int nseg, nyt, nzc;      // tiles along x, y and z
  int ss;                  // shell entries per tile and component (full tile)
  int n1, n2, n3;          // surface nodes: on a z face; on a y face only; on an x face only
  FastDiv fNX, fNY, fnyf, fnxf, fnyo, fpz;   // NX, NY, y faces, x faces, NY - y faces, 2 zc - 1
};
constexpr int Q2_FUSED_POISSON = 8;   // ops value of launch_q2_fused: the scalar Poisson operator
// Once per process, outside stream capture: the fused kernels' resident blocks per device.
cudaError_t q2_fused_prepare();
bool q2_fused_eligible(const Grid& g);
Q2Tiles q2_fused_tiles(const Grid& g, int ops);
// Shell entries (floats) the fused apply writes on grid g.
size_t q2_fused_scratch(const Grid& g);
// epilogue(A u) (ops OP_A) or epilogue(B^T p) (ops OP_BT) on every velocity entry (Dirichlet
// nodes: v = 0 when mask_boundary), or epilogue(L_c u) (ops Q2_FUSED_POISSON, scalar, coefficient
// per element point) on every node.
cudaError_t launch_q2_fused(const Grid& g, int ops, const float* u, const float* p, const float* coef,
                            int coef_nodal, float* shell, int mask_boundary, const Epi<float>& e, cudaStream_t st);
// A apply (ops OP_A: input u, coefficient coef) or B^T apply (OP_BT: input p) with epilogue on a
// vector level of order k: the fused form where it applies, else the element pass and the node pass.
// L_c u with epilogue on a scalar Poisson level of order k (no boundary mask): the same choice.
template <typename T>
cudaError_t launch_apply_poisson_epi(const Grid& g, int k, const void* optab, const T* u, const T* coef, T* Ye,
                                     const Epi<T>& e, cudaStream_t st);
template <typename T>
cudaError_t launch_apply_vec_epi(const Grid& g, int k, const void* optab, int ops, const T* u, const T* p,
                                 const T* coef, int coef_nodal, T* Ye, int mask_boundary, const Epi<T>& e,
                                 cudaStream_t st);

// ---- Assembled K_w = B C_w^-1 B^T (kw_ops.cu), k = 2 and 3: a 27-neighbour block stencil of
// Np x Np blocks per element, stored [o][m][m'][e] in the preconditioner precision.
size_t kw_stencil_entries(const Grid& g, int k);
size_t kw_bref_entries(int k);
// bref: the reference divergence matrix B_e[m][(a, c)] scaled to grid g (FP64, kw_bref_entries).
cudaError_t launch_kw_bref(const Grid& g, int k, const RefTables* dtab, double* bref, cudaStream_t st);
// Kst from bref and the nodal inverse weight cinv (C^-1 or D^-1, zero on Dirichlet nodes).
template <typename T>
cudaError_t launch_kw_assemble(const Grid& g, int k, const double* bref, const double* cinv, T* Kst, cudaStream_t st);
// Jacobi inverse diagonal of K_w from bref (the same quantity as launch_dinv_Kw).
template <typename T>
cudaError_t launch_kw_dinv(const Grid& g, int k, const double* bref, const double* cinv, T* dinv, cudaStream_t st);
// epilogue(K_w p) on every pressure entry.
template <typename T>
cudaError_t launch_kw_apply(const Grid& g, int k, const T* Kst, const T* p, const Epi<T>& e, cudaStream_t st);
