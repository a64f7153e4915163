// Single-kernel applies of the single-precision Q2 operators with their node-wise epilogues, for
// the large row-segment levels: the viscous operator A (Sec. 1.2: a(u,v) = int 2 mu eps(u):eps(v)),
// the gradient B^T (b(v,q) = -int q div v, the first factor of K_w = B C^-1 B^T, whose node
// epilogue is the C^-1 scaling) and the scalar Poisson operator int c grad u . grad v of the
// two-space pressure cycle (Sec. 6).
//
// The two-pass form (q2_ops.cu) writes every element's partial node values to a scratch array
// and sums them in a separate node pass; on the fine level that round trip is more traffic than
// the epilogue's own vectors.  Here the sums are formed on chip:
//   - a block owns a tile of 32 (x) x 4 (y) element columns and a chunk of zc element layers;
//     lane = element along x, warp = element row along y;
//   - each thread marches its column up through the chunk, one element per step (the element
//     arithmetic is q2_body.cuh's); the element's top node plane stays in registers and becomes
//     the next element's bottom plane, so every node plane is complete in z when it is emitted;
//   - an emitted plane is summed along x by one warp shuffle per value (a lane owns x-nodes
//     2 lane and 2 lane + 1) and along y through shared memory (warp w's top node line is added
//     to warp w + 1's bottom line);
//   - a node strictly inside the tile's node box then has its complete value and takes the
//     epilogue at once, with the epilogue's operands fetched into shared memory by asynchronous
//     copies issued before the element is computed; a node on the box surface (shared with a
//     neighbouring tile, or on the domain boundary) has only this tile's part, which goes to a
//     per-tile shell array;
//   - a second kernel visits the surface nodes only, adds the parts of the (1, 2, 4 or 8) tiles
//     through each in the fixed order z, y, x ascending, masks Dirichlet nodes (vector operators)
//     and applies the epilogue.
// Sums are formed in a fixed order throughout: the result is bitwise reproducible.
//
// In-place epilogues (a Chebyshev step updates the vector the operator is applied to): a node
// inside the box is read only by this tile's elements, and it is written after the last of them
// has loaded it (the same thread's earlier steps, or other warps before the block barrier of the
// emit); surface nodes are written only by the second kernel.  The operand slots of a step are
// refilled by the next step's asynchronous copies only after this step's reads of them, in the
// same thread.
#include "elem_common.cuh"
#include "epi.cuh"
#include "fused.h"
#include "kernels.h"
#include "q2_body.cuh"

namespace {

using namespace wb;

constexpr int FBY = 4;     // element rows per tile (one warp each)
constexpr int FSEG = 32;   // elements per tile along x (one lane each)
constexpr int FTHREADS = 32 * FBY;
constexpr int FIX_THREADS = 256;

// Operators: components and resident blocks per SM the register budget is sized for.
template <int OPS>
__host__ __device__ constexpr int fused_nc() {
  return OPS == Q2_FUSED_POISSON ? 1 : 3;
}
template <int OPS>
__host__ __device__ constexpr int fused_min_blocks() {
  return OPS == OP_A ? 2 : (OPS == OP_BT ? 3 : 4);
}
inline int ops_slot(int ops) { return ops == OP_A ? 0 : (ops == OP_BT ? 1 : 2); }

int g_fused_slots[3] = {0, 0, 0};   // resident blocks over the device per operator (set once)

// Epilogue operands (the arrays epi_pre reads, in its order) of each mode.
template <int MODE>
__host__ __device__ constexpr int epi_nops() {
  return MODE == EPI_CHEB_STEP ? 4 : MODE == EPI_CHEB_INIT1 ? 3 : MODE == EPI_STORE ? 0 : 1;
}
template <int MODE>
__device__ __forceinline__ const float* epi_operand(const Epi<float>& E, int k) {
  if (MODE == EPI_SCALE) return E.sc;
  if (MODE == EPI_DINV) return E.dinv;
  if (MODE == EPI_BMINUS) return E.b;
  if (MODE == EPI_SUB) return E.r;
  if (MODE == EPI_CHEB_INIT1) return k == 0 ? E.b : (k == 1 ? E.dinv : E.x);
  if (MODE == EPI_CHEB_STEP) return k == 0 ? E.r : (k == 1 ? E.d : (k == 2 ? E.dinv : E.x));
  return nullptr;
}
// Shared memory of the fused kernel: the y-exchange lines ([warp][component][i][lane]), then per
// thread the epilogue operands of the 8 nodes it emits in one step ([operand][component][node]
// [thread]).
template <int NC, int MODE>
constexpr size_t fused_smem() {
  return sizeof(float) * ((size_t)FBY * NC * 3 * 32 + (size_t)epi_nops<MODE>() * NC * 8 * FTHREADS);
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Index of local node (a, b, c) on the surface of a tile box [0, ax] x [0, by] x [0, cz]:
// bottom plane, top plane, then the ring of each plane in between (front line, back line, then
// the two end nodes of every inner line).
__host__ __device__ inline int shell_index(int a, int b, int c, int ax, int by, int cz) {
  const int px = ax + 1, py = by + 1;
  if (c == 0) return a + px * b;
  if (c == cz) return px * py + a + px * b;
  const int base = 2 * px * py + (c - 1) * (2 * px + 2 * (by - 1));
  if (b == 0) return base + a;
  if (b == by) return base + px + a;
  return base + 2 * px + 2 * (b - 1) + (a == 0 ? 0 : 1);
}

// One emitted node plane (element-local plane L of every thread's current out) at tile-local
// height Zl: sums along x and y, then the epilogue inside the box or the shell on its surface.
template <int NC, int MODE, int L>
__device__ __forceinline__ void emit_plane(const Grid& g, const Q2Tiles& T, const Epi<float>& E, float (&out)[NC][27],
                                           float* ysh, const float* pre, int lane, int w, int nxt, int nyt, int Zl,
                                           int X0, int Y0, int Z0, float* __restrict__ sh) {
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float left = __shfl_up_sync(0xffffffffu, out[c][q2i(2, j, L)], 1);
      if (lane > 0) out[c][q2i(0, j, L)] += left;
    }
  __syncthreads();   // the previous plane's reads of ysh are done
  if (w + 1 < nyt) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int i = 0; i < 3; ++i) ysh[((w * NC + c) * 3 + i) * 32 + lane] = out[c][q2i(i, 2, L)];
  }
  __syncthreads();
  if (w > 0 && w < nyt) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int i = 0; i < 3; ++i) out[c][q2i(i, 0, L)] += ysh[(((w - 1) * NC + c) * 3 + i) * 32 + lane];
  }
  if (lane >= nxt || w >= nyt) return;
  const int ax = 2 * nxt, by = 2 * nyt, cz = 2 * min(T.zc, g.nz - Z0 / 2);
  const size_t nn = (size_t)g.nn;
  const bool zface = Zl == 0 || Zl == cz;
  if (epi_nops<MODE>() > 0) cp_async_wait_all();
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (j == 2 && w != nyt - 1) continue;   // handed to the next warp
    const int Yl = 2 * w + j;
    const bool yface = zface || Yl == 0 || Yl == by;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (i == 2 && lane != nxt - 1) continue;   // handed to the next lane
      const int Xl = 2 * lane + i;
      if (yface || Xl == 0 || Xl == ax) {
        const int si = shell_index(Xl, Yl, Zl, ax, by, cz);
#pragma unroll
        for (int c = 0; c < NC; ++c) sh[(size_t)c * T.ss + si] = out[c][q2i(i, j, L)];
      } else {
        // i, j < 2 here (the i = 2 and j = 2 nodes of a tile's last lane and warp are on its surface)
        const int n = (X0 + Xl) + g.NX * ((Y0 + Yl) + g.NY * (Z0 + Zl));
        const int slot = 4 * L + 2 * j + i;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int k = 0; k < epi_nops<MODE>(); ++k) a[k] = pre[((k * NC + c) * 8 + slot) * FTHREADS + threadIdx.x];
          const EpiOps<float> eo{a[0], a[1], a[2], a[3]};
          epi_post<MODE>(E, (size_t)c * nn + n, eo, out[c][q2i(i, j, L)]);
        }
      }
    }
  }
}

// OPS: OP_A (input u, nodal or per-point coefficient coef), OP_BT (input p, the element's pressure
// modes) or Q2_FUSED_POISSON (scalar input u, coefficient coef per element point).
template <int OPS, int MODE>
__global__ void __launch_bounds__(FTHREADS, fused_min_blocks<OPS>())
k_q2_fused(Grid g, Q2Tiles T, const __grid_constant__ OpTab<float, 3> tb, const float* u, const float* p,
           const float* coef, int coef_nodal, float* __restrict__ shell, Epi<float> E) {
  constexpr bool DA = OPS == OP_A, DBT = OPS == OP_BT, POIS = OPS == Q2_FUSED_POISSON;
  constexpr int NC = fused_nc<OPS>();
  pdl_entry();
  extern __shared__ float fsm[];
  float* ysh = fsm;
  float* pre = fsm + FBY * NC * 3 * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int tile = blockIdx.x;
  const int ts = tile % T.nseg, trest = tile / T.nseg;
  const int ty = trest % T.nyt, tz = trest / T.nyt;
  const int nxt = min(FSEG, g.nx - ts * FSEG), nyt = min(FBY, g.ny - ty * FBY);
  const int ez0 = tz * T.zc, nzt = min(T.zc, g.nz - ez0);
  const int ex = ts * FSEG + lane, ey = ty * FBY + w;
  const bool act = lane < nxt && w < nyt;
  const int X0 = 2 * ts * FSEG, Y0 = 2 * ty * FBY, Z0 = 2 * ez0;
  float* sh = shell + (size_t)tile * NC * T.ss;
  // Dirichlet nodes read as zero: end planes of the element that lie on the domain boundary
  const bool lo_x = ex == 0, hi_x = ex == g.nx - 1, lo_y = ey == 0, hi_y = ey == g.ny - 1;

  float out[NC][27];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int q = 0; q < 27; ++q) out[c][q] = 0.f;
  for (int t = 0; t < nzt; ++t) {
    const int ez = ez0 + t;
    const int n0 = 2 * ex + g.NX * (2 * ey + g.NY * 2 * ez);
    // operands of the epilogue of this step's inner nodes (planes l = 0, 1; i, j = 0, 1), fetched
    // asynchronously while the element is computed
    if (epi_nops<MODE>() > 0 && act) {
#pragma unroll
      for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            if ((i == 0 && lane == 0) || (j == 0 && w == 0) || (l == 0 && t == 0)) continue;   // surface
            const int n = n0 + i + g.NX * (j + g.NY * l);
            const int slot = 4 * l + 2 * j + i;
#pragma unroll
            for (int k = 0; k < epi_nops<MODE>(); ++k)
#pragma unroll
              for (int c = 0; c < NC; ++c) {
                const size_t idx = MODE == EPI_SCALE ? (size_t)n : (size_t)c * g.nn + n;
                cp_async4(pre + ((k * NC + c) * 8 + slot) * FTHREADS + threadIdx.x, epi_operand<MODE>(E, k) + idx);
              }
          }
    }
    const size_t e = (size_t)ex + (size_t)g.nx * ((size_t)ey + (size_t)g.ny * ez);
    if constexpr (POIS) {
      float ur[27], cf[27];
      q2_load_scalar(u, g.NX, g.NY, n0, act, ur);
#pragma unroll
      for (int q = 0; q < 27; ++q) cf[q] = act ? __ldg(coef + e * 27 + q) : 0.f;
      q2_poisson_points<float>(tb, ur, cf, out[0]);
    } else {
      float ur[3][27], mur[27], bacc[4], pm[4] = {0.f, 0.f, 0.f, 0.f};
      if (DA) {
        q2_load_u(u, (size_t)g.nn, g.NX, g.NY, n0, act, lo_x, hi_x, lo_y, hi_y, ez == 0, ez == g.nz - 1, ur);
        q2_load_coef(coef_nodal ? coef + n0 : coef + e * 27, coef_nodal, g.NX, g.NY, act, mur);
      }
      if (DBT && act) {
#pragma unroll
        for (int m = 0; m < 4; ++m) pm[m] = __ldg(p + e * 4 + m);
      }
      q2_stokes_points<DA, DBT, false>(tb, ur, mur, pm, out, bacc);
    }
    emit_plane<NC, MODE, 0>(g, T, E, out, ysh, pre, lane, w, nxt, nyt, 2 * t, X0, Y0, Z0, sh);
    emit_plane<NC, MODE, 1>(g, T, E, out, ysh, pre, lane, w, nxt, nyt, 2 * t + 1, X0, Y0, Z0, sh);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        out[c][q] = out[c][18 + q];
        out[c][9 + q] = 0.f;
        out[c][18 + q] = 0.f;
      }
  }
  emit_plane<NC, MODE, 0>(g, T, E, out, ysh, pre, lane, w, nxt, nyt, 2 * nzt, X0, Y0, Z0, sh);
}

// Tiles along one axis (period P nodes, nt tiles) whose node range holds node X: one, or two
// when X is the face between tiles t0 = t1 - 1 and t1; l0, l1: the node's local coordinates.
struct Span {
  int n, t0, l0, t1, l1;
};
__device__ __forceinline__ Span tiles_through(int X, int P, int nt) {
  Span s;
  s.t1 = min(X / P, nt - 1);
  s.l1 = X - P * s.t1;
  const bool two = s.l1 == 0 && s.t1 > 0;
  s.n = two ? 2 : 1;
  s.t0 = two ? s.t1 - 1 : s.t1;
  s.l0 = two ? P : s.l1;
  return s;
}

// Node coordinate off the tile faces: the q-th node that is not a multiple of P (qd = q / (P - 1)).
__device__ __forceinline__ int off_face(int q, int qd, int P) { return P * qd + 1 + (q - qd * (P - 1)); }

// Surface nodes of all tiles: (1) node planes on a z face, (2) node rows on a y face off the z
// faces, (3) nodes on an x face off both; one thread per node.
template <int NC, int MODE>
__global__ void __launch_bounds__(FIX_THREADS)
k_q2_fused_fix(Grid g, Q2Tiles T, int mask_boundary, const float* __restrict__ shell, Epi<float> E) {
  pdl_entry();
  unsigned id = blockIdx.x * blockDim.x + threadIdx.x;
  const int PX = 2 * FSEG, PY = 2 * FBY, PZ = 2 * T.zc;
  int ix, iy, iz;
  if (id < (unsigned)T.n1) {
    const unsigned r = fdiv(id, T.fNX), kf = fdiv(r, T.fNY);
    ix = (int)(id - r * g.NX);
    iy = (int)(r - kf * g.NY);
    iz = (int)kf < T.nzc ? PZ * (int)kf : g.NZ - 1;
  } else if ((id -= T.n1) < (unsigned)T.n2) {
    const unsigned r = fdiv(id, T.fNX), q = fdiv(r, T.fnyf);
    ix = (int)(id - r * g.NX);
    const int m = (int)(r - q * T.fnyf.d);
    iy = m < T.nyt ? PY * m : g.NY - 1;
    iz = off_face((int)q, (int)fdiv(q, T.fpz), PZ);
  } else if ((id -= T.n2) < (unsigned)T.n3) {
    const unsigned r = fdiv(id, T.fnxf), q = fdiv(r, T.fnyo);
    const int p = (int)(id - r * T.fnxf.d), ry = (int)(r - q * T.fnyo.d);
    ix = p < T.nseg ? PX * p : g.NX - 1;
    iy = off_face(ry, ry / (PY - 1), PY);
    iz = off_face((int)q, (int)fdiv(q, T.fpz), PZ);
  } else {
    return;
  }
  const size_t nn = (size_t)g.nn;
  const int n = ix + g.NX * (iy + g.NY * iz);
  EpiOps<float> eo[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) eo[c] = epi_pre<MODE>(E, (size_t)c * nn + n, n);
  float v[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) v[c] = 0.f;
  if (!(mask_boundary && on_boundary(g, ix, iy, iz))) {
    const Span sx = tiles_through(ix, PX, T.nseg), sy = tiles_through(iy, PY, T.nyt), sz = tiles_through(iz, PZ, T.nzc);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      if (a >= sz.n) break;
      const int tz = a ? sz.t1 : sz.t0, zl = a ? sz.l1 : sz.l0;
      const int cz = 2 * min(T.zc, g.nz - tz * T.zc);
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        if (b >= sy.n) break;
        const int ty = b ? sy.t1 : sy.t0, yl = b ? sy.l1 : sy.l0;
        const int by = 2 * min(FBY, g.ny - ty * FBY);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          if (s >= sx.n) break;
          const int tx = s ? sx.t1 : sx.t0, xl = s ? sx.l1 : sx.l0;
          const int ax = 2 * min(FSEG, g.nx - tx * FSEG);
          const size_t tile = (size_t)tx + (size_t)T.nseg * (ty + (size_t)T.nyt * tz);
          const float* sp = shell + tile * NC * T.ss + shell_index(xl, yl, zl, ax, by, cz);
#pragma unroll
          for (int c = 0; c < NC; ++c) v[c] += __ldg(sp + (size_t)c * T.ss);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) epi_post<MODE>(E, (size_t)c * nn + n, eo[c], v[c]);
}

template <int OPS>
cudaError_t set_smem_attrs() {
  cudaError_t e = cudaSuccess;
  for (int m = EPI_STORE; m <= EPI_BMINUS && e == cudaSuccess; ++m)
    e = epi_dispatch(m, [](auto mm) {
      constexpr int MODE = decltype(mm)::value;
      return cudaFuncSetAttribute(k_q2_fused<OPS, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fused_smem<fused_nc<OPS>(), MODE>());
    });
  return e;
}

template <int OPS>
cudaError_t resident_blocks(int* per_sm) {
  constexpr int MODE = OPS == OP_BT ? EPI_SCALE : EPI_CHEB_STEP;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_q2_fused<OPS, MODE>, FTHREADS,
                                                       fused_smem<fused_nc<OPS>(), MODE>());
}

template <int OPS>
cudaError_t launch_ops(const Grid& g, const Q2Tiles& T, const OpTab<float, 3>& tb, const float* u, const float* p,
                       const float* coef, int coef_nodal, float* shell, int mask_boundary, const Epi<float>& e,
                       cudaStream_t st) {
  constexpr int NC = fused_nc<OPS>();
  const unsigned tiles = (unsigned)(T.nseg * T.nyt * T.nzc);
  const long long nf = (long long)T.n1 + T.n2 + T.n3;
  return epi_dispatch(e.mode, [&](auto m) -> cudaError_t {
    constexpr int MODE = decltype(m)::value;
    wb_launch(k_q2_fused<OPS, MODE>, tiles, FTHREADS, fused_smem<NC, MODE>(), st, g, T, tb, u, p, coef, coef_nodal,
              shell, e);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    wb_launch(k_q2_fused_fix<NC, MODE>, (unsigned)((nf + FIX_THREADS - 1) / FIX_THREADS), FIX_THREADS, 0, st, g, T,
              mask_boundary, shell, e);
    return cudaGetLastError();
  });
}

}  // namespace

cudaError_t q2_fused_prepare() {
  if (g_fused_slots[0] > 0) return cudaSuccess;
  cudaError_t e = set_smem_attrs<OP_A>();
  if (e == cudaSuccess) e = set_smem_attrs<OP_BT>();
  if (e == cudaSuccess) e = set_smem_attrs<Q2_FUSED_POISSON>();
  int dev = 0, nsm = 0, per_sm[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = resident_blocks<OP_A>(&per_sm[0]);
  if (e == cudaSuccess) e = resident_blocks<OP_BT>(&per_sm[1]);
  if (e == cudaSuccess) e = resident_blocks<Q2_FUSED_POISSON>(&per_sm[2]);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < 3; ++i) g_fused_slots[i] = std::max(1, nsm * per_sm[i]);
  return cudaSuccess;
}

// Automatic kernel choice only (the forced row and per-point choices keep the two-pass form), on
// levels whose tiles of four layers or more still fill the device (128^3 / 16 elements: 64^3,
// not 32^3, which would leave 64 tiles for 152 SMs).
bool q2_fused_eligible(const Grid& g) {
  return g.kern == 0 && g.rowk && g.nx >= FSEG && g.ne >= (1 << 17) && (long long)g.nn < (1LL << 30);
}

// Chunk height zc >= 4 (so at most one node plane in eight is a z face, summed by the fix-up):
// the fewest steps per thread (waves of resident blocks x zc), ties to the taller chunk.
Q2Tiles q2_fused_tiles(const Grid& g, int ops) {
  Q2Tiles T{};
  T.nseg = (g.nx + FSEG - 1) / FSEG;
  T.nyt = (g.ny + FBY - 1) / FBY;
  const int si = ops_slot(ops);
  const long long slots = g_fused_slots[si] > 0 ? g_fused_slots[si] : 304;
  long long best = -1;
  for (int zc = std::min(4, g.nz); zc <= g.nz; ++zc) {
    const long long nzc = (g.nz + zc - 1) / zc;
    const long long tiles = (long long)T.nseg * T.nyt * nzc;
    const long long cost = ((tiles + slots - 1) / slots) * zc;
    if (best < 0 || cost <= best) {
      best = cost;
      T.zc = zc;
    }
  }
  T.nzc = (g.nz + T.zc - 1) / T.zc;
  const int px = 2 * FSEG + 1, py = 2 * FBY + 1;
  T.ss = 2 * px * py + (2 * T.zc - 1) * (2 * px + 2 * (py - 2));
  const long long nzf = T.nzc + 1, nyf = T.nyt + 1, nxf = T.nseg + 1;
  T.n1 = (int)(nzf * g.NY * g.NX);
  T.n2 = (int)((g.NZ - nzf) * nyf * g.NX);
  T.n3 = (int)((g.NZ - nzf) * (g.NY - nyf) * nxf);
  T.fNX = make_fastdiv(g.NX);
  T.fNY = make_fastdiv(g.NY);
  T.fnyf = make_fastdiv((unsigned)nyf);
  T.fnxf = make_fastdiv((unsigned)nxf);
  T.fnyo = make_fastdiv((unsigned)(g.NY - nyf));
  T.fpz = make_fastdiv((unsigned)(2 * T.zc - 1));
  return T;
}

size_t q2_fused_scratch(const Grid& g) {
  size_t n = 0;
  const int all_ops[3] = {OP_A, OP_BT, Q2_FUSED_POISSON};
  for (int ops : all_ops) {
    const Q2Tiles T = q2_fused_tiles(g, ops);
    n = std::max(n, (size_t)T.nseg * T.nyt * T.nzc * (ops == Q2_FUSED_POISSON ? 1 : 3) * T.ss);
  }
  return n;
}

cudaError_t launch_q2_fused(const Grid& g, int ops, const float* u, const float* p, const float* coef,
                            int coef_nodal, float* shell, int mask_boundary, const Epi<float>& e, cudaStream_t st) {
  static const RefTables ref = [] {
    RefTables r;
    build_ref_tables(2, &r);
    return r;
  }();
  OpTab<float, 3> tb;
  make_optab<float, 3>(ref, g, &tb);
  const Q2Tiles T = q2_fused_tiles(g, ops);
  switch (ops) {
    case OP_A: return launch_ops<OP_A>(g, T, tb, u, p, coef, coef_nodal, shell, mask_boundary, e, st);
    case OP_BT: return launch_ops<OP_BT>(g, T, tb, u, p, coef, coef_nodal, shell, mask_boundary, e, st);
    case Q2_FUSED_POISSON:
      return launch_ops<Q2_FUSED_POISSON>(g, T, tb, u, p, coef, coef_nodal, shell, mask_boundary, e, st);
    default: return cudaErrorInvalidValue;
  }
}
