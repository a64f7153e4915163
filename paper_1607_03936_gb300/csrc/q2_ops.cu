// Q2 (k = 2) row-segment kernels with one thread per element (warps along element rows): the
// single-precision operator passes, and in both precisions the pressure transfers of the
// two-space cycle and the node pass that all row-segment producers share.
//
// Element pass: a warp owns a row segment of up to 32 consecutive elements along x (fixed ey,
// ez), one thread per element, with the element arithmetic of q2_body.cuh (Sec. 1.2: the viscous
// stress a(u,v) = int 2 mu eps(u):eps(v), b(v,q) = -int q div v) and, for the scalar Poisson
// operator of the two-space pressure cycle (Sec. 6, int c grad u . grad v), the same sums on one
// component.  The operator tables (derivatives scaled by 2/h, weights times |J|, pressure basis)
// are a kernel parameter, so every table entry is a constant-bank operand of the FMAs using it.
// Row assembly: neighbouring threads share an x-face; each thread passes its right face to the
// next lane (one warp shuffle per value) and adds it to its own left face, so the lane holding
// element ex owns the x-nodes 2 ex and 2 ex + 1 of the segment (the last lane also 2 ex + 2).
// The segment's partial node values are stored per x-line [seg][ez][ey][l][j][c][X] with
// coalesced two-float stores.
// Node pass: each mesh node adds the partials of the (up to 2 x 2 x 2) segment lines through it
// in the fixed order z, y, x ascending and hands the sum to the fused epilogue.  No atomics: the
// result is bitwise reproducible.
#include "elem_common.cuh"
#include "epi.cuh"
#include "q2_body.cuh"
#include "fused.h"
#include "kernels.h"

namespace {

using namespace wb;

using Tab2 = OpTab<float, 3>;
constexpr int WARPS = 4;   // row segments per block

__host__ __device__ constexpr int q3(int i, int j, int l) { return i + 3 * (j + 3 * l); }

// Position of this thread: segment, element row and element.
struct RowPos {
  int seg, ey, ez, lane, ex, e;
  bool act, warp_live;
};

__device__ inline RowPos row_pos(const Grid& g, const Rows& rw) {
  RowPos r;
  const unsigned w = blockIdx.x * WARPS + (threadIdx.x >> 5);
  r.lane = threadIdx.x & 31;
  r.warp_live = w < (unsigned)rw.nrows;
  const unsigned rest = fdiv(w, rw.fseg);
  r.seg = (int)(w - rest * rw.nseg);
  r.ez = (int)fdiv(rest, rw.fny);
  r.ey = (int)rest - r.ez * g.ny;
  r.ex = r.seg * Q2_SEG + r.lane;
  r.act = r.warp_live && r.ex < g.nx;
  r.e = r.ex + g.nx * (r.ey + g.ny * r.ez);
  return r;
}

// Two consecutive entries in one 8- or 16-byte store (the address is aligned: even entry of a row
// whose length Q2_ROW_LD is even).
__device__ inline void store2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
__device__ inline void store2(double* p, double a, double b) { *reinterpret_cast<double2*>(p) = make_double2(a, b); }

// x-assembly of NC x 27 register outputs and the store of the segment's x-line partials.
template <int NC, typename T>
__device__ inline void row_store(const Grid& g, const RowPos& rp, T (*out)[27], T* __restrict__ R) {
  const int last = min(Q2_SEG - 1, g.nx - 1 - rp.seg * Q2_SEG);   // lane of the segment's last element
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int jl = 0; jl < 9; ++jl) {
      const T left = __shfl_up_sync(0xffffffffu, out[c][3 * jl + 2], 1);
      if (rp.lane > 0) out[c][3 * jl] += left;
    }
  if (!rp.act) return;
  const size_t line0 = (((size_t)rp.seg * g.nz + rp.ez) * g.ny + rp.ey) * 9;
#pragma unroll
  for (int jl = 0; jl < 9; ++jl)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T* row = R + ((line0 + jl) * NC + c) * Q2_ROW_LD;
      store2(row + 2 * rp.lane, out[c][3 * jl], out[c][3 * jl + 1]);
      if (rp.lane == last) row[2 * rp.lane + 2] = out[c][3 * jl + 2];
    }
}

// Stokes-family element pass (ops: OP_A | OP_BT | OP_B).  Velocity contributions go to the row
// scratch R; the B output (per element and pressure mode) takes the epilogue pe.
template <int OPS>
__global__ void __launch_bounds__(32 * WARPS)
k_q2_elem(Grid g, Rows rw, const __grid_constant__ Tab2 tb, const float* __restrict__ u,
          const float* __restrict__ p, const float* __restrict__ coef, int coef_nodal, float* __restrict__ R,
          Epi<float> pe) {
  pdl_entry();
  constexpr bool DA = OPS & OP_A, DBT = OPS & OP_BT, DB = OPS & OP_B;
  constexpr bool GRAD = DA || DB, SCAT = DA || DBT;
  const RowPos rp = row_pos(g, rw);
  if (!rp.warp_live) return;   // whole warp: no shuffle partner is left behind
  const size_t nn = (size_t)g.nn;
  const int n0 = 2 * rp.ex + g.NX * (2 * rp.ey + g.NY * 2 * rp.ez);
  // Dirichlet nodes read as zero: end planes of the element that lie on the domain boundary
  const bool lo_x = rp.ex == 0, hi_x = rp.ex == g.nx - 1;
  const bool lo_y = rp.ey == 0, hi_y = rp.ey == g.ny - 1;
  const bool lo_z = rp.ez == 0, hi_z = rp.ez == g.nz - 1;

  float ur[3][27], mur[27], out[3][27];
  if (GRAD) q2_load_u(u, nn, g.NX, g.NY, n0, rp.act, lo_x, hi_x, lo_y, hi_y, lo_z, hi_z, ur);
  if (DA) q2_load_coef(coef_nodal ? coef + n0 : coef + (size_t)rp.e * 27, coef_nodal, g.NX, g.NY, rp.act, mur);
  float pm[4] = {0.f, 0.f, 0.f, 0.f};
  if (DBT && rp.act) {
#pragma unroll
    for (int m = 0; m < 4; ++m) pm[m] = __ldg(p + (size_t)rp.e * 4 + m);
  }
  if (SCAT) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int q = 0; q < 27; ++q) out[c][q] = 0.f;
  }
  float bacc[4] = {0.f, 0.f, 0.f, 0.f};
  q2_stokes_points<DA, DBT, DB>(tb, ur, mur, pm, out, bacc);

  if (DB && rp.act) {
#pragma unroll
    for (int m = 0; m < 4; ++m) epi_apply(pe, (size_t)rp.e * 4 + m, 0, bacc[m]);
  }
  if (SCAT) row_store<3, float>(g, rp, out, R);
}

// Scalar Q2 Poisson element pass, c per element point (no Dirichlet rows: Neumann operator).
template <typename T>
__global__ void __launch_bounds__(32 * WARPS)
k_q2_poisson(Grid g, Rows rw, const __grid_constant__ OpTab<T, 3> tb, const T* __restrict__ u,
             const T* __restrict__ coef, T* __restrict__ R) {
  pdl_entry();
  const RowPos rp = row_pos(g, rw);
  if (!rp.warp_live) return;
  const int n0 = 2 * rp.ex + g.NX * (2 * rp.ey + g.NY * 2 * rp.ez);
  T ur[27], cf[27], out[1][27];
  q2_load_scalar(u, g.NX, g.NY, n0, rp.act, ur);
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    cf[q] = rp.act ? __ldg(coef + (size_t)rp.e * 27 + q) : T(0);
    out[0][q] = T(0);
  }
  q2_poisson_points<T>(tb, ur, cf, out[0]);
  row_store<1, T>(g, rp, out, R);
}

// Pressure transfers of the two-space Poisson cycle (Sec. 6), one thread per element (|J|
// cancels between M_d^-1 and the masses):
//   r_c = M_cd M_d^-1 r_d: element part out[q] = W_q sum_m psi_m(q) (Minv r_e)_m, assembled
//   along rows like the operators (the node pass then stores the sums);
template <typename T>
__global__ void __launch_bounds__(32 * WARPS)
k_q2_d2c(Grid g, Rows rw, const __grid_constant__ OpTab<T, 3> tb, const T* __restrict__ rd, T* __restrict__ R) {
  pdl_entry();
  const RowPos rp = row_pos(g, rw);
  if (!rp.warp_live) return;
  T rv[4], v[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) rv[m] = rp.act ? __ldg(rd + (size_t)rp.e * 4 + m) : T(0);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    T a = T(0);
#pragma unroll
    for (int mp = 0; mp < 4; ++mp) a += tb.Minv[m][mp] * rv[mp];
    v[m] = a;
  }
  T out[1][27];
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    T a = T(0);
#pragma unroll
    for (int m = 0; m < 4; ++m) a += tb.Psi[q][m] * v[m];
    out[0][q] = tb.Wref[q] * a;
  }
  row_store<1, T>(g, rp, out, R);
}

//   e_d (+)= M_d^-1 M_dc e_c: e_d[e][m] = sum_m' Minv[m][m'] sum_q W_q psi_m'(q) e_c(node(e, q)).
template <typename T>
__global__ void __launch_bounds__(32 * WARPS)
k_q2_c2d(Grid g, Rows rw, const __grid_constant__ OpTab<T, 3> tb, const T* __restrict__ ec, T* __restrict__ ed,
         int add) {
  pdl_entry();
  const RowPos rp = row_pos(g, rw);
  if (!rp.act) return;
  const int n0 = 2 * rp.ex + g.NX * (2 * rp.ey + g.NY * 2 * rp.ez);
  T mom[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int roff = n0 + g.NX * (j + g.NY * l);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int q = q3(i, j, l);
        const T w = tb.Wref[q] * __ldg(ec + roff + i);
#pragma unroll
        for (int m = 0; m < 4; ++m) mom[m] += tb.Psi[q][m] * w;
      }
    }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    T a = T(0);
#pragma unroll
    for (int mp = 0; mp < 4; ++mp) a += tb.Minv[m][mp] * mom[mp];
    T* dst = ed + (size_t)rp.e * 4 + m;
    *dst = add ? *dst + a : a;
  }
}

// Node pass: grid (x blocks, y rows, z planes), z (and y) strided so the launch is about one
// wave.  Lines through node (ix, iy, iz): along z the element rows ez = iz / 2 (l = 1) for odd
// iz, else (iz / 2 - 1, l = 2) and (iz / 2, l = 0) where they exist; the same along y; along x
// the segment s = ix / 64 at X = ix - 64 s, and also s - 1 at X = 64 when ix is a segment's
// first node.  The epilogue operands are loaded before the partials.
template <typename T, int NC, int MODE>
__global__ void k_q2_gather(Grid g, int nseg, int mask_boundary, const T* __restrict__ R, Epi<T> E) {
  pdl_entry();
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  if (ix >= g.NX) return;
  const int s = ix >> 6, X = ix & 63;
  const bool prev = X == 0 && s > 0, cur = s < nseg;
  const size_t per_seg = (size_t)g.nz * g.ny * 9;
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
        int zr[2] = {0, 0}, zl[2] = {0, 0}, nzr = 0, yr[2] = {0, 0}, yl[2] = {0, 0}, nyr = 0;
        if (iz & 1) {
          zr[0] = iz >> 1; zl[0] = 1; nzr = 1;
        } else {
          if (iz > 0) { zr[0] = (iz >> 1) - 1; zl[0] = 2; nzr = 1; }
          if ((iz >> 1) < g.nz) { zr[nzr] = iz >> 1; zl[nzr] = 0; ++nzr; }
        }
        if (iy & 1) {
          yr[0] = iy >> 1; yl[0] = 1; nyr = 1;
        } else {
          if (iy > 0) { yr[0] = (iy >> 1) - 1; yl[0] = 2; nyr = 1; }
          if ((iy >> 1) < g.ny) { yr[nyr] = iy >> 1; yl[nyr] = 0; ++nyr; }
        }
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          if (a < nzr) {
#pragma unroll
            for (int b = 0; b < 2; ++b) {
              if (b < nyr) {
                const size_t rowl = ((size_t)zr[a] * g.ny + yr[b]) * 9 + 3 * zl[a] + yl[b];   // within a segment
                if (prev) {
                  const T* src = R + ((s - 1) * per_seg + rowl) * NC * Q2_ROW_LD + 2 * Q2_SEG;
#pragma unroll
                  for (int c = 0; c < NC; ++c) v[c] += __ldg(src + c * Q2_ROW_LD);
                }
                if (cur) {
                  const T* src = R + ((size_t)s * per_seg + rowl) * NC * Q2_ROW_LD + X;
#pragma unroll
                  for (int c = 0; c < NC; ++c) v[c] += __ldg(src + c * Q2_ROW_LD);
                }
              }
            }
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) epi_post<MODE>(E, (size_t)c * g.nn + n, eo[c], v[c]);
    }
}

const RefTables& ref_tables_q2() {
  static const RefTables t = [] {
    RefTables r;
    build_ref_tables(2, &r);
    return r;
  }();
  return t;
}

template <typename T>
OpTab<T, 3> q2_tab(const Grid& g) {
  OpTab<T, 3> t;
  make_optab<T, 3>(ref_tables_q2(), g, &t);
  return t;
}

unsigned elem_grid(const Rows& rw) { return (unsigned)((rw.nrows + WARPS - 1) / WARPS); }

}  // namespace

size_t q2_row_scratch(const Grid& g, int ncomp) {
  const Rows rw = make_rows(g);
  return (size_t)rw.nrows * 9 * ncomp * Q2_ROW_LD;
}

cudaError_t launch_q2_elem(const Grid& g, int ops, const float* u, const float* p, const float* coef, int coef_nodal,
                           float* R, const Epi<float>& pe, cudaStream_t st) {
  const Rows rw = make_rows(g);
  const Tab2 tb = q2_tab<float>(g);
  const unsigned nbk = elem_grid(rw), nt = 32 * WARPS;
  switch (ops) {
    case OP_A: wb_launch(k_q2_elem<OP_A>, nbk, nt, 0, st, g, rw, tb, u, p, coef, coef_nodal, R, pe); break;
    case OP_BT: wb_launch(k_q2_elem<OP_BT>, nbk, nt, 0, st, g, rw, tb, u, p, coef, coef_nodal, R, pe); break;
    case OP_B: wb_launch(k_q2_elem<OP_B>, nbk, nt, 0, st, g, rw, tb, u, p, coef, coef_nodal, R, pe); break;
    case OP_A | OP_BT | OP_B:
      wb_launch(k_q2_elem<OP_A | OP_BT | OP_B>, nbk, nt, 0, st, g, rw, tb, u, p, coef, coef_nodal, R, pe);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_q2_poisson(const Grid& g, const T* u, const T* coef, T* R, cudaStream_t st) {
  const Rows rw = make_rows(g);
  wb_launch(k_q2_poisson<T>, elem_grid(rw), 32 * WARPS, 0, st, g, rw, q2_tab<T>(g), u, coef, R);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_q2_gather(const Grid& g, int ncomp, int mask_boundary, const T* R, const Epi<T>& e,
                             cudaStream_t st) {
  const Rows rw = make_rows(g);
  dim3 grid;
  int bs;
  node_pass_geometry(g, grid, bs);
  return epi_dispatch(e.mode, [&](auto m) {
    constexpr int MODE = decltype(m)::value;
    if (ncomp == 3)
      wb_launch(k_q2_gather<T, 3, MODE>, grid, bs, 0, st, g, rw.nseg, mask_boundary, R, e);
    else if (ncomp == 1)
      wb_launch(k_q2_gather<T, 1, MODE>, grid, bs, 0, st, g, rw.nseg, mask_boundary, R, e);
    else
      return cudaErrorInvalidValue;
    return cudaGetLastError();
  });
}

template <typename T>
cudaError_t launch_q2_d2c(const Grid& g, const T* rd, T* rc, T* R, cudaStream_t st) {
  const Rows rw = make_rows(g);
  wb_launch(k_q2_d2c<T>, elem_grid(rw), 32 * WARPS, 0, st, g, rw, q2_tab<T>(g), rd, R);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  Epi<T> ep;
  ep.mode = EPI_STORE;
  ep.y = rc;
  return launch_q2_gather<T>(g, 1, 0, R, ep, st);
}

template <typename T>
cudaError_t launch_q2_c2d(const Grid& g, const T* ec, T* ed, int add, cudaStream_t st) {
  const Rows rw = make_rows(g);
  wb_launch(k_q2_c2d<T>, elem_grid(rw), 32 * WARPS, 0, st, g, rw, q2_tab<T>(g), ec, ed, add);
  return cudaGetLastError();
}

template cudaError_t launch_q2_poisson<float>(const Grid&, const float*, const float*, float*, cudaStream_t);
#define WB_Q2_INST(T)                                                                                        \
  template cudaError_t launch_q2_gather<T>(const Grid&, int, int, const T*, const Epi<T>&, cudaStream_t);  \
  template cudaError_t launch_q2_d2c<T>(const Grid&, const T*, T*, T*, cudaStream_t);                       \
  template cudaError_t launch_q2_c2d<T>(const Grid&, const T*, T*, int, cudaStream_t);
WB_Q2_INST(float)
WB_Q2_INST(double)
