// Q2 (k = 2) double-precision element passes: one warp per element point, one lane per element.
//
// A block owns a row segment of up to 32 consecutive elements along x (fixed ey, ez) -- the
// segments and row-scratch layout of the single-precision row kernels, so the node pass
// (launch_q2_gather) is shared -- and has 28 warps: one per GLL point of the element (lane e of
// the warp of point q works on point q of element e of the segment) and one spare.  The
// operators are those of Sec. 1.2, a(u, v) = int 2 mu eps(u) : eps(v) and b(v, q) = -int q div v,
// and the scalar Poisson operator int c grad u . grad v of the two-space pressure cycle (Sec. 6),
// all by GLL quadrature at the nodes.
//
// Why this shape.  The FP64 pipe of GB300 retires 2 operations per clock and SM, so the FP64
// passes are bound by their operation count and by how full their warps are.  Every warp here is
// full, and because a warp's point is fixed, each 1-D derivative sum is a constant expression: on
// the Q2 GLL nodes (-1, 0, 1) the derivative matrix is D = Dt / 2 with
//   Dt = [[-3, 4, -1], [-1, 0, 1], [1, -4, 3]]   (row: point, column: basis function),
// so a derivative at a line position costs 2, 1 or 2 operations instead of 3 FMAs, and a
// transposed sum 2 or 3.  On an isotropic mesh (h equal on all axes) the scale kappa = 1/h (the
// physical derivative is kappa Dt) folds into the point weights; otherwise the transposed sums are
// scaled per axis.  The points are spread over the warps so that the four SMSPs get equal FP64
// work (kPermA, kPermP).
//
// Phases per segment k, two barriers each ([load k | A | forward k, finish k-1 | B | backward k]):
//   load      nodal velocity (Dirichlet nodes as zero) from registers into shared [c][q][lane],
//             then the next segment's inputs are requested into registers (software prefetch);
//   forward   the reference derivatives at the warp's point, the weighted stress into shared
//             [slot][q][lane] and, for B, the weighted divergence;
//   backward  y_c at the warp's point, sum over axes d of the transposed derivative sums of the
//             stress S_cd, into the output tile [c][q][lane]; for B, the divergence summed along
//             x-lines;
//   finish    (during the next segment's forward phase) one warp per node x-line (l, j, c) of the
//             segment writes its 65 partial node values (node 2m: point 0 of element m plus point
//             2 of element m - 1; node 2m + 1: point 1 of element m), coalesced; for B four warps
//             finish B u per pressure mode.
// The flat variants at the end serve levels whose rows are too short for full warps.
#include "elem_common.cuh"
#include "epi.cuh"
#include "fused.h"
#include "kernels.h"

namespace {

using namespace wb;

constexpr int NPT = 27;        // element points
constexpr int NWB = 28;        // warps per block: one per element point and one spare (see kPermA)
constexpr int NT = 32 * NWB;
constexpr int PL = NPT * 32;   // doubles per shared plane [q][lane]

// Point of each warp (27: none).  Warp w runs on SMSP w mod 4; the FP64 operations of a point
// depend on its line positions (2, 1, 2 for a derivative, 2, 2, 2 / 3, 2, 3 for a transposed
// sum), so the points are spread such that the four SMSPs get equal shares in the forward and
// backward phases (found by a local search over the per-point operation counts).
constexpr int kPermA[NWB] = {15, 20, 3, 25, 10, 6, 7, 1, 19, 18, 16, 11, 13, 27,
                             4, 5, 8, 2, 17, 22, 21, 24, 12, 9, 23, 0, 26, 14};
constexpr int kPermP[NWB] = {11, 21, 6, 1, 3, 22, 27, 12, 24, 23, 8, 15, 9, 17,
                             0, 14, 13, 5, 20, 25, 16, 4, 26, 10, 19, 7, 18, 2};
__constant__ int c_permA[NWB] = {15, 20, 3, 25, 10, 6, 7, 1, 19, 18, 16, 11, 13, 27,
                                 4, 5, 8, 2, 17, 22, 21, 24, 12, 9, 23, 0, 26, 14};
__constant__ int c_permP[NWB] = {11, 21, 6, 1, 3, 22, 27, 12, 24, 23, 8, 15, 9, 17,
                                 0, 14, 13, 5, 20, 25, 16, 4, 26, 10, 19, 7, 18, 2};

struct Coef64 {
  double H[27];    // isotropic: W_q |J| kappa^2; otherwise W_q |J|
  double T[27];    // isotropic: W_q |J| kappa;   otherwise W_q |J|
  double kap[3];   // kappa_d = 1 / h_d
};

__host__ __device__ constexpr int pt(int i, int j, int l) { return i + 3 * (j + 3 * l); }

// Stress slot of (c, d): the diagonal in 0..2, then xy, xz, yz.
__host__ __device__ constexpr int slot(int c, int d) {
  return c == d ? c : (c + d == 1 ? 3 : (c + d == 2 ? 4 : 5));
}

// Dt[P][.] . (v0, v1, v2): reference derivative at line position P.
template <int P>
__device__ __forceinline__ double dfw(double v0, double v1, double v2) {
  if constexpr (P == 0) return fma(4.0, v1, fma(-3.0, v0, -v2));
  else if constexpr (P == 1) return v2 - v0;
  else return fma(3.0, v2, fma(-4.0, v1, v0));
}
// Dt[.][P] . (s0, s1, s2): transposed sum; column P of Dt is (-3, -1, 1), (4, 0, -4), (-1, 1, 3).
template <int P>
__device__ __forceinline__ double dbw(double s0, double s1, double s2) {
  if constexpr (P == 0) return fma(-3.0, s0, s2 - s1);
  else if constexpr (P == 1) return 4.0 * (s0 - s2);
  else return fma(3.0, s2, s1 - s0);
}
// acc + Dt[.][P] . (s0, s1, s2)
template <int P>
__device__ __forceinline__ double dbw_acc(double s0, double s1, double s2, double acc) {
  if constexpr (P == 0) return fma(-3.0, s0, (acc + s2) - s1);
  else if constexpr (P == 1) return fma(4.0, s0 - s2, acc);
  else return fma(3.0, s2, (acc + s1) - s0);
}

// Shared layout (doubles): velocity [3][q][lane], output [3][q][lane], stress [NS][q][lane],
// weighted divergence [q][lane], divergence x-line sums [2][9][lane], pressure modes [4][lane].
template <int OPS, int YLD = 32>
struct Lay {
  static constexpr bool DA = OPS & OP_A, DBT = OPS & OP_BT, DB = OPS & OP_B;
  static constexpr int NS = DA ? 6 : (DBT ? 1 : 0);
  static constexpr int U = 0;
  static constexpr int Y = U + 3 * PL;   // output [c][q][YLD] (YLD 33: padded for transposed reads)
  static constexpr int S = Y + 3 * NPT * YLD;
  static constexpr int DIV = S + NS * PL;
  static constexpr int RED = DIV + (DB ? PL : 0);
  static constexpr int P = RED + (DB ? 2 * 9 * 32 : 0);
  static constexpr int TOTAL = P + (DBT ? 4 * 32 : 0);
};

template <int OPS, bool ISO, int Q, int YLD = 32>
__device__ __forceinline__ void forward(const Coef64& cf, double* __restrict__ sh, int lane, double mu) {
  using LY = Lay<OPS, YLD>;
  constexpr int I = Q % 3, J = (Q / 3) % 3, L = Q / 9;
  constexpr bool DA = LY::DA, DBT = LY::DBT, DB = LY::DB;
  const double* su = sh + LY::U + lane;
  double* sS = sh + LY::S + Q * 32 + lane;   // this point's entry of stress plane `slot`: sS[slot * PL]
  auto U = [&](int c, int qq) { return su[(c * NPT + qq) * 32]; };
  // reference derivatives g[c][d] = Dt-sum of component c along axis d (only the diagonal for B)
  double g[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (!(DA || DB)) break;
    if (DA || c == 0) g[c][0] = dfw<I>(U(c, pt(0, J, L)), U(c, pt(1, J, L)), U(c, pt(2, J, L)));
    if (DA || c == 1) g[c][1] = dfw<J>(U(c, pt(I, 0, L)), U(c, pt(I, 1, L)), U(c, pt(I, 2, L)));
    if (DA || c == 2) g[c][2] = dfw<L>(U(c, pt(I, J, 0)), U(c, pt(I, J, 1)), U(c, pt(I, J, 2)));
  }
  if constexpr (DB) {
    // W_q |J| div u = T_q (kappa-weighted trace of g)
    const double tr = ISO ? (g[0][0] + g[1][1]) + g[2][2]
                          : fma(cf.kap[2], g[2][2], fma(cf.kap[1], g[1][1], cf.kap[0] * g[0][0]));
    sh[LY::DIV + Q * 32 + lane] = cf.T[Q] * tr;
  }
  double t = 0.0;
  if constexpr (DBT) {
    // p at the point: psi = (1, xi, eta, zeta) on the nodes -1, 0, 1
    const double* sp = sh + LY::P + lane;
    double pq = sp[0];
    if constexpr (I == 0) pq -= sp[32];
    if constexpr (I == 2) pq += sp[32];
    if constexpr (J == 0) pq -= sp[64];
    if constexpr (J == 2) pq += sp[64];
    if constexpr (L == 0) pq -= sp[96];
    if constexpr (L == 2) pq += sp[96];
    t = cf.T[Q] * pq;
  }
  if constexpr (DA) {
    const double h = cf.H[Q] * mu;
    if constexpr (ISO) {
      // kappa S: diagonal 2 h g_cc - t, off-diagonal h (g_cd + g_dc)
      const double f = h + h;
#pragma unroll
      for (int c = 0; c < 3; ++c) sS[slot(c, c) * PL] = DBT ? fma(f, g[c][c], -t) : f * g[c][c];
      sS[3 * PL] = h * (g[0][1] + g[1][0]);
      sS[4 * PL] = h * (g[0][2] + g[2][0]);
      sS[5 * PL] = h * (g[1][2] + g[2][1]);
    } else {
      // S: diagonal 2 h kappa_c g_cc - t, off-diagonal h (kappa_d g_cd + kappa_c g_dc)
      const double hk[3] = {h * cf.kap[0], h * cf.kap[1], h * cf.kap[2]};
#pragma unroll
      for (int c = 0; c < 3; ++c) sS[slot(c, c) * PL] = fma(hk[c], g[c][c], fma(hk[c], g[c][c], -t));
      sS[3 * PL] = fma(hk[1], g[0][1], hk[0] * g[1][0]);
      sS[4 * PL] = fma(hk[2], g[0][2], hk[0] * g[2][0]);
      sS[5 * PL] = fma(hk[2], g[1][2], hk[1] * g[2][1]);
    }
  } else if constexpr (DBT) {
    sS[0] = -t;
  }
}

template <int OPS, bool ISO, int Q, int YLD = 32>
__device__ __forceinline__ void backward(const Coef64& cf, double* __restrict__ sh, int lane) {
  using LY = Lay<OPS, YLD>;
  constexpr int I = Q % 3, J = (Q / 3) % 3, L = Q / 9;
  constexpr bool DA = LY::DA;
  const double* sS = sh + LY::S + lane;
  double* sy = sh + LY::Y + lane;
  auto S = [&](int s, int qq) { return sS[(s * NPT + qq) * 32]; };
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double y;
    if constexpr (DA) {
      const int s0 = slot(c, 0), s1 = slot(c, 1), s2 = slot(c, 2);
      if constexpr (ISO) {
        y = dbw<I>(S(s0, pt(0, J, L)), S(s0, pt(1, J, L)), S(s0, pt(2, J, L)));
        y = dbw_acc<J>(S(s1, pt(I, 0, L)), S(s1, pt(I, 1, L)), S(s1, pt(I, 2, L)), y);
        y = dbw_acc<L>(S(s2, pt(I, J, 0)), S(s2, pt(I, J, 1)), S(s2, pt(I, J, 2)), y);
      } else {
        y = cf.kap[0] * dbw<I>(S(s0, pt(0, J, L)), S(s0, pt(1, J, L)), S(s0, pt(2, J, L)));
        y = fma(cf.kap[1], dbw<J>(S(s1, pt(I, 0, L)), S(s1, pt(I, 1, L)), S(s1, pt(I, 2, L))), y);
        y = fma(cf.kap[2], dbw<L>(S(s2, pt(I, J, 0)), S(s2, pt(I, J, 1)), S(s2, pt(I, J, 2))), y);
      }
    } else {
      // B^T alone: the stress is -t on the diagonal, so only axis c contributes to y_c
      if (c == 0) y = dbw<I>(S(0, pt(0, J, L)), S(0, pt(1, J, L)), S(0, pt(2, J, L)));
      else if (c == 1) y = dbw<J>(S(0, pt(I, 0, L)), S(0, pt(I, 1, L)), S(0, pt(I, 2, L)));
      else y = dbw<L>(S(0, pt(I, J, 0)), S(0, pt(I, J, 1)), S(0, pt(I, J, 2)));
      if constexpr (!ISO) y *= cf.kap[c];
    }
    sy[(c * NPT + Q) * YLD] = y;
  }
}

#define WB_W28(X) X(0) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) \
  X(14) X(15) X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27)

// Segment index -> first element row and element coordinates.
struct Seg {
  int seg, ey, ez, last;   // last: lane of the segment's last element
};

__device__ __forceinline__ Seg seg_of(const Grid& g, const Rows& rw, int w) {
  Seg s;
  const unsigned rest = fdiv((unsigned)w, rw.fseg);
  s.seg = w - (int)rest * rw.nseg;
  s.ez = (int)fdiv(rest, rw.fny);
  s.ey = (int)rest - s.ez * g.ny;
  s.last = min(Q2_SEG - 1, g.nx - 1 - s.seg * Q2_SEG);
  return s;
}

// Node x-lines of a finished segment from the output tile, and B u for its elements.
template <int OPS>
__device__ __forceinline__ void finish_seg(const Grid& g, const Seg& s, const double* __restrict__ sh, int warp,
                                           int lane, double* __restrict__ R, const Epi<double>& pe) {
  using LY = Lay<OPS>;
  if ((LY::DA || LY::DBT) && warp < 27) {
    // warp = (jl, c) owns the node x-line (j, l) of component c
    const int jl = warp / 3, c = warp - 3 * jl;
    const double* y0 = sh + LY::Y + (c * NPT + 3 * jl) * 32;   // points 0, 1, 2 of the line
    double* row = R + ((((size_t)s.seg * g.nz + s.ez) * g.ny + s.ey) * 9 + jl) * 3 * Q2_ROW_LD +
                  (size_t)c * Q2_ROW_LD;
    const int xmax = 2 * s.last + 2;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int X = lane + 32 * k;
      if (X <= xmax) {
        const int m = X >> 1;
        double v;
        if (X & 1) {
          v = y0[32 + m];
        } else {
          v = m <= s.last ? y0[m] : 0.0;
          if (m >= 1) v += y0[64 + m - 1];
        }
        row[X] = v;
      }
    }
  }
  if (LY::DB && warp < 4 && lane <= s.last) {
    // B u = -sum_q psi_m(q) W_q |J| div u(q); psi = (1, xi, eta, zeta), x-line jl = j + 3 l
    const double* T = sh + LY::RED + lane;
    const double* X = T + 9 * 32;
    double v;
    if (warp == 0) {
      v = T[0];
#pragma unroll
      for (int jl = 1; jl < 9; ++jl) v += T[jl * 32];
    } else if (warp == 1) {
      v = X[0];
#pragma unroll
      for (int jl = 1; jl < 9; ++jl) v += X[jl * 32];
    } else if (warp == 2) {
      v = T[2 * 32] - T[0];
#pragma unroll
      for (int l = 1; l < 3; ++l) v += T[(2 + 3 * l) * 32] - T[(3 * l) * 32];
    } else {
      v = T[6 * 32] - T[0];
#pragma unroll
      for (int j = 1; j < 3; ++j) v += T[(j + 6) * 32] - T[j * 32];
    }
    const int e = s.seg * Q2_SEG + lane + g.nx * (s.ey + g.ny * s.ez);
    epi_apply(pe, (size_t)e * 4 + warp, 0, -v);
  }
}

// Two barriers per segment: [load k | A | forward k, finish k-1 | B | backward k].  Hazards:
// the velocity tile is written (load k+1) after barrier B of k, when forward k has read it; the
// stress and divergence are written (forward k+1) after barrier A of k+1, when backward k has read
// them; the output tile and line sums are written (backward k+1) after barrier B of k+1, when
// finish k (in the forward phase of k+1) has read them.
template <int OPS, bool ISO>
__global__ void __launch_bounds__(NT, 1)
k_q2_elem64(Grid g, Rows rw, const __grid_constant__ Coef64 cf, const double* __restrict__ u,
            const double* __restrict__ p, const double* __restrict__ coef, int coef_nodal, double* __restrict__ R,
            Epi<double> pe) {
  pdl_entry();
  using LY = Lay<OPS>;
  constexpr bool DA = LY::DA, DBT = LY::DBT, DB = LY::DB, GRAD = DA || DB, SCAT = DA || DBT;
  extern __shared__ double sh[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = c_permA[warp];   // this warp's element point (27: none)
  const int I = q % 3, J = (q / 3) % 3, L = q / 9;
  const size_t nn = (size_t)g.nn;

  // inputs of one segment for this thread (point q of element `lane`)
  double un[3] = {0.0, 0.0, 0.0}, mun = 0.0, pn = 0.0;
  auto fetch = [&](int w) {
    const Seg s = seg_of(g, rw, w);
    const int ex = s.seg * Q2_SEG + lane;
    const bool act = lane <= s.last && q < NPT;
    const int ix = 2 * ex + I, iy = 2 * s.ey + J, iz = 2 * s.ez + L;
    const int n = ix + g.NX * (iy + g.NY * iz);
    const int e = ex + g.nx * (s.ey + g.ny * s.ez);
    if (GRAD) {
      const bool live = act && !on_boundary(g, ix, iy, iz);
#pragma unroll
      for (int c = 0; c < 3; ++c) un[c] = live ? __ldg(u + c * nn + n) : 0.0;
    }
    if (DA) mun = act ? __ldg(coef_nodal ? coef + n : coef + (size_t)e * 27 + q) : 0.0;
    if (DBT && warp < 4) pn = lane <= s.last ? __ldg(p + (size_t)e * 4 + warp) : 0.0;
  };

  int w = blockIdx.x;
  if (w >= rw.nrows) return;   // whole block
  fetch(w);
  Seg prev{0, 0, 0, -1};
  for (; w < rw.nrows; w += gridDim.x) {
    const Seg s = seg_of(g, rw, w);
    // load
    if (GRAD && q < NPT) {
#pragma unroll
      for (int c = 0; c < 3; ++c) sh[LY::U + (c * NPT + q) * 32 + lane] = un[c];
    }
    if (DBT && warp < 4) sh[LY::P + warp * 32 + lane] = pn;
    const double mu = mun;
    __syncthreads();
    if (w + (int)gridDim.x < rw.nrows) fetch(w + gridDim.x);
    // forward k; the previous segment's output goes out meanwhile
    switch (warp) {
#define WB_F(W) \
  case W: if constexpr (kPermA[W] < NPT) forward<OPS, ISO, kPermA[W]>(cf, sh, lane, mu); break;
      WB_W28(WB_F)
#undef WB_F
    }
    if (prev.last >= 0) finish_seg<OPS>(g, prev, sh, warp, lane, R, pe);
    __syncthreads();
    // backward (and, for B, x-line sums of the weighted divergence: T = d0 + d1 + d2, X = d2 - d0)
    if (SCAT) {
      switch (warp) {
#define WB_B(W) \
  case W: if constexpr (kPermA[W] < NPT) backward<OPS, ISO, kPermA[W]>(cf, sh, lane); break;
        WB_W28(WB_B)
#undef WB_B
      }
    }
    if (DB && warp < 9) {
      const double* dv = sh + LY::DIV + lane;
      const double d0 = dv[(3 * warp) * 32], d1 = dv[(3 * warp + 1) * 32], d2 = dv[(3 * warp + 2) * 32];
      sh[LY::RED + warp * 32 + lane] = (d0 + d1) + d2;
      sh[LY::RED + (9 + warp) * 32 + lane] = d2 - d0;
    }
    prev = s;
  }
  __syncthreads();
  finish_seg<OPS>(g, prev, sh, warp, lane, R, pe);
}

// Scalar Q2 Poisson element pass (the continuous Q2 level of the two-space pressure cycle, Sec.
// 6: int c grad u . grad v, c per element point, no Dirichlet rows), same segment and warp
// layout and the same two-barrier pipeline: y = sum_d Dt^T (W_q |J| kappa_d^2 c g_d), g_d the
// reference derivative along axis d.  Shared: u [q][lane], output [q][lane], fluxes [3][q][lane].
struct PoisCoef64 {
  double Wk[3][27];   // W_q |J| kappa_d^2
};

// Poisson shared layout (doubles): u [q][32], output [q][YLD], fluxes [3][q][32] from pois_F.
template <int YLD>
__host__ __device__ constexpr int pois_F() { return PL + NPT * YLD; }

template <bool ISO, int Q, int YLD = 32>
__device__ __forceinline__ void pois_forward(const PoisCoef64& cf, double* __restrict__ sh, int lane, double c) {
  constexpr int I = Q % 3, J = (Q / 3) % 3, L = Q / 9;
  const double* su = sh + lane;
  double* sF = sh + pois_F<YLD>() + Q * 32 + lane;
  const double g0 = dfw<I>(su[pt(0, J, L) * 32], su[pt(1, J, L) * 32], su[pt(2, J, L) * 32]);
  const double g1 = dfw<J>(su[pt(I, 0, L) * 32], su[pt(I, 1, L) * 32], su[pt(I, 2, L) * 32]);
  const double g2 = dfw<L>(su[pt(I, J, 0) * 32], su[pt(I, J, 1) * 32], su[pt(I, J, 2) * 32]);
  if constexpr (ISO) {
    const double f = cf.Wk[0][Q] * c;
    sF[0] = f * g0;
    sF[PL] = f * g1;
    sF[2 * PL] = f * g2;
  } else {
    sF[0] = cf.Wk[0][Q] * c * g0;
    sF[PL] = cf.Wk[1][Q] * c * g1;
    sF[2 * PL] = cf.Wk[2][Q] * c * g2;
  }
}

template <int Q, int YLD = 32>
__device__ __forceinline__ void pois_backward(double* __restrict__ sh, int lane) {
  constexpr int I = Q % 3, J = (Q / 3) % 3, L = Q / 9;
  const double* sF = sh + pois_F<YLD>() + lane;
  double y = dbw<I>(sF[pt(0, J, L) * 32], sF[pt(1, J, L) * 32], sF[pt(2, J, L) * 32]);
  y = dbw_acc<J>(sF[PL + pt(I, 0, L) * 32], sF[PL + pt(I, 1, L) * 32], sF[PL + pt(I, 2, L) * 32], y);
  y = dbw_acc<L>(sF[2 * PL + pt(I, J, 0) * 32], sF[2 * PL + pt(I, J, 1) * 32], sF[2 * PL + pt(I, J, 2) * 32], y);
  sh[PL + Q * YLD + lane] = y;
}

constexpr int POIS_SMEM = 5 * PL;                       // doubles, row kernel
constexpr int POIS_SMEM_FLAT = pois_F<33>() + 3 * PL;   // doubles, flat kernel

__device__ __forceinline__ void pois_finish(const Grid& g, const Seg& s, const double* __restrict__ sh, int warp,
                                            int lane, double* __restrict__ R) {
  if (warp >= 9) return;
  // node x-line jl = warp of the segment: node 2m = point 0 of element m + point 2 of m - 1
  const double* y0 = sh + PL + 3 * warp * 32;
  double* row = R + (((size_t)s.seg * g.nz + s.ez) * g.ny + s.ey) * 9 * Q2_ROW_LD + (size_t)warp * Q2_ROW_LD;
  const int xmax = 2 * s.last + 2;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int X = lane + 32 * k;
    if (X <= xmax) {
      const int m = X >> 1;
      double v;
      if (X & 1) {
        v = y0[32 + m];
      } else {
        v = m <= s.last ? y0[m] : 0.0;
        if (m >= 1) v += y0[64 + m - 1];
      }
      row[X] = v;
    }
  }
}

template <bool ISO>
__global__ void __launch_bounds__(NT, 2)
k_q2_poisson64(Grid g, Rows rw, const __grid_constant__ PoisCoef64 cf, const double* __restrict__ u,
               const double* __restrict__ coef, double* __restrict__ R) {
  pdl_entry();
  extern __shared__ double sh[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = c_permP[warp];   // this warp's element point (27: none)
  const int I = q % 3, J = (q / 3) % 3, L = q / 9;
  double un = 0.0, cn = 0.0;
  auto fetch = [&](int w) {
    const Seg s = seg_of(g, rw, w);
    const int ex = s.seg * Q2_SEG + lane;
    if (lane <= s.last && q < NPT) {
      const int n = (2 * ex + I) + g.NX * ((2 * s.ey + J) + g.NY * (2 * s.ez + L));
      un = __ldg(u + n);
      cn = __ldg(coef + (size_t)(ex + g.nx * (s.ey + g.ny * s.ez)) * 27 + q);
    } else {
      un = 0.0;
      cn = 0.0;
    }
  };
  int w = blockIdx.x;
  if (w >= rw.nrows) return;
  fetch(w);
  Seg prev{0, 0, 0, -1};
  for (; w < rw.nrows; w += gridDim.x) {
    const Seg s = seg_of(g, rw, w);
    if (q < NPT) sh[q * 32 + lane] = un;
    const double c = cn;
    __syncthreads();
    if (w + (int)gridDim.x < rw.nrows) fetch(w + gridDim.x);
    switch (warp) {
#define WB_F(W) \
  case W: if constexpr (kPermP[W] < NPT) pois_forward<ISO, kPermP[W]>(cf, sh, lane, c); break;
      WB_W28(WB_F)
#undef WB_F
    }
    if (prev.last >= 0) pois_finish(g, prev, sh, warp, lane, R);
    __syncthreads();
    switch (warp) {
#define WB_B(W) \
  case W: if constexpr (kPermP[W] < NPT) pois_backward<kPermP[W]>(sh, lane); break;
      WB_W28(WB_B)
#undef WB_B
    }
    prev = s;
  }
  __syncthreads();
  pois_finish(g, prev, sh, warp, lane, R);
}

// ---- Flat variants for levels below the row-segment size (k = 2, FP64): block w owns the 32
// consecutive elements 32 w .. 32 w + 31 in linear order (lane = element), so short rows still
// fill the warps; the output goes to the element-major scratch [E][ncomp][27] of the per-point
// kernels (read by their node pass), written through the padded tile [c][q][33] so that the
// transposed reads are nearly free of bank conflicts.  A only (coarse levels apply nothing else).
constexpr int FLAT_YLD = 33;

template <bool ISO>
__global__ void __launch_bounds__(NT, 1)
k_q2_elem64_flat(Grid g, int nblk, const __grid_constant__ Coef64 cf, const double* __restrict__ u,
                 const double* __restrict__ coef, int coef_nodal, double* __restrict__ Ye) {
  pdl_entry();
  using LY = Lay<OP_A, FLAT_YLD>;
  extern __shared__ double sh[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = c_permA[warp];
  const int I = q % 3, J = (q / 3) % 3, L = q / 9;
  const size_t nn = (size_t)g.nn;
  double un[3] = {0.0, 0.0, 0.0}, mun = 0.0;
  auto fetch = [&](int w) {
    const int e = w * 32 + lane;
    const bool act = e < g.ne && q < NPT;
    const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
    const int ix = 2 * ex + I, iy = 2 * ey + J, iz = 2 * ez + L;
    const int n = ix + g.NX * (iy + g.NY * iz);
    const bool live = act && !on_boundary(g, ix, iy, iz);
#pragma unroll
    for (int c = 0; c < 3; ++c) un[c] = live ? __ldg(u + c * nn + n) : 0.0;
    mun = act ? __ldg(coef_nodal ? coef + n : coef + (size_t)e * 27 + q) : 0.0;
  };
  // element-major store of a finished block of elements from the output tile
  auto finish = [&](int w) {
    const int e0 = w * 32, cnt = min(32, g.ne - e0);
    for (int t = threadIdx.x; t < cnt * 81; t += NT) {
      const int el = t / 81, r = t - 81 * el, c = r / 27, qq = r - 27 * c;
      Ye[(size_t)e0 * 81 + t] = sh[LY::Y + (c * NPT + qq) * FLAT_YLD + el];
    }
  };
  int w = blockIdx.x;
  if (w >= nblk) return;
  fetch(w);
  int prev = -1;
  for (; w < nblk; w += gridDim.x) {
    if (q < NPT) {
#pragma unroll
      for (int c = 0; c < 3; ++c) sh[LY::U + (c * NPT + q) * 32 + lane] = un[c];
    }
    const double mu = mun;
    __syncthreads();
    if (w + (int)gridDim.x < nblk) fetch(w + gridDim.x);
    switch (warp) {
#define WB_F(W) \
  case W: if constexpr (kPermA[W] < NPT) forward<OP_A, ISO, kPermA[W], FLAT_YLD>(cf, sh, lane, mu); break;
      WB_W28(WB_F)
#undef WB_F
    }
    if (prev >= 0) finish(prev);
    __syncthreads();
    switch (warp) {
#define WB_B(W) \
  case W: if constexpr (kPermA[W] < NPT) backward<OP_A, ISO, kPermA[W], FLAT_YLD>(cf, sh, lane); break;
      WB_W28(WB_B)
#undef WB_B
    }
    prev = w;
  }
  __syncthreads();
  finish(prev);
}

template <bool ISO>
__global__ void __launch_bounds__(NT, 2)
k_q2_poisson64_flat(Grid g, int nblk, const __grid_constant__ PoisCoef64 cf, const double* __restrict__ u,
                    const double* __restrict__ coef, double* __restrict__ Ye) {
  pdl_entry();
  extern __shared__ double sh[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = c_permP[warp];
  const int I = q % 3, J = (q / 3) % 3, L = q / 9;
  double un = 0.0, cn = 0.0;
  auto fetch = [&](int w) {
    const int e = w * 32 + lane;
    if (e < g.ne && q < NPT) {
      const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
      un = __ldg(u + (2 * ex + I) + g.NX * ((2 * ey + J) + g.NY * (2 * ez + L)));
      cn = __ldg(coef + (size_t)e * 27 + q);
    } else {
      un = 0.0;
      cn = 0.0;
    }
  };
  auto finish = [&](int w) {
    const int e0 = w * 32, cnt = min(32, g.ne - e0);
    for (int t = threadIdx.x; t < cnt * 27; t += NT) {
      const int el = t / 27, qq = t - 27 * el;
      Ye[(size_t)e0 * 27 + t] = sh[PL + qq * FLAT_YLD + el];
    }
  };
  int w = blockIdx.x;
  if (w >= nblk) return;
  fetch(w);
  int prev = -1;
  for (; w < nblk; w += gridDim.x) {
    if (q < NPT) sh[q * 32 + lane] = un;
    const double c = cn;
    __syncthreads();
    if (w + (int)gridDim.x < nblk) fetch(w + gridDim.x);
    switch (warp) {
#define WB_F(W) \
  case W: if constexpr (kPermP[W] < NPT) pois_forward<ISO, kPermP[W], FLAT_YLD>(cf, sh, lane, c); break;
      WB_W28(WB_F)
#undef WB_F
    }
    if (prev >= 0) finish(prev);
    __syncthreads();
    switch (warp) {
#define WB_B(W) \
  case W: if constexpr (kPermP[W] < NPT) pois_backward<kPermP[W], FLAT_YLD>(sh, lane); break;
      WB_W28(WB_B)
#undef WB_B
    }
    prev = w;
  }
  __syncthreads();
  finish(prev);
}

int g_nsm = 0;

// Per instantiation: the dynamic shared-memory opt-in and the resident blocks per SM, set once
// (q2_elem64_prepare, called at context creation, before any stream capture).
template <int OPS, bool ISO>
int& blocks_per_sm() {
  static int b = -1;
  return b;
}

template <int OPS, bool ISO>
cudaError_t prepare_one() {
  constexpr size_t smem = sizeof(double) * Lay<OPS>::TOTAL;
  if (blocks_per_sm<OPS, ISO>() > 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_q2_elem64<OPS, ISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_q2_elem64<OPS, ISO>, NT, smem)) != cudaSuccess)
    return e;
  blocks_per_sm<OPS, ISO>() = occ > 0 ? occ : 1;
  return cudaSuccess;
}

template <int OPS, bool ISO>
cudaError_t launch_one(const Grid& g, const Rows& rw, const Coef64& cf, const double* u, const double* p,
                       const double* coef, int coef_nodal, double* R, const Epi<double>& pe, cudaStream_t st) {
  if (blocks_per_sm<OPS, ISO>() < 0) {
    const cudaError_t e = q2_elem64_prepare();
    if (e != cudaSuccess) return e;
  }
  const long long cap = (long long)g_nsm * blocks_per_sm<OPS, ISO>();
  const unsigned grid = (unsigned)(rw.nrows < cap ? rw.nrows : cap);
  wb_launch(k_q2_elem64<OPS, ISO>, grid, NT, sizeof(double) * Lay<OPS>::TOTAL, st, g, rw, cf, u, p, coef, coef_nodal,
            R, pe);
  return cudaGetLastError();
}

template <bool ISO>
int& pois_blocks_per_sm() {
  static int b = -1;
  return b;
}

template <bool ISO>
cudaError_t prepare_pois() {
  constexpr size_t smem = sizeof(double) * POIS_SMEM;
  if (pois_blocks_per_sm<ISO>() > 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_q2_poisson64<ISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_q2_poisson64<ISO>, NT, smem)) != cudaSuccess) return e;
  pois_blocks_per_sm<ISO>() = occ > 0 ? occ : 1;
  return cudaSuccess;
}

template <bool ISO>
cudaError_t launch_pois(const Grid& g, const Rows& rw, const PoisCoef64& cf, const double* u, const double* coef,
                        double* R, cudaStream_t st) {
  if (pois_blocks_per_sm<ISO>() < 0) {
    const cudaError_t e = q2_elem64_prepare();
    if (e != cudaSuccess) return e;
  }
  const long long cap = (long long)g_nsm * pois_blocks_per_sm<ISO>();
  const unsigned grid = (unsigned)(rw.nrows < cap ? rw.nrows : cap);
  wb_launch(k_q2_poisson64<ISO>, grid, NT, sizeof(double) * POIS_SMEM, st, g, rw, cf, u, coef, R);
  return cudaGetLastError();
}

template <typename K>
cudaError_t prepare_kernel(K kernel, size_t smem, int& bps) {
  if (bps > 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, NT, smem)) != cudaSuccess) return e;
  bps = occ > 0 ? occ : 1;
  return cudaSuccess;
}

int g_flat_bps[2][2] = {{-1, -1}, {-1, -1}};   // [pass: 0 A, 1 Poisson][ISO]
constexpr size_t FLAT_A_SMEM = sizeof(double) * Lay<OP_A, FLAT_YLD>::TOTAL;
constexpr size_t FLAT_P_SMEM = sizeof(double) * POIS_SMEM_FLAT;

cudaError_t prepare_flat() {
  cudaError_t e;
  if ((e = prepare_kernel(k_q2_elem64_flat<false>, FLAT_A_SMEM, g_flat_bps[0][0])) != cudaSuccess) return e;
  if ((e = prepare_kernel(k_q2_elem64_flat<true>, FLAT_A_SMEM, g_flat_bps[0][1])) != cudaSuccess) return e;
  if ((e = prepare_kernel(k_q2_poisson64_flat<false>, FLAT_P_SMEM, g_flat_bps[1][0])) != cudaSuccess) return e;
  return prepare_kernel(k_q2_poisson64_flat<true>, FLAT_P_SMEM, g_flat_bps[1][1]);
}

unsigned flat_grid(int nblk, int bps) {
  const long long cap = (long long)g_nsm * bps;
  return (unsigned)(nblk < cap ? nblk : cap);
}

}  // namespace

cudaError_t launch_q2_elem64_flat(const Grid& g, const double* u, const double* coef, int coef_nodal, double* Ye,
                                  cudaStream_t st) {
  const int nblk = (g.ne + 31) / 32;
  if (nblk == 0) return cudaSuccess;
  if (g_flat_bps[0][0] < 0) {
    const cudaError_t e = q2_elem64_prepare();
    if (e != cudaSuccess) return e;
  }
  const bool iso = g.h[0] == g.h[1] && g.h[1] == g.h[2];
  const double w1[3] = {1.0 / 3.0, 4.0 / 3.0, 1.0 / 3.0};
  Coef64 cf;
  for (int d = 0; d < 3; ++d) cf.kap[d] = 0.5 * g.s[d];
  for (int q = 0; q < 27; ++q) {
    const double W = w1[q % 3] * w1[(q / 3) % 3] * w1[q / 9] * g.detJ;
    cf.H[q] = iso ? W * cf.kap[0] * cf.kap[0] : W;
    cf.T[q] = iso ? W * cf.kap[0] : W;
  }
  if (iso)
    wb_launch(k_q2_elem64_flat<true>, flat_grid(nblk, g_flat_bps[0][1]), NT, FLAT_A_SMEM, st, g, nblk, cf, u, coef,
              coef_nodal, Ye);
  else
    wb_launch(k_q2_elem64_flat<false>, flat_grid(nblk, g_flat_bps[0][0]), NT, FLAT_A_SMEM, st, g, nblk, cf, u, coef,
              coef_nodal, Ye);
  return cudaGetLastError();
}

cudaError_t launch_q2_poisson64_flat(const Grid& g, const double* u, const double* coef, double* Ye, cudaStream_t st) {
  const int nblk = (g.ne + 31) / 32;
  if (nblk == 0) return cudaSuccess;
  if (g_flat_bps[1][0] < 0) {
    const cudaError_t e = q2_elem64_prepare();
    if (e != cudaSuccess) return e;
  }
  const bool iso = g.h[0] == g.h[1] && g.h[1] == g.h[2];
  const double w1[3] = {1.0 / 3.0, 4.0 / 3.0, 1.0 / 3.0};
  PoisCoef64 cf;
  for (int q = 0; q < 27; ++q) {
    const double W = w1[q % 3] * w1[(q / 3) % 3] * w1[q / 9] * g.detJ;
    for (int d = 0; d < 3; ++d) cf.Wk[d][q] = W * (0.25 * g.s[d] * g.s[d]);
  }
  if (iso)
    wb_launch(k_q2_poisson64_flat<true>, flat_grid(nblk, g_flat_bps[1][1]), NT, FLAT_P_SMEM, st, g, nblk, cf, u, coef,
              Ye);
  else
    wb_launch(k_q2_poisson64_flat<false>, flat_grid(nblk, g_flat_bps[1][0]), NT, FLAT_P_SMEM, st, g, nblk, cf, u,
              coef, Ye);
  return cudaGetLastError();
}

cudaError_t q2_elem64_prepare() {
  if (g_nsm == 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e;
  if ((e = prepare_one<OP_A, true>()) != cudaSuccess) return e;
  if ((e = prepare_one<OP_A, false>()) != cudaSuccess) return e;
  if ((e = prepare_one<OP_A | OP_BT | OP_B, true>()) != cudaSuccess) return e;
  if ((e = prepare_one<OP_A | OP_BT | OP_B, false>()) != cudaSuccess) return e;
  if ((e = prepare_one<OP_BT, false>()) != cudaSuccess) return e;
  if ((e = prepare_one<OP_B, false>()) != cudaSuccess) return e;
  if ((e = prepare_pois<true>()) != cudaSuccess) return e;
  if ((e = prepare_pois<false>()) != cudaSuccess) return e;
  return prepare_flat();
}

cudaError_t launch_q2_poisson64(const Grid& g, const double* u, const double* coef, double* R, cudaStream_t st) {
  const Rows rw = make_rows(g);
  if (rw.nrows == 0) return cudaSuccess;
  const bool iso = g.h[0] == g.h[1] && g.h[1] == g.h[2];
  const double w1[3] = {1.0 / 3.0, 4.0 / 3.0, 1.0 / 3.0};
  PoisCoef64 cf;
  for (int q = 0; q < 27; ++q) {
    const double W = w1[q % 3] * w1[(q / 3) % 3] * w1[q / 9] * g.detJ;
    for (int d = 0; d < 3; ++d) cf.Wk[d][q] = W * (0.25 * g.s[d] * g.s[d]);
  }
  return iso ? launch_pois<true>(g, rw, cf, u, coef, R, st) : launch_pois<false>(g, rw, cf, u, coef, R, st);
}

cudaError_t launch_q2_elem64(const Grid& g, int ops, const double* u, const double* p, const double* coef,
                             int coef_nodal, double* R, const Epi<double>& pe, cudaStream_t st) {
  const Rows rw = make_rows(g);
  if (rw.nrows == 0) return cudaSuccess;
  // the isotropic form is taken by the passes with A (B^T or B alone have little FP64 work)
  const bool iso = (ops & OP_A) && g.h[0] == g.h[1] && g.h[1] == g.h[2];
  // GLL weights of the Q2 nodes (-1, 0, 1): 1/3, 4/3, 1/3
  const double w1[3] = {1.0 / 3.0, 4.0 / 3.0, 1.0 / 3.0};
  Coef64 cf;
  for (int d = 0; d < 3; ++d) cf.kap[d] = 0.5 * g.s[d];
  for (int q = 0; q < 27; ++q) {
    const double W = w1[q % 3] * w1[(q / 3) % 3] * w1[q / 9] * g.detJ;
    cf.H[q] = iso ? W * cf.kap[0] * cf.kap[0] : W;
    cf.T[q] = iso ? W * cf.kap[0] : W;
  }
  switch (ops) {
    case OP_A:
      return iso ? launch_one<OP_A, true>(g, rw, cf, u, p, coef, coef_nodal, R, pe, st)
                 : launch_one<OP_A, false>(g, rw, cf, u, p, coef, coef_nodal, R, pe, st);
    case OP_A | OP_BT | OP_B:
      return iso ? launch_one<OP_A | OP_BT | OP_B, true>(g, rw, cf, u, p, coef, coef_nodal, R, pe, st)
                 : launch_one<OP_A | OP_BT | OP_B, false>(g, rw, cf, u, p, coef, coef_nodal, R, pe, st);
    case OP_BT: return launch_one<OP_BT, false>(g, rw, cf, u, p, coef, coef_nodal, R, pe, st);
    case OP_B: return launch_one<OP_B, false>(g, rw, cf, u, p, coef, coef_nodal, R, pe, st);
    default: return cudaErrorInvalidValue;
  }
}
