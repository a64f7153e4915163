// Per-element arithmetic of the Q2 kernels with one thread per element (q2_ops.cu: element pass
// of the two-pass apply; q2_fused.cu: the fused apply): the single-precision Stokes family and the
// scalar Poisson operator.  The element's 27 nodal values per component sit in registers; the
// gradient at each of the 27 GLL points is formed by 1-D derivative sums along the three axes (sum
// factorisation with the 3 x 3 derivative matrix), then the quadrature-weighted stress (or flux),
// and the transposed derivative sums accumulate into 27 register outputs per component (Sec. 1.2:
// a(u,v) = int 2 mu eps(u):eps(v), b(v,q) = -int q div v).  The operator table (derivatives scaled
// by 2/h, weights times |J|, pressure basis) is a kernel parameter, so every entry is a
// constant-bank operand.
#pragma once

#include "elem_common.cuh"

namespace wb {

__host__ __device__ constexpr int q2i(int i, int j, int l) { return i + 3 * (j + 3 * l); }

// Entries of the Q2 GLL derivative matrix D[i][a] = l_a'(x_i) that can be nonzero: the middle basis
// function is even about the middle node, so D[1][1] = 0 exactly (for every element size, since
// the table holds D scaled by 2/h).  The sums below skip that term at compile time; adding the exact
// zero would not change the result.
__host__ __device__ constexpr bool q2d(int i, int a) { return !(i == 1 && a == 1); }

// The element's nodal values of 3 components starting at node n0 (its lowest corner), with the
// nodes on Dirichlet faces of the domain read as zero; lo_*/hi_*: the element touches that face.
__device__ __forceinline__ void q2_load_u(const float* __restrict__ u, size_t nn, int NX, int NY, int n0, bool act,
                                          bool lo_x, bool hi_x, bool lo_y, bool hi_y, bool lo_z, bool hi_z,
                                          float (&ur)[3][27]) {
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int roff = n0 + NX * (j + NY * l);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const bool bnd = (i == 0 && lo_x) || (i == 2 && hi_x) || (j == 0 && lo_y) || (j == 2 && hi_y) ||
                         (l == 0 && lo_z) || (l == 2 && hi_z);
#pragma unroll
        for (int c = 0; c < 3; ++c) ur[c][q2i(i, j, l)] = (act && !bnd) ? __ldg(u + c * nn + roff + i) : 0.f;
      }
    }
}

// The coefficient at the 27 points: nodal (coef + n0 + node offset) or per element point.
__device__ __forceinline__ void q2_load_coef(const float* __restrict__ base, int nodal, int NX, int NY, bool act,
                                             float (&mur)[27]) {
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int i = q % 3, j = (q / 3) % 3, l = q / 9;
    const int mo = nodal ? i + NX * (j + NY * l) : q;
    mur[q] = act ? __ldg(base + mo) : 0.f;
  }
}

// Point loop of the Stokes family: DA (viscous stress, coefficient mur), DBT (pressure gradient
// from the element's modes pm) and DB (divergence into bacc).  Velocity outputs accumulate into
// out (DA or DBT).
template <bool DA, bool DBT, bool DB>
__device__ __forceinline__ void q2_stokes_points(const OpTab<float, 3>& tb, const float (&ur)[3][27],
                                                 const float (&mur)[27], const float (&pm)[4], float (&out)[3][27],
                                                 float (&bacc)[4]) {
  constexpr bool GRAD = DA || DB, SCAT = DA || DBT;
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int q = q2i(i, j, l);
        const float W = tb.W3[q];
        float G[3][3];
        if (GRAD) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              if (q2d(i, a)) a0 += tb.Ds[0][i][a] * ur[c][q2i(a, j, l)];
              if (q2d(j, a)) a1 += tb.Ds[1][j][a] * ur[c][q2i(i, a, l)];
              if (q2d(l, a)) a2 += tb.Ds[2][l][a] * ur[c][q2i(i, j, a)];
            }
            G[c][0] = a0;
            G[c][1] = a1;
            G[c][2] = a2;
          }
        }
        if (DB) {
          const float dv = W * (G[0][0] + G[1][1] + G[2][2]);
#pragma unroll
          for (int m = 0; m < 4; ++m) bacc[m] -= tb.Psi[q][m] * dv;
        }
        if (SCAT) {
          float sd[3] = {0.f, 0.f, 0.f};   // diagonal stress entries
          float sxy = 0.f, sxz = 0.f, syz = 0.f;
          if (DA) {
            const float f = 2.f * W * mur[q], hf = W * mur[q];
            sd[0] = f * G[0][0];
            sd[1] = f * G[1][1];
            sd[2] = f * G[2][2];
            sxy = hf * (G[0][1] + G[1][0]);
            sxz = hf * (G[0][2] + G[2][0]);
            syz = hf * (G[1][2] + G[2][1]);
          }
          if (DBT) {
            float pq = 0.f;
#pragma unroll
            for (int m = 0; m < 4; ++m) pq += tb.Psi[q][m] * pm[m];
            const float tq = W * pq;
            sd[0] -= tq;
            sd[1] -= tq;
            sd[2] -= tq;
          }
          // output component c, derivative direction d: out_c(node on the d-line) += Ds[d] S_cd
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (q2d(i, a)) out[0][q2i(a, j, l)] += tb.Ds[0][i][a] * sd[0];
            if (q2d(j, a)) out[1][q2i(i, a, l)] += tb.Ds[1][j][a] * sd[1];
            if (q2d(l, a)) out[2][q2i(i, j, a)] += tb.Ds[2][l][a] * sd[2];
            if (DA) {
              if (q2d(j, a)) out[0][q2i(i, a, l)] += tb.Ds[1][j][a] * sxy;
              if (q2d(l, a)) out[0][q2i(i, j, a)] += tb.Ds[2][l][a] * sxz;
              if (q2d(i, a)) out[1][q2i(a, j, l)] += tb.Ds[0][i][a] * sxy;
              if (q2d(l, a)) out[1][q2i(i, j, a)] += tb.Ds[2][l][a] * syz;
              if (q2d(i, a)) out[2][q2i(a, j, l)] += tb.Ds[0][i][a] * sxz;
              if (q2d(j, a)) out[2][q2i(i, a, l)] += tb.Ds[1][j][a] * syz;
            }
          }
        }
      }
}

// One component's 27 nodal values starting at node n0 (no Dirichlet masking: the scalar
// pressure-Poisson operators are Neumann operators).
template <typename T>
__device__ __forceinline__ void q2_load_scalar(const T* __restrict__ u, int NX, int NY, int n0, bool act,
                                               T (&ur)[27]) {
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) ur[q2i(i, j, l)] = act ? __ldg(u + n0 + i + NX * (j + NY * l)) : T(0);
}

// Point loop of the scalar Q2 Poisson operator int c grad u . grad v (the continuous
// pressure-Poisson operator of the two-space cycle, Sec. 6), cf: c at the 27 points.
template <typename T>
__device__ __forceinline__ void q2_poisson_points(const OpTab<T, 3>& tb, const T (&ur)[27], const T (&cf)[27],
                                                  T (&out)[27]) {
#pragma unroll
  for (int l = 0; l < 3; ++l)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int q = q2i(i, j, l);
        T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (q2d(i, a)) a0 += tb.Ds[0][i][a] * ur[q2i(a, j, l)];
          if (q2d(j, a)) a1 += tb.Ds[1][j][a] * ur[q2i(i, a, l)];
          if (q2d(l, a)) a2 += tb.Ds[2][l][a] * ur[q2i(i, j, a)];
        }
        const T f = tb.W3[q] * cf[q];
        a0 *= f;
        a1 *= f;
        a2 *= f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (q2d(i, a)) out[q2i(a, j, l)] += tb.Ds[0][i][a] * a0;
          if (q2d(j, a)) out[q2i(i, a, l)] += tb.Ds[1][j][a] * a1;
          if (q2d(l, a)) out[q2i(i, j, a)] += tb.Ds[2][l][a] * a2;
        }
      }
}

}  // namespace wb
