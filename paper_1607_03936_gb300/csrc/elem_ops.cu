// Element-batched, sum-factorised Q_k x P_{k-1}^disc operators (Sec. 1.2) and the
// setup kernels that share their index maps: diagonals, lumped weights, coefficient
// coarsening, pressure transfers and nested Q_k transfers (Sec. 6).
//
// Thread mapping: one thread per element point, EPB elements per block.  The
// element tile (velocity, coefficient) is gathered into shared memory, gradients
// are formed by 1-D derivative sums along each axis (n FMAs per entry), the
// quadrature-weighted stress is stored back, and the transposed derivative sums
// give each node's contribution.  Scatter-add is deterministic: an apply runs
// as 8 launches, one per parity colour (ex%2, ey%2, ez%2); elements of one colour
// share no nodes, so every node is updated by plain read-modify-writes in a
// fixed colour order.
#include "elem_common.cuh"
#include "kernels.h"

namespace {

using namespace wb;

// Colour-scatter kernels (used by the allocation-free entry point) build their tables in the block.
template <typename T, int N>
__device__ inline void load_optab(OpTab<T, N>& s, const RefTables* __restrict__ tab, const Grid& g, bool need_psi) {
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP;
  for (int t = threadIdx.x; t < 3 * N * N; t += blockDim.x) {
    const int d = t / (N * N), r = t % (N * N);
    s.Ds[d][r / N][r % N] = T(g.s[d] * tab->D[r / N][r % N]);
  }
  for (int q = threadIdx.x; q < N3; q += blockDim.x) {
    const int i = q % N, j = (q / N) % N, l = q / (N * N);
    s.W3[q] = T(tab->w[i] * tab->w[j] * tab->w[l] * g.detJ);
    if (need_psi)
      for (int m = 0; m < NP; ++m)
        s.Psi[q][m] = T(tab->pw[i][tab->ex[m][0]] * tab->pw[j][tab->ex[m][1]] * tab->pw[l][tab->ex[m][2]]);
  }
}

// ------------------------------------------------------------------ Stokes family

template <typename T, int N, int OPS>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_stokes(Grid g, const RefTables* __restrict__ tab, int colour, int count, const T* __restrict__ u,
         const T* __restrict__ us, const T* __restrict__ p, const T* __restrict__ coef, int coef_nodal,
         T* __restrict__ yu, T* __restrict__ yp) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP, EPB = Cfg<N>::EPB, K = N - 1;
  constexpr bool DA = OPS & OP_A, DBT = OPS & OP_BT, DB = OPS & OP_B;
  constexpr bool SCAT = DA || DBT, GRAD = DA || DB;
  constexpr int NS = DA ? 6 : 1;      // stored stress components (B^T alone needs only -W p)
  __shared__ OpTab<T, N> st;
  __shared__ T su[GRAD ? EPB : 1][3][N3];
  __shared__ T sS[SCAT ? EPB : 1][NS][N3];
  __shared__ T sdiv[DB ? EPB : 1][N3];
  load_optab(st, tab, g, DB || DBT);

  const int tid = threadIdx.x;
  const int le = tid / N3, q = tid - le * N3;
  const int i = q % N, j = (q / N) % N, l = q / (N * N);
  const int eidx = blockIdx.x * EPB + le;
  const bool act = eidx < count;
  int e = 0, node = 0;
  bool interior = false;
  if (act) {
    int ex, ey, ez;
    colour_element(g, colour, eidx, ex, ey, ez);
    e = ex + g.nx * (ey + g.ny * ez);
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
  __syncthreads();   // tables and tile loaded
  if (act && DBT) {
#pragma unroll
    for (int m = 0; m < NP; ++m) pq += st.Psi[q][m] * p[(size_t)e * NP + m];
  }
  if (act) {
    const T Wq = st.W3[q];
    if (DA) {
      T G[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int a = 0; a < N; ++a) {
          a0 += st.Ds[0][i][a] * su[GRAD ? le : 0][c][a + N * (j + N * l)];
          a1 += st.Ds[1][j][a] * su[GRAD ? le : 0][c][i + N * (a + N * l)];
          a2 += st.Ds[2][l][a] * su[GRAD ? le : 0][c][i + N * (j + N * a)];
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
        // divergence only: the three diagonal derivatives
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
  if (!act) return;
  if (DB && q < NP) {
    const int m = q;
    T acc = 0;
#pragma unroll
    for (int qq = 0; qq < N3; ++qq) acc += st.Psi[qq][m] * sdiv[DB ? le : 0][qq];
    yp[(size_t)e * NP + m] = -acc;
  }
  if (SCAT && interior) {
    const T* S = &sS[SCAT ? le : 0][0][0];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T acc = 0;
      if (DA) {
        const int i0 = sym_index(c, 0), i1 = sym_index(c, 1), i2 = sym_index(c, 2);
#pragma unroll
        for (int a = 0; a < N; ++a) {
          acc += st.Ds[0][a][i] * S[i0 * N3 + a + N * (j + N * l)];
          acc += st.Ds[1][a][j] * S[i1 * N3 + i + N * (a + N * l)];
          acc += st.Ds[2][a][l] * S[i2 * N3 + i + N * (j + N * a)];
        }
      } else {
        // B^T alone: y_c = sum_a Ds[c][a][q_c] (-W p)(q with axis c -> a)
#pragma unroll
        for (int a = 0; a < N; ++a) {
          const int qa = c == 0 ? a + N * (j + N * l) : (c == 1 ? i + N * (a + N * l) : i + N * (j + N * a));
          const int qc = c == 0 ? i : (c == 1 ? j : l);
          acc += st.Ds[c][a][qc] * S[qa];
        }
      }
      yu[(size_t)c * g.nn + node] += acc;
    }
  }
}

template <typename T, int N, int OPS>
cudaError_t run_stokes(const Grid& g, const RefTables* tab, const T* u, const T* us, const T* p, const T* coef,
                       int coef_nodal, T* yu, T* yp, cudaStream_t st) {
  constexpr int EPB = Cfg<N>::EPB, TH = Cfg<N>::THREADS;
  constexpr bool SCAT = (OPS & OP_A) || (OPS & OP_BT);
  if (SCAT) {
    cudaError_t e = cudaMemsetAsync(yu, 0, sizeof(T) * 3 * (size_t)g.nn, st);
    if (e != cudaSuccess) return e;
    for (int c = 0; c < 8; ++c) {
      int cnt = colour_count(g, c);
      if (cnt == 0) continue;
      wb_launch(k_stokes<T, N, OPS>, (cnt + EPB - 1) / EPB, TH, 0, st, g, tab, c, cnt, u, us, p, coef, coef_nodal, yu, yp);
    }
  } else {
    wb_launch(k_stokes<T, N, OPS>, (g.ne + EPB - 1) / EPB, TH, 0, st, g, tab, -1, g.ne, u, us, p, coef, coef_nodal, yu, yp);
  }
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t dispatch_ops(const Grid& g, const RefTables* tab, int ops, const T* u, const T* us, const T* p,
                         const T* coef, int cn, T* yu, T* yp, cudaStream_t st) {
  switch (ops) {
    case OP_A: return run_stokes<T, N, OP_A>(g, tab, u, us, p, coef, cn, yu, yp, st);
    case OP_BT: return run_stokes<T, N, OP_BT>(g, tab, u, us, p, coef, cn, yu, yp, st);
    case OP_B: return run_stokes<T, N, OP_B>(g, tab, u, us, p, coef, cn, yu, yp, st);
    case OP_A | OP_BT | OP_B: return run_stokes<T, N, OP_A | OP_BT | OP_B>(g, tab, u, us, p, coef, cn, yu, yp, st);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------------ scalar Poisson

template <typename T, int N>
__global__ void __launch_bounds__(Cfg<N>::THREADS)
k_poisson(Grid g, const RefTables* __restrict__ tab, int colour, int count, const T* __restrict__ u,
          const T* __restrict__ coef, T* __restrict__ y) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, EPB = Cfg<N>::EPB, K = N - 1;
  __shared__ OpTab<T, N> st;
  __shared__ T su[EPB][N3];
  __shared__ T sF[EPB][3][N3];
  load_optab(st, tab, g, false);
  const int tid = threadIdx.x;
  const int le = tid / N3, q = tid - le * N3;
  const int i = q % N, j = (q / N) % N, l = q / (N * N);
  const int eidx = blockIdx.x * EPB + le;
  const bool act = eidx < count;
  int e = 0, node = 0;
  if (act) {
    int ex, ey, ez;
    colour_element(g, colour, eidx, ex, ey, ez);
    e = ex + g.nx * (ey + g.ny * ez);
    node = (K * ex + i) + g.NX * ((K * ey + j) + g.NY * (K * ez + l));
    su[le][q] = u[node];
  }
  __syncthreads();
  if (act) {
    T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
    for (int a = 0; a < N; ++a) {
      a0 += st.Ds[0][i][a] * su[le][a + N * (j + N * l)];
      a1 += st.Ds[1][j][a] * su[le][i + N * (a + N * l)];
      a2 += st.Ds[2][l][a] * su[le][i + N * (j + N * a)];
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
    acc += st.Ds[0][a][i] * sF[le][0][a + N * (j + N * l)];
    acc += st.Ds[1][a][j] * sF[le][1][i + N * (a + N * l)];
    acc += st.Ds[2][a][l] * sF[le][2][i + N * (j + N * a)];
  }
  y[node] += acc;
}

template <typename T, int N>
cudaError_t run_poisson(const Grid& g, const RefTables* tab, const T* u, const T* coef, T* y, cudaStream_t st) {
  constexpr int EPB = Cfg<N>::EPB, TH = Cfg<N>::THREADS;
  cudaError_t e = cudaMemsetAsync(y, 0, sizeof(T) * (size_t)g.nn, st);
  if (e != cudaSuccess) return e;
  for (int c = 0; c < 8; ++c) {
    int cnt = colour_count(g, c);
    if (cnt == 0) continue;
    wb_launch(k_poisson<T, N>, (cnt + EPB - 1) / EPB, TH, 0, st, g, tab, c, cnt, u, coef, y);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ dense coarsest assembly (FP64)

// One block per (element of a colour, local input DOF): the element operator applied to a unit
// vector gives one column of the element matrix, added into the dense matrix.
template <int N, bool VEC>
__global__ void __launch_bounds__(Cfg<N>::N3)
k_dense_assemble(Grid g, const RefTables* __restrict__ tab, int colour, const double* __restrict__ coef,
                 int coef_nodal, const int* __restrict__ map, int nfree, double* __restrict__ M, int ld) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, K = N - 1, NC = VEC ? 3 : 1, NS = VEC ? 6 : 3;
  __shared__ SmTab<double, N> st;
  __shared__ double su[NC][N3];
  __shared__ double sS[NS][N3];
  load_tab(st, tab);
  const int q = threadIdx.x;
  const int i = q % N, j = (q / N) % N, l = q / (N * N);
  int ex, ey, ez;
  colour_element(g, colour, blockIdx.x, ex, ey, ez);
  const int e = ex + g.nx * (ey + g.ny * ez);
  const int col = blockIdx.y, cin = col / N3, qin = col % N3;
  auto node_of = [&](int qq) {
    int ii = qq % N, jj = (qq / N) % N, ll = qq / (N * N);
    return (K * ex + ii) + g.NX * ((K * ey + jj) + g.NY * (K * ez + ll));
  };
  const int nin = node_of(qin);
  if (map[nin] < 0) return;  // eliminated (Dirichlet) input: zero column, uniform per block
  const int node = node_of(q);
  for (int c = 0; c < NC; ++c) su[c][q] = (c == cin && q == qin) ? 1.0 : 0.0;
  __syncthreads();
  const double* s = g.s;
  const double Wq = st.w[i] * st.w[j] * st.w[l] * g.detJ;
  const double cq = coef_nodal ? coef[node] : coef[(size_t)e * N3 + q];
  double G[NC][3];
  for (int c = 0; c < NC; ++c) {
    double a0 = 0, a1 = 0, a2 = 0;
    for (int a = 0; a < N; ++a) {
      a0 += st.D[i][a] * su[c][a + N * (j + N * l)];
      a1 += st.D[j][a] * su[c][i + N * (a + N * l)];
      a2 += st.D[l][a] * su[c][i + N * (j + N * a)];
    }
    G[c][0] = s[0] * a0;
    G[c][1] = s[1] * a1;
    G[c][2] = s[2] * a2;
  }
  if constexpr (VEC) {
    const double f = Wq * 2.0 * cq;
    sS[0][q] = f * G[0][0];
    sS[1][q] = f * G[1][1];
    sS[2][q] = f * G[2][2];
    sS[3][q] = f * 0.5 * (G[0][1] + G[1][0]);
    sS[4][q] = f * 0.5 * (G[0][2] + G[2][0]);
    sS[5][q] = f * 0.5 * (G[1][2] + G[2][1]);
  } else {
    for (int d = 0; d < 3; ++d) sS[d][q] = Wq * cq * G[0][d];
  }
  __syncthreads();
  if (map[node] < 0) return;
  const int cg = VEC ? cin * nfree + map[nin] : map[nin];
  for (int c = 0; c < NC; ++c) {
    const int i0 = VEC ? sym_index(c, 0) : 0, i1 = VEC ? sym_index(c, 1) : 1, i2 = VEC ? sym_index(c, 2) : 2;
    double a0 = 0, a1 = 0, a2 = 0;
    for (int a = 0; a < N; ++a) {
      a0 += st.D[a][i] * sS[i0][a + N * (j + N * l)];
      a1 += st.D[a][j] * sS[i1][i + N * (a + N * l)];
      a2 += st.D[a][l] * sS[i2][i + N * (j + N * a)];
    }
    const int rg = VEC ? c * nfree + map[node] : map[node];
    M[(size_t)rg * ld + cg] += s[0] * a0 + s[1] * a1 + s[2] * a2;
  }
}

// ------------------------------------------------------------------ node-centric helpers

template <typename T, int N, bool VEC>
__global__ void k_dinv_stiff(Grid g, const RefTables* __restrict__ tab, const T* __restrict__ coef, int coef_nodal,
                             T* __restrict__ dinv) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, K = N - 1;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int ix = n % g.NX, iy = (n / g.NX) % g.NY, iz = n / (g.NX * g.NY);
  const bool bnd = on_boundary(g, ix, iy, iz);
  double acc[3] = {0, 0, 0};   // per axis d: sum_e sum_i W |J| c (2/h_d)^2 D[i][a_d]^2
  for_elements_of_node(g, K, ix, iy, iz, [&](int e, int ex, int ey, int ez, int a0, int a1, int a2) {
    const int a[3] = {a0, a1, a2};
    for (int d = 0; d < 3; ++d) {
      const double sd = g.s[d];
      for (int ii = 0; ii < N; ++ii) {
        int qq[3] = {a0, a1, a2};
        qq[d] = ii;
        const int q = qq[0] + N * (qq[1] + N * qq[2]);
        double cq;
        if (coef_nodal) {
          const int nd = (K * ex + qq[0]) + g.NX * ((K * ey + qq[1]) + g.NY * (K * ez + qq[2]));
          cq = (double)coef[nd];
        } else {
          cq = (double)coef[(size_t)e * N3 + q];
        }
        const double Wq = tab->w[qq[0]] * tab->w[qq[1]] * tab->w[qq[2]] * g.detJ;
        const double Dv = tab->D[ii][a[d]] * sd;
        acc[d] += Wq * cq * Dv * Dv;
      }
    }
  });
  if (VEC) {
    // A: sum_q W|J| mu (|grad phi|^2 + (d_c phi)^2), the 2 mu eps:eps diagonal
    const double tot = acc[0] + acc[1] + acc[2];
    for (int c = 0; c < 3; ++c) dinv[(size_t)c * g.nn + n] = bnd ? T(0) : T(1.0 / (tot + acc[c]));
  } else {
    dinv[n] = T(1.0 / (acc[0] + acc[1] + acc[2]));
  }
}

// diag(B C^-1 B^T) per (element, mode): sum over element velocity DOFs of B_e[m][(c,a)]^2 cinv(a).
template <typename T, int N>
__global__ void k_dinv_Kw(Grid g, const RefTables* __restrict__ tab, const T* __restrict__ cinv, int per_dof,
                          T* __restrict__ dinv) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP, K = N - 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.ne * NP) return;
  const int e = t / NP, m = t % NP;
  const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
  double acc = 0.0;
  for (int q = 0; q < N3; ++q) {
    const int a[3] = {q % N, (q / N) % N, q / (N * N)};
    const int node = (K * ex + a[0]) + g.NX * ((K * ey + a[1]) + g.NY * (K * ez + a[2]));
    for (int c = 0; c < 3; ++c) {
      const double ci = (double)cinv[(per_dof ? (size_t)c * g.nn : 0) + node];
      if (ci == 0.0) continue;
      double b = 0.0;
      for (int ii = 0; ii < N; ++ii) {
        int qq[3] = {a[0], a[1], a[2]};
        qq[c] = ii;
        const double Wq = tab->w[qq[0]] * tab->w[qq[1]] * tab->w[qq[2]];
        const double ps = tab->pw[qq[0]][tab->ex[m][0]] * tab->pw[qq[1]][tab->ex[m][1]] * tab->pw[qq[2]][tab->ex[m][2]];
        b += Wq * ps * tab->D[ii][a[c]];
      }
      b *= -g.s[c] * g.detJ;
      acc += b * b * ci;
    }
  }
  dinv[t] = acc > 0.0 ? T(1.0 / acc) : T(0);   // a zero diagonal (single-element mesh, constant mode) is skipped
}

// C(n) = sum_{e containing n} a(e) W_q |J| sqrt(mu(n))  (mu == nullptr: the plain lumped mass)
__global__ void k_lumped(Grid g, int K, const RefTables* __restrict__ tab, const double* __restrict__ mu, double amp,
                         double* __restrict__ out) {
  pdl_entry();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int ix = n % g.NX, iy = (n / g.NX) % g.NY, iz = n / (g.NX * g.NY);
  double acc = 0.0;
  for_elements_of_node(g, K, ix, iy, iz, [&](int, int ex, int ey, int ez, int a0, int a1, int a2) {
    const bool bnd_el = ex == 0 || ey == 0 || ez == 0 || ex == g.nx - 1 || ey == g.ny - 1 || ez == g.nz - 1;
    acc += (bnd_el ? amp : 1.0) * tab->w[a0] * tab->w[a1] * tab->w[a2] * g.detJ;
  });
  out[n] = mu ? acc * sqrt(mu[n]) : acc;
}

// p-coarsening of a per-point coefficient from Q_k (N = k + 1 points per axis) to Q1 on the same
// element: the normalised L^2-adjoint of element-wise trilinear interpolation, per axis
// T[v][a] = W_a l1_v(x_a) / sum_a' W_a' l1_v(x_a'), l1_0 = (1 - x)/2, l1_1 = (1 + x)/2 on the
// Q_k GLL points x_a with weights W_a; c1(v) = sum_{a,b,c} T[v0][a] T[v1][b] T[v2][c] c(a, b, c).
// Non-negative weights, constants preserved (Sec. 6, as the h-coarsening of the coefficient).
template <int N>
__global__ void k_pcoarsen_coef(Grid g, const RefTables* __restrict__ tab, const double* __restrict__ cf,
                                double* __restrict__ cc) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.ne * 8) return;
  const int e = (int)(t >> 3), v = (int)(t & 7);
  const int vi[3] = {v & 1, (v >> 1) & 1, v >> 2};
  double T[3][N];
  for (int d = 0; d < 3; ++d) {
    double den = 0.0;
    for (int a = 0; a < N; ++a) {
      const double l1 = vi[d] ? 0.5 * (1.0 + tab->x[a]) : 0.5 * (1.0 - tab->x[a]);
      T[d][a] = tab->w[a] * l1;
      den += T[d][a];
    }
    for (int a = 0; a < N; ++a) T[d][a] /= den;
  }
  const double* ce = cf + (size_t)e * N3;
  double acc = 0.0;
  for (int c = 0; c < N; ++c)
    for (int b = 0; b < N; ++b)
      for (int a = 0; a < N; ++a) acc += T[0][a] * T[1][b] * T[2][c] * ce[a + N * (b + N * c)];
  cc[t] = acc;
}

// p-transfers between Q1 on grid g1 (vertices, (n+1)^3 per axis counts) and Q_k on the same
// mesh (node grid k n + 1 per axis), for k >= 3 (at k = 2 the Q_k node grid is that of Q1 on the
// refined mesh, and the nested h-transfer kernels serve).  Per axis the Q1 vertex function v takes
// the value (1 + x_a)/2 at local GLL node a of element v - 1 and (1 - x_a)/2 at node a of element v.
__device__ inline double p_weight(int i, int v, int k, const double* x) {
  if (i < k * v) {
    const int a = i - k * (v - 1);
    return (a >= 0 && a <= k) ? 0.5 * (1.0 + x[a]) : 0.0;
  }
  const int a = i - k * v;
  return a <= k ? 0.5 * (1.0 - x[a]) : 0.0;
}

// out_f (+)= P in_c: one thread per Q_k node, the 2 x 2 x 2 vertices of its element
template <typename T>
__global__ void k_p_prolong(Grid g1, int k, const RefTables* __restrict__ tab, int ncomp, const T* __restrict__ in_c,
                            T* __restrict__ out_f, int add) {
  pdl_entry();
  const int NXf = k * g1.nx + 1, NYf = k * g1.ny + 1, NZf = k * g1.nz + 1;
  const long long nnf = (long long)NXf * NYf * NZf;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnf) return;
  const int ix = (int)(t % NXf), iy = (int)((t / NXf) % NYf), iz = (int)(t / ((long long)NXf * NYf));
  const int ex = min(ix / k, g1.nx - 1), ey = min(iy / k, g1.ny - 1), ez = min(iz / k, g1.nz - 1);
  double wx[2], wy[2], wz[2];
  for (int s = 0; s < 2; ++s) {
    wx[s] = p_weight(ix, ex + s, k, tab->x);
    wy[s] = p_weight(iy, ey + s, k, tab->x);
    wz[s] = p_weight(iz, ez + s, k, tab->x);
  }
  for (int c = 0; c < ncomp; ++c) {
    double acc = 0.0;
    for (int sz = 0; sz < 2; ++sz)
      for (int sy = 0; sy < 2; ++sy)
        for (int sx = 0; sx < 2; ++sx)
          acc += wx[sx] * wy[sy] * wz[sz] *
                 (double)in_c[(size_t)c * g1.nn + (ex + sx) + g1.NX * ((ey + sy) + (size_t)g1.NY * (ez + sz))];
    T* o = out_f + (size_t)c * nnf + t;
    *o = add ? *o + T(acc) : T(acc);
  }
}

// out_c = P^T in_f: one thread per Q1 vertex, the Q_k nodes of the up to 2 x 2 x 2 elements around
// it; Dirichlet vertices zeroed when mask_dirichlet
template <typename T>
__global__ void k_p_restrict(Grid g1, int k, const RefTables* __restrict__ tab, int ncomp, const T* __restrict__ in_f,
                             T* __restrict__ out_c, int mask_dirichlet) {
  pdl_entry();
  const int NXf = k * g1.nx + 1, NYf = k * g1.ny + 1, NZf = k * g1.nz + 1;
  const long long nnf = (long long)NXf * NYf * NZf;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g1.nn) return;
  const int vx = t % g1.NX, vy = (t / g1.NX) % g1.NY, vz = t / (g1.NX * g1.NY);
  const bool bnd = mask_dirichlet && on_boundary(g1, vx, vy, vz);
  const int x0 = max(0, k * (vx - 1)), x1 = min(NXf - 1, k * (vx + 1));
  const int y0 = max(0, k * (vy - 1)), y1 = min(NYf - 1, k * (vy + 1));
  const int z0 = max(0, k * (vz - 1)), z1 = min(NZf - 1, k * (vz + 1));
  for (int c = 0; c < ncomp; ++c) {
    double acc = 0.0;
    if (!bnd)
      for (int iz = z0; iz <= z1; ++iz) {
        const double wz = p_weight(iz, vz, k, tab->x);
        for (int iy = y0; iy <= y1; ++iy) {
          const double wy = wz * p_weight(iy, vy, k, tab->x);
          const T* row = in_f + (size_t)c * nnf + (size_t)NXf * (iy + (size_t)NYf * iz);
          for (int ix = x0; ix <= x1; ++ix) acc += wy * p_weight(ix, vx, k, tab->x) * (double)row[ix];
        }
      }
    out_c[(size_t)c * g1.nn + t] = T(acc);
  }
}

// The w-BFBT weight at every element point (FP64, [ne][N^3]): sqrt(mu) (grad = 0, Eq. wbfbt) or
// (mu^2 + |grad mu_h|^2)^(1/4) (grad = 1, the viscosity-gradient weights of the remark in
// Sec. 4), grad mu_h being the gradient of the element's Q_k interpolant of the nodal viscosity.
template <int N>
__global__ void k_weight_points(Grid g, const RefTables* __restrict__ tab, const double* __restrict__ mu, int grad,
                                double* __restrict__ w) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, K = N - 1;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.ne * N3) return;
  const int e = (int)(t / N3), q = (int)(t % N3);
  const int i = q % N, j = (q / N) % N, l = q / (N * N);
  const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
  const long long base = (long long)K * ex + (long long)g.NX * (K * ey + (long long)g.NY * K * ez);
  auto at = [&](int a, int b, int c) { return mu[base + a + (long long)g.NX * (b + (long long)g.NY * c)]; };
  const double m0 = at(i, j, l);
  if (!grad) {
    w[t] = sqrt(m0);
    return;
  }
  double gx = 0.0, gy = 0.0, gz = 0.0;
  for (int a = 0; a < N; ++a) {
    gx += tab->D[i][a] * at(a, j, l);
    gy += tab->D[j][a] * at(i, a, l);
    gz += tab->D[l][a] * at(i, j, a);
  }
  gx *= g.s[0];
  gy *= g.s[1];
  gz *= g.s[2];
  w[t] = sqrt(sqrt(m0 * m0 + gx * gx + gy * gy + gz * gz));
}

// M~_u(a w) per node from the point weights: sum over the elements at the node of a(e) W_q |J| w_e(q).
template <int N>
__global__ void k_lumped_pts(Grid g, const RefTables* __restrict__ tab, const double* __restrict__ wp, double amp,
                             double* __restrict__ out) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, K = N - 1;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int ix = n % g.NX, iy = (n / g.NX) % g.NY, iz = n / (g.NX * g.NY);
  double acc = 0.0;
  for_elements_of_node(g, K, ix, iy, iz, [&](int e, int ex, int ey, int ez, int a0, int a1, int a2) {
    const bool bnd_el = ex == 0 || ey == 0 || ez == 0 || ex == g.nx - 1 || ey == g.ny - 1 || ez == g.nz - 1;
    acc += (bnd_el ? amp : 1.0) * tab->w[a0] * tab->w[a1] * tab->w[a2] * g.detJ *
           wp[(size_t)e * N3 + a0 + N * (a1 + N * a2)];
  });
  out[n] = acc;
}

// Poisson coefficient c = 1 / (a(e) w) per element point from the point weights.
template <typename T, int N>
__global__ void k_poisson_coef_pts(Grid g, const double* __restrict__ wp, double amp, T* __restrict__ c) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.ne * N3) return;
  const int e = (int)(t / N3);
  const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
  const bool bnd_el = ex == 0 || ey == 0 || ez == 0 || ex == g.nx - 1 || ey == g.ny - 1 || ez == g.nz - 1;
  c[t] = T(1.0 / ((bnd_el ? amp : 1.0) * wp[t]));
}

// r_c(n) = sum_{e containing n} W_q sum_m psi_m(q) sum_m' minv[m][m'] r_d[e][m']   (|J| cancels)
template <typename T, int N>
__global__ void k_disc_to_cont(Grid g, const RefTables* __restrict__ tab, const T* __restrict__ rd, T* __restrict__ rc) {
  pdl_entry();
  constexpr int NP = Cfg<N>::NP, K = N - 1;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int ix = n % g.NX, iy = (n / g.NX) % g.NY, iz = n / (g.NX * g.NY);
  double acc = 0.0;
  for_elements_of_node(g, K, ix, iy, iz, [&](int e, int, int, int, int a0, int a1, int a2) {
    double v[NP];
    for (int m = 0; m < NP; ++m) v[m] = (double)rd[(size_t)e * NP + m];
    double s = 0.0;
    for (int m = 0; m < NP; ++m) {
      double mv = 0.0;
      for (int mp = 0; mp < NP; ++mp) mv += tab->minv[m][mp] * v[mp];
      s += tab->pw[a0][tab->ex[m][0]] * tab->pw[a1][tab->ex[m][1]] * tab->pw[a2][tab->ex[m][2]] * mv;
    }
    acc += tab->w[a0] * tab->w[a1] * tab->w[a2] * s;
  });
  rc[n] = T(acc);
}

// e_d[e][m] (+)= sum_m' minv[m][m'] sum_q W_q psi_m'(q) e_c(node(e, q))   (|J| cancels)
template <typename T, int N>
__global__ void k_cont_to_disc(Grid g, const RefTables* __restrict__ tab, const T* __restrict__ ec, T* __restrict__ ed,
                               int add) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, NP = Cfg<N>::NP, K = N - 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.ne) return;
  const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
  double gm[NP];
  for (int m = 0; m < NP; ++m) gm[m] = 0.0;
  for (int q = 0; q < N3; ++q) {
    const int a0 = q % N, a1 = (q / N) % N, a2 = q / (N * N);
    const int node = (K * ex + a0) + g.NX * ((K * ey + a1) + g.NY * (K * ez + a2));
    const double v = tab->w[a0] * tab->w[a1] * tab->w[a2] * (double)ec[node];
    for (int m = 0; m < NP; ++m)
      gm[m] += tab->pw[a0][tab->ex[m][0]] * tab->pw[a1][tab->ex[m][1]] * tab->pw[a2][tab->ex[m][2]] * v;
  }
  for (int m = 0; m < NP; ++m) {
    double s = 0.0;
    for (int mp = 0; mp < NP; ++mp) s += tab->minv[m][mp] * gm[mp];
    ed[(size_t)e * NP + m] = add ? T((double)ed[(size_t)e * NP + m] + s) : T(s);
  }
}

template <typename T, int N>
__global__ void k_poisson_coef0(Grid g, const double* __restrict__ mu, double amp, int pointwise_mu_only,
                                T* __restrict__ c) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3, K = N - 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.ne * N3) return;
  const int e = t / N3, q = t % N3;
  const int ex = e % g.nx, ey = (e / g.nx) % g.ny, ez = e / (g.nx * g.ny);
  const int node = (K * ex + q % N) + g.NX * ((K * ey + (q / N) % N) + g.NY * (K * ez + q / (N * N)));
  if (pointwise_mu_only) {
    c[t] = T(mu[node]);
    return;
  }
  const bool bnd_el = ex == 0 || ey == 0 || ez == 0 || ex == g.nx - 1 || ey == g.ny - 1 || ez == g.nz - 1;
  c[t] = T(1.0 / ((bnd_el ? amp : 1.0) * sqrt(mu[node])));
}

// c_E(q) = sum_{children s} sum_{q'} Tc[sz][l][l'] Tc[sy][j][j'] Tc[sx][i][i'] c_e(q')
template <typename T, int N>
__global__ void k_coarsen_coef(Grid gf, const RefTables* __restrict__ tab, const T* __restrict__ cf, T* __restrict__ cc) {
  pdl_entry();
  constexpr int N3 = Cfg<N>::N3;
  const int ncx = gf.nx / 2, ncy = gf.ny / 2, ncz = gf.nz / 2;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncx * ncy * ncz * N3) return;
  const int E = t / N3, q = t % N3;
  const int i = q % N, j = (q / N) % N, l = q / (N * N);
  const int X = E % ncx, Y = (E / ncx) % ncy, Z = E / (ncx * ncy);
  double acc = 0.0;
  for (int sz = 0; sz < 2; ++sz)
    for (int sy = 0; sy < 2; ++sy)
      for (int sx = 0; sx < 2; ++sx) {
        const int e = (2 * X + sx) + gf.nx * ((2 * Y + sy) + gf.ny * (2 * Z + sz));
        const T* c = cf + (size_t)e * N3;
        for (int lp = 0; lp < N; ++lp) {
          const double wz = tab->Tc[sz][l][lp];
          if (wz == 0.0) continue;
          for (int jp = 0; jp < N; ++jp) {
            const double wy = tab->Tc[sy][j][jp];
            if (wy == 0.0) continue;
            for (int ip = 0; ip < N; ++ip) acc += wz * wy * tab->Tc[sx][i][ip] * (double)c[ip + N * (jp + N * lp)];
          }
        }
      }
  cc[t] = T(acc);
}

// ------------------------------------------------------------------ nested transfers (1-D passes)

// One axis of P (prolong) or P^T (restrict) on an array with fast-to-slow extents d[0..2].
template <typename T>
__global__ void k_pass(const RefTables* __restrict__ tab, int K, int axis, int d0, int d1, int d2, int nc_el, int prolong,
                       const T* __restrict__ in, T* __restrict__ out, int add) {
  pdl_entry();
  // output extents: the axis extent becomes the fine (prolong) or coarse (restrict) count
  const int nfine = 2 * K * nc_el + 1, ncoarse = K * nc_el + 1;
  int od[3] = {d0, d1, d2};
  od[axis] = prolong ? nfine : ncoarse;
  const long long tot = (long long)od[0] * od[1] * od[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= tot) return;
  int o[3];
  o[0] = (int)(t % od[0]);
  o[1] = (int)((t / od[0]) % od[1]);
  o[2] = (int)(t / ((long long)od[0] * od[1]));
  const int id[3] = {d0, d1, d2};
  auto in_index = [&](int r) {
    int c[3] = {o[0], o[1], o[2]};
    c[axis] = r;
    return (long long)c[0] + (long long)id[0] * (c[1] + (long long)id[1] * c[2]);
  };
  const int nf_el = 2 * nc_el;
  double acc = 0.0;
  if (prolong) {
    const int i_f = o[axis];
    int ef = i_f / K;
    if (ef > nf_el - 1) ef = nf_el - 1;
    const int a = i_f - K * ef, ec = ef / 2, s = ef % 2;
    for (int b = 0; b <= K; ++b) acc += tab->P1[s][a][b] * (double)in[in_index(K * ec + b)];
  } else {
    const int i_c = o[axis];
    int lo = 2 * i_c - 2 * K, hi = 2 * i_c + 2 * K;
    if (lo < 0) lo = 0;
    if (hi > nfine - 1) hi = nfine - 1;
    for (int i_f = lo; i_f <= hi; ++i_f) {
      int ef = i_f / K;
      if (ef > nf_el - 1) ef = nf_el - 1;
      const int a = i_f - K * ef, ec = ef / 2, s = ef % 2;
      const int b = i_c - K * ec;
      if (b < 0 || b > K) continue;
      acc += tab->P1[s][a][b] * (double)in[in_index(i_f)];
    }
  }
  out[t] = add ? T((double)out[t] + acc) : T(acc);
}

template <typename T>
__global__ void k_mask_boundary(Grid g, int ncomp, T* __restrict__ v) {
  pdl_entry();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int ix = n % g.NX, iy = (n / g.NX) % g.NY, iz = n / (g.NX * g.NY);
  if (on_boundary(g, ix, iy, iz))
    for (int c = 0; c < ncomp; ++c) v[(size_t)c * g.nn + n] = T(0);
}

// ------------------------------------------------------------------ sinker setup (Sec. 2.1)

struct Centres {
  double c[128][3];
  double x[WB_MAXN];   // GLL nodes
};

// Brick coordinate of node index idx along axis d: element e = idx / K (the last node belongs to the
// last element), local GLL node a = idx - K e.
__device__ inline double brick_coord(const Grid& g, int K, const Centres& cs, int d, int idx) {
  const int ne[3] = {g.nx, g.ny, g.nz};
  int e = idx / K;
  if (e > ne[d] - 1) e = ne[d] - 1;
  const int a = idx - K * e;
  return e * g.h[d] + (cs.x[a] + 1.0) * 0.5 * g.h[d];
}

// mu and f_z of Sec. 2.1 at point x: chi = prod_s (1 - exp(-delta max(0, |x - c_s| - omega/2)^2)),
// mu = (mu_max - mu_min)(1 - chi) + mu_min with mu_max/min = dr^(+-1/2), f = (0, 0, beta (chi - 1)).
__device__ inline void sinker_point(const double (&x)[3], const Centres& cs, int ns, double omega, double delta,
                                    double dr, double beta, double& mu, double& fz) {
  double chi = 1.0;
  for (int s = 0; s < ns; ++s) {
    const double dx = x[0] - cs.c[s][0], dy = x[1] - cs.c[s][1], dz = x[2] - cs.c[s][2];
    double r = sqrt(dx * dx + dy * dy + dz * dz) - 0.5 * omega;
    r = r > 0.0 ? r : 0.0;
    // for delta r^2 > 40, exp(-delta r^2) < 2^-54 and 1 - exp(...) rounds to exactly 1 in FP64:
    // skipping the factor leaves chi bitwise unchanged
    const double t = delta * r * r;
    if (t > 40.0) continue;
    chi *= 1.0 - exp(-t);
  }
  const double mu_min = 1.0 / sqrt(dr), mu_max = sqrt(dr);
  mu = (mu_max - mu_min) * (1.0 - chi) + mu_min;
  fz = beta * (chi - 1.0);
}

// X: given nodal coordinates [3][nn] (the mapped form), or null for the brick's GLL nodes.
__global__ void k_sinker(Grid g, int K, Centres cs, const double* __restrict__ X, int ns, double omega,
                         double delta, double dr, double beta, double* __restrict__ mu, double* __restrict__ f) {
  pdl_entry();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int idx[3] = {n % g.NX, (n / g.NX) % g.NY, n / (g.NX * g.NY)};
  double x[3];
  for (int d = 0; d < 3; ++d) x[d] = X ? X[(size_t)d * g.nn + n] : brick_coord(g, K, cs, d, idx[d]);
  double m, fz;
  sinker_point(x, cs, ns, omega, delta, dr, beta, m, fz);
  mu[n] = m;
  if (f) {
    f[n] = 0.0;
    f[(size_t)g.nn + n] = 0.0;
    f[2 * (size_t)g.nn + n] = fz;
  }
}

// The brick's nodal coordinates [3][nn].
__global__ void k_node_coords(Grid g, int K, Centres cs, double* __restrict__ X) {
  pdl_entry();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int idx[3] = {n % g.NX, (n / g.NX) % g.NY, n / (g.NX * g.NY)};
  for (int d = 0; d < 3; ++d) X[(size_t)d * g.nn + n] = brick_coord(g, K, cs, d, idx[d]);
}

inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

// ================================================================== launchers

#define WB_DISPATCH_N(k, CALL) \
  switch (k) {                 \
    case 1: { constexpr int N = 2; return CALL; } \
    case 2: { constexpr int N = 3; return CALL; } \
    case 3: { constexpr int N = 4; return CALL; } \
    case 4: { constexpr int N = 5; return CALL; } \
    default: return cudaErrorInvalidValue; \
  }

template <typename T>
cudaError_t launch_stokes(const Grid& g, int k, const RefTables* dtab, int ops, const T* u, const T* us, const T* p,
                          const T* coef, int cn, T* yu, T* yp, cudaStream_t st) {
  WB_DISPATCH_N(k, (dispatch_ops<T, N>(g, dtab, ops, u, us, p, coef, cn, yu, yp, st)));
}

template <typename T>
cudaError_t launch_poisson(const Grid& g, int k, const RefTables* dtab, const T* u, const T* coef, T* y,
                           cudaStream_t st) {
  WB_DISPATCH_N(k, (run_poisson<T, N>(g, dtab, u, coef, y, st)));
}

namespace {
template <int N, bool VEC>
cudaError_t run_dense(const Grid& g, const RefTables* tab, const double* coef, int cn, const int* map, int nfree,
                      double* M, int ld, cudaStream_t st) {
  constexpr int N3 = Cfg<N>::N3;
  for (int c = 0; c < 8; ++c) {
    int cnt = colour_count(g, c);
    if (cnt == 0) continue;
    dim3 grid(cnt, (VEC ? 3 : 1) * N3);
    wb_launch(k_dense_assemble<N, VEC>, grid, N3, 0, st, g, tab, c, coef, cn, map, nfree, M, ld);
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_assemble_dense_A(const Grid& g, int k, const RefTables* dtab, const double* coef, int cn,
                                    const int* map, int nfree, double* M, int ld, cudaStream_t st) {
  WB_DISPATCH_N(k, (run_dense<N, true>(g, dtab, coef, cn, map, nfree, M, ld, st)));
}

namespace {
__global__ void k_iota(int n, int* m) {
  pdl_entry();
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) m[t] = t;
}
}  // namespace

cudaError_t launch_assemble_dense_L_mapped(const Grid& g, int k, const RefTables* dtab, const double* coef,
                                           const int* map, double* M, int ld, cudaStream_t st) {
  WB_DISPATCH_N(k, (run_dense<N, false>(g, dtab, coef, 0, map, g.nn, M, ld, st)));
}

cudaError_t launch_identity_map(int n, int* m, cudaStream_t st) {
  wb_launch(k_iota, blocks_for(n, 256), 256, 0, st, n, m);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dinv_A(const Grid& g, int k, const RefTables* dtab, const T* coef, int cn, T* dinv,
                          cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_dinv_stiff<T, N, true>, blocks_for(g.nn, 128), 128, 0, st, g, dtab, coef, cn, dinv)),
                    cudaGetLastError()));
}

template <typename T>
cudaError_t launch_dinv_L(const Grid& g, int k, const RefTables* dtab, const T* coef, T* dinv, cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_dinv_stiff<T, N, false>, blocks_for(g.nn, 128), 128, 0, st, g, dtab, coef, 0, dinv)),
                    cudaGetLastError()));
}

template <typename T>
cudaError_t launch_dinv_Kw(const Grid& g, int k, const RefTables* dtab, const T* cinv, int per_dof, T* dinv,
                           cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_dinv_Kw<T, N>, blocks_for((long long)g.ne * Cfg<N>::NP, 128), 128, 0, st, g, dtab, cinv,
                               per_dof, dinv)),
                    cudaGetLastError()));
}

cudaError_t launch_lumped_weight(const Grid& g, int k, const RefTables* dtab, const double* mu, double a, double* out,
                                 cudaStream_t st) {
  wb_launch(k_lumped, blocks_for(g.nn, 128), 128, 0, st, g, k, dtab, mu, a, out);
  return cudaGetLastError();
}

cudaError_t launch_lumped_mass(const Grid& g, int k, const RefTables* dtab, double* out, cudaStream_t st) {
  wb_launch(k_lumped, blocks_for(g.nn, 128), 128, 0, st, g, k, dtab, nullptr, 1.0, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_p_prolong(const Grid& g1, int k, const RefTables* dtab, int ncomp, const T* in_c, T* out_f, int add,
                             cudaStream_t st) {
  const long long nnf = (long long)(k * g1.nx + 1) * (k * g1.ny + 1) * (k * g1.nz + 1);
  wb_launch(k_p_prolong<T>, blocks_for(nnf, 128), 128, 0, st, g1, k, dtab, ncomp, in_c, out_f, add);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_p_restrict(const Grid& g1, int k, const RefTables* dtab, int ncomp, const T* in_f, T* out_c,
                              int mask_dirichlet, cudaStream_t st) {
  wb_launch(k_p_restrict<T>, blocks_for(g1.nn, 128), 128, 0, st, g1, k, dtab, ncomp, in_f, out_c, mask_dirichlet);
  return cudaGetLastError();
}
template cudaError_t launch_p_prolong<double>(const Grid&, int, const RefTables*, int, const double*, double*, int,
                                              cudaStream_t);
template cudaError_t launch_p_prolong<float>(const Grid&, int, const RefTables*, int, const float*, float*, int,
                                             cudaStream_t);
template cudaError_t launch_p_restrict<double>(const Grid&, int, const RefTables*, int, const double*, double*, int,
                                               cudaStream_t);
template cudaError_t launch_p_restrict<float>(const Grid&, int, const RefTables*, int, const float*, float*, int,
                                              cudaStream_t);

cudaError_t launch_pcoarsen_coef(const Grid& g, int k, const RefTables* dtab, const double* cf, double* cc,
                                 cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_pcoarsen_coef<N>, blocks_for((long long)g.ne * 8, 128), 128, 0, st, g, dtab, cf, cc)),
                    cudaGetLastError()));
}

cudaError_t launch_weight_points(const Grid& g, int k, const RefTables* dtab, const double* mu, int grad, double* w,
                                 cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_weight_points<N>, blocks_for((long long)g.ne * Cfg<N>::N3, 128), 128, 0, st, g, dtab,
                               mu, grad, w)),
                    cudaGetLastError()));
}

cudaError_t launch_lumped_weight_pts(const Grid& g, int k, const RefTables* dtab, const double* wp, double a,
                                     double* out, cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_lumped_pts<N>, blocks_for(g.nn, 128), 128, 0, st, g, dtab, wp, a, out)),
                    cudaGetLastError()));
}

template <typename T>
cudaError_t launch_poisson_coef_pts(const Grid& g, int k, const double* wp, double a, T* c, cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_poisson_coef_pts<T, N>, blocks_for((long long)g.ne * Cfg<N>::N3, 128), 128, 0, st, g,
                               wp, a, c)),
                    cudaGetLastError()));
}
template cudaError_t launch_poisson_coef_pts<double>(const Grid&, int, const double*, double, double*, cudaStream_t);

template <typename T>
cudaError_t launch_poisson_coef0(const Grid& g, int k, const double* mu, double a, T* c, cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_poisson_coef0<T, N>, blocks_for((long long)g.ne * Cfg<N>::N3, 128), 128, 0, st, g, mu, a, 0, c)),
                    cudaGetLastError()));
}

template <typename T>
cudaError_t launch_nodal_to_points(const Grid& g, int k, const double* mu, T* c, cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_poisson_coef0<T, N>, blocks_for((long long)g.ne * Cfg<N>::N3, 128), 128, 0, st, g, mu, 1.0, 1, c)),
                    cudaGetLastError()));
}

template <typename T>
cudaError_t launch_coarsen_coef(const Grid& gf, int k, const RefTables* dtab, const T* cf, T* cc, cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_coarsen_coef<T, N>, blocks_for((long long)(gf.ne / 8) * Cfg<N>::N3, 128), 128, 0, st, gf, dtab, cf, cc)),
                    cudaGetLastError()));
}

template <typename T>
cudaError_t launch_disc_to_cont(const Grid& g, int k, const RefTables* dtab, const T* rd, T* rc, cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_disc_to_cont<T, N>, blocks_for(g.nn, 128), 128, 0, st, g, dtab, rd, rc)), cudaGetLastError()));
}

template <typename T>
cudaError_t launch_cont_to_disc(const Grid& g, int k, const RefTables* dtab, const T* ec, T* ed, int add,
                                cudaStream_t st) {
  WB_DISPATCH_N(k, ((wb_launch(k_cont_to_disc<T, N>, blocks_for(g.ne, 128), 128, 0, st, g, dtab, ec, ed, add)), cudaGetLastError()));
}

size_t transfer_work_size(const Grid& gc, int k) {
  const size_t ncx = gc.NX, ncy = gc.NY, ncz = gc.NZ;
  const size_t nfx = 2 * k * gc.nx + 1, nfy = 2 * k * gc.ny + 1, nfz = 2 * k * gc.nz + 1;
  size_t a = ncz * ncy * nfx, b = nfz * nfy * ncx;      // first pass (prolong / restrict)
  size_t c = ncz * nfy * nfx, d = nfz * ncy * ncx;      // second pass
  size_t m1 = a > b ? a : b, m2 = c > d ? c : d;
  return m1 > m2 ? m1 : m2;
}

template <typename T>
cudaError_t launch_prolong(const Grid& gc, int k, const RefTables* dtab, int ncomp, const T* in_c, T* out_f, int add,
                           T* w1, T* w2, cudaStream_t st) {
  const int ncx = gc.NX, ncy = gc.NY, ncz = gc.NZ;
  const int nfx = 2 * k * gc.nx + 1, nfy = 2 * k * gc.ny + 1, nfz = 2 * k * gc.nz + 1;
  const size_t nc = (size_t)ncx * ncy * ncz, nf = (size_t)nfx * nfy * nfz;
  const int bs = 256;
  for (int c = 0; c < ncomp; ++c) {
    const T* in = in_c + c * nc;
    T* out = out_f + c * nf;
    wb_launch(k_pass<T>, blocks_for((long long)nfx * ncy * ncz, bs), bs, 0, st, dtab, k, 0, ncx, ncy, ncz, gc.nx, 1, in, w1, 0);
    wb_launch(k_pass<T>, blocks_for((long long)nfx * nfy * ncz, bs), bs, 0, st, dtab, k, 1, nfx, ncy, ncz, gc.ny, 1, w1, w2, 0);
    wb_launch(k_pass<T>, blocks_for((long long)nfx * nfy * nfz, bs), bs, 0, st, dtab, k, 2, nfx, nfy, ncz, gc.nz, 1, w2, out, add);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const Grid& gc, int k, const RefTables* dtab, int ncomp, const T* in_f, T* out_c,
                            int mask, T* w1, T* w2, cudaStream_t st) {
  const int ncx = gc.NX, ncy = gc.NY, ncz = gc.NZ;
  const int nfx = 2 * k * gc.nx + 1, nfy = 2 * k * gc.ny + 1, nfz = 2 * k * gc.nz + 1;
  const size_t nc = (size_t)ncx * ncy * ncz, nf = (size_t)nfx * nfy * nfz;
  const int bs = 256;
  for (int c = 0; c < ncomp; ++c) {
    const T* in = in_f + c * nf;
    T* out = out_c + c * nc;
    wb_launch(k_pass<T>, blocks_for((long long)ncx * nfy * nfz, bs), bs, 0, st, dtab, k, 0, nfx, nfy, nfz, gc.nx, 0, in, w1, 0);
    wb_launch(k_pass<T>, blocks_for((long long)ncx * ncy * nfz, bs), bs, 0, st, dtab, k, 1, ncx, nfy, nfz, gc.ny, 0, w1, w2, 0);
    wb_launch(k_pass<T>, blocks_for((long long)ncx * ncy * ncz, bs), bs, 0, st, dtab, k, 2, ncx, ncy, nfz, gc.nz, 0, w2, out, 0);
  }
  if (mask) wb_launch(k_mask_boundary<T>, blocks_for(gc.nn, 256), 256, 0, st, gc, ncomp, out_c);
  return cudaGetLastError();
}

cudaError_t launch_sinker(const Grid& g, int k, const RefTables& htab, const double* centres, int ns, double omega,
                          double delta, double dr, double beta, double* mu, double* f, cudaStream_t st,
                          const double* X) {
  if (ns < 0 || ns > 128) return cudaErrorInvalidValue;
  Centres cs;
  for (int s = 0; s < ns; ++s)
    for (int d = 0; d < 3; ++d) cs.c[s][d] = centres[3 * s + d];
  for (int a = 0; a < WB_MAXN; ++a) cs.x[a] = htab.x[a];
  wb_launch(k_sinker, blocks_for(g.nn, 128), 128, 0, st, g, k, cs, X, ns, omega, delta, dr, beta, mu, f);
  return cudaGetLastError();
}

cudaError_t launch_node_coords(const Grid& g, int k, const RefTables& htab, double* X, cudaStream_t st) {
  Centres cs;
  for (int a = 0; a < WB_MAXN; ++a) cs.x[a] = htab.x[a];
  wb_launch(k_node_coords, blocks_for(g.nn, 128), 128, 0, st, g, k, cs, X);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mask_boundary(const Grid& g, int ncomp, T* v, cudaStream_t st) {
  wb_launch(k_mask_boundary<T>, blocks_for(g.nn, 256), 256, 0, st, g, ncomp, v);
  return cudaGetLastError();
}

namespace {
// u_i = top 53 bits of the (i+1)-th SplitMix64 output of state `seed`, shifted to [-0.5, 0.5)
// (SplitMix64: Steele, Lea & Flood, OOPSLA 2014).
template <typename T>
__global__ void k_splitmix_start(long long n, unsigned long long seed, T* __restrict__ v) {
  pdl_entry();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long z = seed + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  v[i] = T((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
}

// F_c(n) = lm(n) f_c(n) on interior nodes, 0 on the boundary
__global__ void k_load_vector(Grid g, const double* __restrict__ lm, const double* __restrict__ f, double* __restrict__ F) {
  pdl_entry();
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= g.nn) return;
  const int ix = n % g.NX, iy = (n / g.NX) % g.NY, iz = n / (g.NX * g.NY);
  const bool b = on_boundary(g, ix, iy, iz);
  for (int c = 0; c < 3; ++c) F[(size_t)c * g.nn + n] = b ? 0.0 : lm[n] * f[(size_t)c * g.nn + n];
}
}  // namespace

template <typename T>
cudaError_t launch_splitmix_start(long long n, unsigned long long seed, T* v, cudaStream_t st) {
  wb_launch(k_splitmix_start<T>, blocks_for(n, 256), 256, 0, st, n, seed, v);
  return cudaGetLastError();
}

cudaError_t launch_load_vector(const Grid& g, const double* lm, const double* f, double* F, cudaStream_t st) {
  wb_launch(k_load_vector, blocks_for(g.nn, 256), 256, 0, st, g, lm, f, F);
  return cudaGetLastError();
}

// explicit instantiations
#define WB_INST(T)                                                                                                  \
  template cudaError_t launch_stokes<T>(const Grid&, int, const RefTables*, int, const T*, const T*, const T*,      \
                                        const T*, int, T*, T*, cudaStream_t);                                       \
  template cudaError_t launch_poisson<T>(const Grid&, int, const RefTables*, const T*, const T*, T*, cudaStream_t); \
  template cudaError_t launch_dinv_A<T>(const Grid&, int, const RefTables*, const T*, int, T*, cudaStream_t);       \
  template cudaError_t launch_dinv_L<T>(const Grid&, int, const RefTables*, const T*, T*, cudaStream_t);            \
  template cudaError_t launch_dinv_Kw<T>(const Grid&, int, const RefTables*, const T*, int, T*, cudaStream_t);           \
  template cudaError_t launch_poisson_coef0<T>(const Grid&, int, const double*, double, T*, cudaStream_t);          \
  template cudaError_t launch_nodal_to_points<T>(const Grid&, int, const double*, T*, cudaStream_t);                \
  template cudaError_t launch_coarsen_coef<T>(const Grid&, int, const RefTables*, const T*, T*, cudaStream_t);      \
  template cudaError_t launch_disc_to_cont<T>(const Grid&, int, const RefTables*, const T*, T*, cudaStream_t);      \
  template cudaError_t launch_cont_to_disc<T>(const Grid&, int, const RefTables*, const T*, T*, int, cudaStream_t); \
  template cudaError_t launch_prolong<T>(const Grid&, int, const RefTables*, int, const T*, T*, int, T*, T*,        \
                                         cudaStream_t);                                                             \
  template cudaError_t launch_restrict<T>(const Grid&, int, const RefTables*, int, const T*, T*, int, T*, T*,       \
                                          cudaStream_t);
WB_INST(double)
WB_INST(float)
template cudaError_t launch_mask_boundary<double>(const Grid&, int, double*, cudaStream_t);
template cudaError_t launch_mask_boundary<float>(const Grid&, int, float*, cudaStream_t);
template cudaError_t launch_splitmix_start<double>(long long, unsigned long long, double*, cudaStream_t);
template cudaError_t launch_splitmix_start<float>(long long, unsigned long long, float*, cudaStream_t);
