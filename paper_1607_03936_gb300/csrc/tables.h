// Reference-element tables for the Q_k x P_{k-1}^disc pair (Sec. 1.2), built on the host.
#pragma once

#define WB_MAXN 5    // k + 1 for k <= 4
#define WB_MAXNP 20  // k (k+1) (k+2) / 6 for k <= 4

struct RefTables {
  int k, n, np;
  double x[WB_MAXN];                 // GLL nodes on [-1, 1]
  double w[WB_MAXN];                 // GLL weights
  double D[WB_MAXN][WB_MAXN];        // D[i][j] = l_j'(x_i)
  double pw[WB_MAXN][WB_MAXN];       // pw[i][a] = x_i^a
  int ex[WB_MAXNP][3];               // pressure monomial exponents, psi_m = xi^a eta^b zeta^c
  double minv[WB_MAXNP][WB_MAXNP];   // inverse of the reference pressure mass (|J| = 1)
  double P1[2][WB_MAXN][WB_MAXN];    // P1[s][a][b] = l_b((x_a + 2s - 1) / 2): child s of a coarse cell
  double Tc[2][WB_MAXN][WB_MAXN];    // coefficient coarsening weights per axis, Tc[s][i][i']
};

// Fill t for order k in {1, 2, 3, 4} (k = 1: the trilinear levels of the p-coarsened viscous
// multigrid; the solver itself takes k >= 2); returns false for other k.
bool build_ref_tables(int k, RefTables* t);
