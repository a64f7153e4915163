// Host construction of the 1-D GLL tables, the P_{k-1} monomial basis data and
// the per-axis transfer weights.  Everything is computed from its definition:
//  * GLL nodes: -1, +1 and the roots of P_k', found by Newton's method on P_k'
//    from Chebyshev-Gauss-Lobatto starting points; weights 2 / (k (k+1) P_k(x)^2).
//  * Differentiation: barycentric weights lambda_j = 1 / prod_{m != j} (x_j - x_m),
//    D[i][j] = (lambda_j / lambda_i) / (x_i - x_j), D[i][i] = -sum_{j != i} D[i][j].
//  * Pressure basis: monomials of total degree <= k-1, ordered by degree and then
//    lexicographically descending in the exponent triple.
//  * Nested interpolation between a coarse cell and its two children per axis,
//    and the coefficient-coarsening weights (normalised L^2-adjoint of per-axis
//    piecewise-linear interpolation on the GLL sub-grid, Sec. 6).
#include "tables.h"

#include <cmath>
#include <cstring>

namespace {

// Legendre P_k(x) and P_{k-1}(x) by the three-term recurrence.
void legendre(int k, double x, double* pk, double* pkm1) {
  double p0 = 1.0, p1 = x;
  if (k == 0) { *pk = 1.0; *pkm1 = 0.0; return; }
  for (int j = 2; j <= k; ++j) {
    double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  *pk = p1;
  *pkm1 = p0;
}

double lagrange(const double* x, int n, int b, double t) {
  double v = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != b) v *= (t - x[m]) / (x[b] - x[m]);
  return v;
}

double hat(const double* x, int n, int i, double t) {
  if (i > 0 && t >= x[i - 1] && t <= x[i]) return (t - x[i - 1]) / (x[i] - x[i - 1]);
  if (i < n - 1 && t >= x[i] && t <= x[i + 1]) return (x[i + 1] - t) / (x[i + 1] - x[i]);
  return 0.0;
}

bool invert(int n, double a[WB_MAXNP][WB_MAXNP], double inv[WB_MAXNP][WB_MAXNP]) {
  double m[WB_MAXNP][2 * WB_MAXNP];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) m[i][j] = j < n ? a[i][j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(m[r][c]) > std::fabs(m[piv][c])) piv = r;
    if (m[piv][c] == 0.0) return false;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) { double t = m[c][j]; m[c][j] = m[piv][j]; m[piv][j] = t; }
    double d = m[c][c];
    for (int j = 0; j < 2 * n; ++j) m[c][j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = m[r][c];
      if (f != 0.0)
        for (int j = 0; j < 2 * n; ++j) m[r][j] -= f * m[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) inv[i][j] = m[i][j + n];
  return true;
}

}  // namespace

bool build_ref_tables(int k, RefTables* t) {
  if (k < 1 || k > 4) return false;
  std::memset(t, 0, sizeof(*t));
  const int n = k + 1;
  t->k = k;
  t->n = n;
  t->np = k * (k + 1) * (k + 2) / 6;

  // GLL nodes
  t->x[0] = -1.0;
  t->x[k] = 1.0;
  const double pi = 3.14159265358979323846;
  for (int i = 1; i < k; ++i) {
    double x = -std::cos(pi * i / k);
    for (int it = 0; it < 100; ++it) {
      double pk, pkm1;
      legendre(k, x, &pk, &pkm1);
      double dp = k * (x * pk - pkm1) / (x * x - 1.0);            // P_k'
      double d2p = (2.0 * x * dp - k * (k + 1.0) * pk) / (1.0 - x * x);  // Legendre ODE
      double dx = dp / d2p;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    t->x[i] = x;
  }
  // symmetrise (the node set is symmetric about 0)
  for (int i = 0; i < n / 2; ++i) {
    double s = 0.5 * (t->x[n - 1 - i] - t->x[i]);
    t->x[i] = -s;
    t->x[n - 1 - i] = s;
  }
  if (n % 2) t->x[n / 2] = 0.0;
  for (int i = 0; i < n; ++i) {
    double pk, pkm1;
    legendre(k, t->x[i], &pk, &pkm1);
    t->w[i] = 2.0 / (k * (k + 1.0) * pk * pk);
  }
  // barycentric differentiation matrix
  double lam[WB_MAXN];
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) p *= (t->x[j] - t->x[m]);
    lam[j] = 1.0 / p;
  }
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      t->D[i][j] = (lam[j] / lam[i]) / (t->x[i] - t->x[j]);
      s += t->D[i][j];
    }
    t->D[i][i] = -s;
  }
  for (int i = 0; i < n; ++i) {
    double v = 1.0;
    for (int a = 0; a < n; ++a) { t->pw[i][a] = v; v *= t->x[i]; }
  }
  // pressure exponents: total degree d = 0..k-1, (a,b,c) descending lexicographic
  int m = 0;
  for (int d = 0; d < k; ++d)
    for (int a = d; a >= 0; --a)
      for (int b = d - a; b >= 0; --b) {
        int c = d - a - b;
        t->ex[m][0] = a; t->ex[m][1] = b; t->ex[m][2] = c;
        ++m;
      }
  // reference pressure mass with GLL quadrature (exact for degree <= 2k-1 per axis)
  double mass[WB_MAXNP][WB_MAXNP];
  for (int r = 0; r < t->np; ++r)
    for (int c = 0; c < t->np; ++c) {
      double s = 0.0;
      for (int l = 0; l < n; ++l)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            double W = t->w[i] * t->w[j] * t->w[l];
            double pr = t->pw[i][t->ex[r][0]] * t->pw[j][t->ex[r][1]] * t->pw[l][t->ex[r][2]];
            double pc = t->pw[i][t->ex[c][0]] * t->pw[j][t->ex[c][1]] * t->pw[l][t->ex[c][2]];
            s += W * pr * pc;
          }
      mass[r][c] = s;
    }
  if (!invert(t->np, mass, t->minv)) return false;
  // transfers between a coarse cell and its two children along one axis
  for (int s = 0; s < 2; ++s)
    for (int a = 0; a < n; ++a) {
      double tc = 0.5 * (t->x[a] + 2.0 * s - 1.0);
      for (int b = 0; b < n; ++b) t->P1[s][a][b] = lagrange(t->x, n, b, tc);
    }
  for (int i = 0; i < n; ++i) {
    double den = 0.0;
    for (int s = 0; s < 2; ++s)
      for (int ip = 0; ip < n; ++ip) den += t->w[ip] * hat(t->x, n, i, 0.5 * (t->x[ip] + 2.0 * s - 1.0));
    for (int s = 0; s < 2; ++s)
      for (int ip = 0; ip < n; ++ip)
        t->Tc[s][i][ip] = t->w[ip] * hat(t->x, n, i, 0.5 * (t->x[ip] + 2.0 * s - 1.0)) / den;
  }
  return true;
}
