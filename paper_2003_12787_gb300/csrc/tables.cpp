// Reference-element tables of the library (host, extended precision).
//
// Gauss-Legendre nodes on [0,1] (Sec. II-A: nodal Lagrange basis on
// Gauss-Legendre points, N points per dimension), the collocation derivative
// matrix D_ij = phi_j'(xi_i) and the face interpolation vectors phi_j(0),
// phi_j(1). Nodes: Newton's method on the Legendre polynomial from a cosine
// initial guess; D and phi: barycentric Lagrange formulas (Berrut & Trefethen,
// SIAM Review 46(3), 2004), with the diagonal of D from the zero row sum.
// Arithmetic in long double, rounded to double once at the end.
#include <cmath>

#include "stp_internal.h"

namespace stp {
namespace {

using ld = long double;

// P_n(x) and P_n'(x) on [-1,1] by the Bonnet recurrence.
void legendre_pair(int n, ld x, ld* p, ld* dp) {
  ld p0 = 1.0L, p1 = x;
  if (n == 0) { *p = 1.0L; *dp = 0.0L; return; }
  for (int k = 2; k <= n; ++k) {
    ld p2 = ((2.0L * k - 1.0L) * x * p1 - (k - 1.0L) * p0) / (ld)k;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = (ld)n * (x * p1 - p0) / (x * x - 1.0L);
}

}  // namespace

bool make_tables(int N, HostTables* t) {
  if (N < 1 || N > kMaxNodes) return false;
  t->N = N;
  const ld pi = 3.141592653589793238462643383279502884L;
  ld x[kMaxNodes];
  for (int i = 0; i < N; ++i) {
    // i-th largest root on [-1,1]
    ld r = cosl(pi * ((ld)i + 0.75L) / ((ld)N + 0.5L));
    bool ok = false;
    for (int it = 0; it < 100; ++it) {
      ld p, dp;
      if (N == 1) { r = 0.0L; ok = true; break; }
      legendre_pair(N, r, &p, &dp);
      ld step = p / dp;
      r -= step;
      if (fabsl(step) <= 4.0L * 1.1e-19L * (1.0L + fabsl(r))) { ok = true; break; }
    }
    if (!ok) return false;
    x[N - 1 - i] = 0.5L * (1.0L + r);  // ascending on [0,1]
  }
  // barycentric weights
  ld w[kMaxNodes];
  for (int j = 0; j < N; ++j) {
    ld prod = 1.0L;
    for (int k = 0; k < N; ++k)
      if (k != j) prod *= (x[j] - x[k]);
    w[j] = 1.0L / prod;
  }
  for (int i = 0; i < N; ++i) {
    ld diag = 0.0L;
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      ld dij = (w[j] / w[i]) / (x[i] - x[j]);
      t->D[i * N + j] = (double)dij;
      diag -= dij;
    }
    t->D[i * N + i] = (double)diag;
    t->nodes[i] = (double)x[i];
  }
  for (int side = 0; side < 2; ++side) {
    const ld a = side ? 1.0L : 0.0L;
    ld den = 0.0L;
    for (int k = 0; k < N; ++k) den += w[k] / (a - x[k]);
    for (int j = 0; j < N; ++j) {
      ld v = (w[j] / (a - x[j])) / den;
      (side ? t->phi1 : t->phi0)[j] = (double)v;
    }
  }
  return true;
}

void make_step_matrices(const HostTables& t, double dx, double dt, double* Dk) {
  const int N = t.N;
  for (int k = 0; k < N; ++k) {
    const ld s = (ld)dt / ((ld)(k + 2) * (ld)dx);
    for (int i = 0; i < N * N; ++i) Dk[k * N * N + i] = (double)((ld)t.D[i] * s);
  }
}

}  // namespace stp
