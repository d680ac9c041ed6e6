// Reference-element tables of the library (host, extended precision).
//
// Nodes on [0,1] (Sec. II-A: nodal Lagrange basis on Gauss-Legendre or
// Gauss-Lobatto points, N points per dimension), the collocation derivative
// matrix D_ij = phi_j'(xi_i) and the face interpolation vectors phi_j(0),
// phi_j(1). Gauss-Legendre nodes: Newton's method on P_N from a cosine
// initial guess. Gauss-Lobatto nodes: the end points and Newton's method on
// P_{N-1}' (second derivative from the Legendre equation) from the
// Chebyshev-Lobatto points. D and phi: barycentric Lagrange formulas (Berrut
// & Trefethen, SIAM Review 46(3), 2004), with the diagonal of D from the zero
// row sum; phi is a unit vector where the face coincides with a node.
// Arithmetic in long double, rounded to double once at the end.
#include <cmath>
#include <cstdint>
#include <cstring>

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

// Gauss-Lobatto points on [-1,1], descending into x[0..N-1] (N >= 2).
bool lobatto_points(int N, ld* x) {
  const ld pi = 3.141592653589793238462643383279502884L;
  const int n = N - 1;
  x[0] = 1.0L;
  x[N - 1] = -1.0L;
  for (int i = 1; i < N - 1; ++i) {
    ld r = cosl(pi * (ld)i / (ld)n);
    bool ok = false;
    for (int it = 0; it < 100; ++it) {
      ld p, dp;
      legendre_pair(n, r, &p, &dp);
      const ld d2p = (2.0L * r * dp - (ld)n * (n + 1) * p) / (1.0L - r * r);
      const ld step = dp / d2p;
      r -= step;
      if (fabsl(step) <= 4.0L * 1.1e-19L * (1.0L + fabsl(r))) { ok = true; break; }
    }
    if (!ok) return false;
    x[i] = r;
  }
  return true;
}

bool make_tables(int N, HostTables* t, int family) {
  if (N < 1 || N > kMaxNodes) return false;
  if (family != STP_NODES_GAUSS_LEGENDRE && family != STP_NODES_GAUSS_LOBATTO) return false;
  if (family == STP_NODES_GAUSS_LOBATTO && N < 2) return false;
  t->N = N;
  t->family = family;
  const ld pi = 3.141592653589793238462643383279502884L;
  ld x[kMaxNodes];
  if (family == STP_NODES_GAUSS_LOBATTO) {
    ld r[kMaxNodes];
    if (!lobatto_points(N, r)) return false;
    for (int i = 0; i < N; ++i) x[N - 1 - i] = 0.5L * (1.0L + r[i]);  // ascending on [0,1]
  }
  for (int i = 0; i < N && family == STP_NODES_GAUSS_LEGENDRE; ++i) {
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
  // quadrature weights on [0,1]: Gauss-Legendre 1/((1-t^2) P_N'(t)^2),
  // Gauss-Lobatto 1/(N (N-1) P_{N-1}(t)^2), t = 2x - 1
  for (int i = 0; i < N; ++i) {
    const ld tt = 2.0L * x[i] - 1.0L;
    ld p, dp;
    if (family == STP_NODES_GAUSS_LOBATTO) {
      legendre_pair(N - 1, tt, &p, &dp);
      t->weights[i] = (double)(1.0L / ((ld)N * (ld)(N - 1) * p * p));
    } else if (N == 1) {
      t->weights[i] = 1.0;
    } else {
      legendre_pair(N, tt, &p, &dp);
      t->weights[i] = (double)(1.0L / ((1.0L - tt * tt) * dp * dp));
    }
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
    double* phi = side ? t->phi1 : t->phi0;
    int hit = -1;
    for (int k = 0; k < N; ++k)
      if (x[k] == a) hit = k;
    if (hit >= 0) {  // the face point is a node
      for (int j = 0; j < N; ++j) phi[j] = j == hit ? 1.0 : 0.0;
      continue;
    }
    ld den = 0.0L;
    for (int k = 0; k < N; ++k) den += w[k] / (a - x[k]);
    for (int j = 0; j < N; ++j) phi[j] = (double)((w[j] / (a - x[j])) / den);
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

namespace stp {
namespace {

// IEEE binary16 (bf16 = false) or bfloat16 bits of v, which must be exactly
// representable (checked; false otherwise).
bool encode16(double v, bool bf16, uint16_t* bits) {
  if (v == 0.0) { *bits = 0; return true; }
  const uint16_t sign = v < 0 ? 0x8000u : 0u;
  const double a = std::fabs(v);
  int ex;
  const double m = std::frexp(a, &ex);  // a = m 2^ex, m in [0.5, 1)
  const int mbits = bf16 ? 7 : 10, bias = bf16 ? 127 : 15;
  const int E = ex - 1 + bias;
  if (E >= (bf16 ? 255 : 31)) return false;
  double frac;
  uint32_t e_field;
  if (E >= 1) {
    frac = std::ldexp(2.0 * m - 1.0, mbits);
    e_field = (uint32_t)E;
  } else {  // subnormal: a = frac 2^(1 - bias - mbits)
    frac = std::ldexp(a, bias - 1 + mbits);
    e_field = 0;
  }
  if (frac != std::floor(frac) || frac >= std::ldexp(1.0, mbits)) return false;
  *bits = (uint16_t)(sign | (e_field << mbits) | (uint32_t)frac);
  return true;
}

}  // namespace

bool make_tc_tiles(const HostTables& t, int eD, unsigned char* out) {
  const int N = t.N;
  std::memset(out, 0, kTcRegionBytes);
  if (N > 10) return true;  // the tensor-core kernel covers N <= 10
  for (int type = 0; type < 2; ++type) {
    const bool bf16 = type == 1;
    const int W = bf16 ? 8 : 10, c = bf16 ? 0 : 6;
    for (int i = 0; i < N; ++i)
      for (int l = 0; l < N; ++l) {
        double dig[3];
        double x = std::ldexp(t.D[i * N + l], W - 1 - eD);
        for (int d = 0; d < 3; ++d) {
          dig[d] = std::nearbyint(x);
          x = std::ldexp(x - dig[d], W);
        }
        for (int T = 1; T <= 3; ++T) {
          unsigned char* op = out + (type * 3 + (T - 1)) * kTcOperandBytes;
          for (int s = 0; s < T; ++s) {
            const int k = N * s + l, chunk = k >> 4, kk = k & 15;
            auto put = [&](int row, double v) {
              uint16_t b;
              if (!encode16(v, bf16, &b)) return false;
              const int off = chunk * kTcChunkBytes + (row >> 3) * 256 + (kk >> 3) * 128 + (row & 7) * 16 + (kk & 7) * 2;
              std::memcpy(op + off, &b, 2);
              return true;
            };
            if (s == 0 && !put(i, dig[0])) return false;
            if (s <= 1 && !put(N + i, std::ldexp(dig[1 - s], c))) return false;
            if (!put(2 * N + i, std::ldexp(dig[2 - s], c - W))) return false;
          }
        }
      }
  }
  return true;
}

}  // namespace stp
