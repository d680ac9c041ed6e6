/*
 * Plain FP64 CPU oracle of the linear ADER-DG Space-Time Predictor (STP).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline use it. It shares no code, header, table or constant generator with
 * the CUDA library; it is written to be slow and obviously correct.
 *
 * What it computes (Gallard et al., "Vectorization and Minimization of Memory
 * Footprint for Linear High-Order Discontinuous Galerkin Schemes", arXiv
 * 2003.12787):
 *   - Sec. II-A: nodal tensor-product Lagrange basis on N Gauss-Legendre (or,
 *     as the paper allows, Gauss-Lobatto) nodes per dimension of the
 *     reference cube [0,1]^3; the discrete derivative operator D; N nodes per
 *     dimension ("order N" in the paper's wording).
 *   - Eq. (exahypeTimeAverage) and the recurrence below it: the Taylor series
 *     of the cell-local solution in time, built from powers of the volume
 *     operator V applied to q(t_n): p_o = V p_{o-1}.
 *   - Sec. II-B: the STP outputs the time-averaged degrees of freedom and
 *     their projection onto the element faces.
 *   - Sec. VI (benchmark setup): 3-D elastic wave equation, 3 velocities and
 *     6 stresses, 3 material parameters per node; on curvilinear meshes 9
 *     geometry parameters per node more (oracle_stp_curvilinear).
 *
 * Readings (the paper is silent or its pseudocode is garbled on these):
 *   - The operator is taken in the form q_t + sum_d B_d dq/dx_d = 0, so one CK
 *     step is  q^(k+1) = - sum_d B_d(x) (D_d q^(k)) / h.
 *   - K Taylor terms q^(0..K-1); the default reading is K = N + 1 (the sum in
 *     Eq. (exahypeTimeAverage) runs over o = 0..N).
 *   - The output is the time AVERAGE  sum_k dt^k/(k+1)! q^(k)  (the paper's
 *     integral divided by dt).
 *   - D_ij = phi_j'(xi_i) (strong collocation form), nodes on [0,1],
 *     derivatives divided by the element side h.
 *   - Quantity order (v1,v2,v3,s11,s22,s33,s12,s13,s23); material (rho,cp,cs)
 *     with lambda = rho (cp^2 - 2 cs^2), mu = rho cs^2 (textbook
 *     velocity-stress elasticity).
 *   - Faces ordered x-,x+,y-,y+,z-,z+; in-plane indices are the two remaining
 *     dimensions in (slower, faster) order.
 *
 * Layouts (row-major, last index fastest):
 *   q, avg:   [E][N][N][N][9]   (element, z, y, x, quantity)
 *   params:   [E][N][N][N][3]   (rho, cp, cs)
 *   faces:    [E][6][N][N][9]
 *   terms:    [E][K][N][N][N][9]  (optional: every q^(k), unscaled)
 *   metric:   [E][N][N][N][9]   (curvilinear elements: dxi_d/dx_j at 3d + j)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define M 9 /* quantities of the elastic system */

/* Legendre polynomial P_n(x) on [-1,1] by the three-term (Bonnet) recurrence. */
static double legendre(int n, double x) {
  double p0 = 1.0, p1 = x;
  if (n == 0) return p0;
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

/* Derivative P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1), valid inside (-1,1). */
static double legendre_deriv(int n, double x) {
  return n * (x * legendre(n, x) - legendre(n - 1, x)) / (x * x - 1.0);
}

/*
 * Gauss-Legendre nodes xi[0..N-1] (ascending) and weights w[0..N-1] on [0,1].
 * The nodes are the N roots of P_N(2 xi - 1): every root is bracketed by a
 * sign change on a fine uniform grid and then bisected down to adjacent
 * doubles. Weights: w = 1 / ((1 - t^2) P_N'(t)^2) for t = 2 xi - 1 (the [-1,1]
 * weight 2/((1-t^2)P_N'(t)^2) halved for the unit interval).
 * Returns 0, or -1 if fewer than N roots were found.
 */
int oracle_gl_nodes(int N, double* xi, double* w) {
  if (N < 1 || N > 64) return -1;
  int found = 0;
  const int samples = 4000 * N;
  double a = -1.0, fa = legendre(N, a);
  for (int s = 1; s <= samples && found < N; ++s) {
    double b = -1.0 + 2.0 * s / samples;
    double fb = legendre(N, b);
    if (fb == 0.0) { /* root exactly on the grid */
      xi[found++] = b;
      a = b; fa = fb;
      /* step past it so the same root is not bracketed again */
      continue;
    }
    if (fa != 0.0 && ((fa < 0.0) != (fb < 0.0))) {
      double lo = a, hi = b, flo = fa;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double fm = legendre(N, mid);
        if (fm == 0.0) { lo = hi = mid; break; }
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      xi[found++] = 0.5 * (lo + hi);
    }
    a = b; fa = fb;
  }
  if (found != N) return -1;
  for (int i = 0; i < N; ++i) {
    double t = xi[i];
    double dp = legendre_deriv(N, t);
    if (w) w[i] = 1.0 / ((1.0 - t * t) * dp * dp);
    xi[i] = 0.5 * (t + 1.0);
  }
  return 0;
}

/*
 * Gauss-Lobatto nodes xi[0..N-1] (ascending, N >= 2) and weights w on [0,1]:
 * the end points and the N-2 roots of P_{N-1}'(2 xi - 1), each interior root
 * bracketed by a sign change on a fine uniform grid of the open interval and
 * bisected down to adjacent doubles. Weights: 1 / (N (N-1) P_{N-1}(t)^2) for
 * t = 2 xi - 1 (the [-1,1] weight 2/(N(N-1) P_{N-1}(t)^2) halved).
 * Returns 0, or -1 if fewer than N-2 interior roots were found.
 */
int oracle_gll_nodes(int N, double* xi, double* w) {
  if (N < 2 || N > 64) return -1;
  const int n = N - 1;
  double t[64];
  t[0] = -1.0;
  int found = 1;
  const int samples = 4000 * N;
  double a = -1.0 + 1.0 / samples, fa = legendre_deriv(n, a);
  for (int s = 1; s < samples && found < N - 1; ++s) {
    double b = -1.0 + (2.0 * s + 1.0) / samples;  /* stays inside (-1,1) */
    double fb = legendre_deriv(n, b);
    if (fb == 0.0) {
      t[found++] = b;
      a = b; fa = fb;
      continue;
    }
    if (fa != 0.0 && ((fa < 0.0) != (fb < 0.0))) {
      double lo = a, hi = b, flo = fa;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double fm = legendre_deriv(n, mid);
        if (fm == 0.0) { lo = hi = mid; break; }
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      t[found++] = 0.5 * (lo + hi);
    }
    a = b; fa = fb;
  }
  if (found != N - 1) return -1;
  t[N - 1] = 1.0;
  for (int i = 0; i < N; ++i) {
    double p = legendre(n, t[i]);
    if (w) w[i] = 1.0 / (N * (N - 1.0) * p * p);
    xi[i] = 0.5 * (t[i] + 1.0);
  }
  return 0;
}

/* Lagrange basis phi_j(x) = prod_{l != j} (x - xi_l) / (xi_j - xi_l). */
static double lagrange(int N, const double* xi, int j, double x) {
  double v = 1.0;
  for (int l = 0; l < N; ++l)
    if (l != j) v *= (x - xi[l]) / (xi[j] - xi[l]);
  return v;
}

/* phi_j'(x) by the product rule on the same definition. */
static double lagrange_deriv(int N, const double* xi, int j, double x) {
  double s = 0.0;
  for (int m = 0; m < N; ++m) {
    if (m == j) continue;
    double t = 1.0 / (xi[j] - xi[m]);
    for (int l = 0; l < N; ++l)
      if (l != j && l != m) t *= (x - xi[l]) / (xi[j] - xi[l]);
    s += t;
  }
  return s;
}

/*
 * Tables of the reference element: D[i*N+j] = phi_j'(xi_i), phi0[j] = phi_j(0),
 * phi1[j] = phi_j(1). nodes: 0 Gauss-Legendre, 1 Gauss-Lobatto. Any output
 * pointer may be NULL.
 */
int oracle_tables_nodes(int nodes, int N, double* xi_out, double* D, double* phi0, double* phi1) {
  double xi[64];
  if (nodes == 0) {
    if (oracle_gl_nodes(N, xi, NULL) != 0) return -1;
  } else if (nodes == 1) {
    if (oracle_gll_nodes(N, xi, NULL) != 0) return -1;
  } else {
    return -1;
  }
  if (xi_out) memcpy(xi_out, xi, sizeof(double) * N);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      if (D) D[i * N + j] = lagrange_deriv(N, xi, j, xi[i]);
  for (int j = 0; j < N; ++j) {
    if (phi0) phi0[j] = lagrange(N, xi, j, 0.0);
    if (phi1) phi1[j] = lagrange(N, xi, j, 1.0);
  }
  return 0;
}

/* Gauss-Legendre tables (the default node family). */
int oracle_tables(int N, double* xi_out, double* D, double* phi0, double* phi1) {
  return oracle_tables_nodes(0, N, xi_out, D, phi0, phi1);
}

/*
 * B_d (9x9, row r = equation of quantity r, column s = d/dx_d of quantity s)
 * of the elastic system written as q_t + sum_d B_d dq/dx_d = 0:
 *   rho dv_i/dt = sum_j d sigma_ij / dx_j
 *   d sigma_ij/dt = lambda delta_ij div v + mu (dv_i/dx_j + dv_j/dx_i)
 * Quantity indices: v1 0, v2 1, v3 2, s11 3, s22 4, s33 5, s12 6, s13 7, s23 8.
 */
static void elastic_B(int d, double rho, double cp, double cs, double B[M][M]) {
  const double lam = rho * (cp * cp - 2.0 * cs * cs);
  const double mu = rho * cs * cs;
  static const int sig[3][3] = {{3, 6, 7}, {6, 4, 8}, {7, 8, 5}};
  memset(B, 0, sizeof(double) * M * M);
  /* velocities: dv_i/dt = (1/rho) d sigma_{i d}/dx_d */
  for (int i = 0; i < 3; ++i) B[i][sig[i][d]] = -1.0 / rho;
  /* normal stresses: d s_ii/dt = lambda dv_d/dx_d + 2 mu delta_id dv_d/dx_d */
  for (int i = 0; i < 3; ++i) B[3 + i][d] = -(lam + (i == d ? 2.0 * mu : 0.0));
  /* shear stresses s_ij (i<j): mu (dv_i/dx_j + dv_j/dx_i) */
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j) {
      int r = sig[i][j];
      if (d == j) B[r][i] += -mu;
      if (d == i) B[r][j] += -mu;
    }
}

/* B_d as a row-major 9x9 array, for the corrector (corrector_oracle.c) and
   the tests */
void oracle_elastic_B(int d, double rho, double cp, double cs, double* B) {
  double b[M][M];
  elastic_B(d, rho, cp, cs, b);
  memcpy(B, b, sizeof(b));
}

/* flat index of node (z,y,x) quantity s inside one element */
#define NODE(z, y, x) (((z) * N + (y)) * N + (x))

/*
 * One element. q, params, avg, faces point at that element's blocks; terms
 * (may be NULL) at its [K][N][N][N][9] block. metric (may be NULL) points at
 * the element's [N][N][N][9] block of inverse Jacobians; without it the
 * element is a cube of side h.
 */
static void stp_element(int N, int K, double h, double dt, const double* D,
                        const double* phi0, const double* phi1, const double* q,
                        const double* params, const double* metric, const double* src,
                        double* avg, double* faces, double* terms, double* p, double* pn,
                        double* g) {
  const int n3 = N * N * N;
  memcpy(p, q, sizeof(double) * n3 * M);
  memcpy(avg, q, sizeof(double) * n3 * M);
  if (terms) memcpy(terms, q, sizeof(double) * n3 * M);
  double c = 1.0; /* dt^k / (k+1)! for the term being added */
  for (int k = 0; k + 1 < K; ++k) {
    /* pn = - sum_d B_d (D_d p) / h  : one application of the volume operator */
    memset(pn, 0, sizeof(double) * n3 * M);
    for (int d = 0; d < 3; ++d) {
      /* g = (1/h) D applied along dimension d, all 9 quantities (h = 1 on
         curvilinear elements, whose metric carries the scale) */
      for (int z = 0; z < N; ++z)
        for (int y = 0; y < N; ++y)
          for (int x = 0; x < N; ++x) {
            int i = (d == 0) ? x : (d == 1) ? y : z;
            for (int s = 0; s < M; ++s) {
              double acc = 0.0;
              for (int l = 0; l < N; ++l) {
                int zz = (d == 2) ? l : z, yy = (d == 1) ? l : y, xx = (d == 0) ? l : x;
                acc += D[i * N + l] * p[NODE(zz, yy, xx) * M + s];
              }
              g[NODE(z, y, x) * M + s] = acc / h;
            }
          }
      for (int n = 0; n < n3; ++n) {
        double B[M][M];
        if (metric) {
          /* reference direction d carries every physical direction j:
             Bt_d = sum_j G[d][j] B_j, G[d][j] = dxi_d/dx_j at this node */
          memset(B, 0, sizeof(double) * M * M);
          for (int j = 0; j < 3; ++j) {
            double Bj[M][M];
            elastic_B(j, params[n * 3 + 0], params[n * 3 + 1], params[n * 3 + 2], Bj);
            const double gdj = metric[n * 9 + 3 * d + j];
            for (int r = 0; r < M; ++r)
              for (int s = 0; s < M; ++s) B[r][s] += gdj * Bj[r][s];
          }
        } else {
          elastic_B(d, params[n * 3 + 0], params[n * 3 + 1], params[n * 3 + 2], B);
        }
        for (int r = 0; r < M; ++r) {
          double acc = 0.0;
          for (int s = 0; s < M; ++s) acc += B[r][s] * g[n * M + s];
          pn[n * M + r] -= acc;
        }
      }
    }
    memcpy(p, pn, sizeof(double) * n3 * M);
    /* point sources of this element: q^(k+1) = L q^(k) + s^(k) */
    if (src)
      for (int t = 0; t < n3 * M; ++t) p[t] += src[(size_t)k * n3 * M + t];
    c = c * dt / (double)(k + 2);
    for (int t = 0; t < n3 * M; ++t) avg[t] += c * p[t];
    if (terms) memcpy(terms + (size_t)(k + 1) * n3 * M, p, sizeof(double) * n3 * M);
  }
  /* faces: phi(side)^T applied along dimension d to avg */
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side) {
      const double* phi = side ? phi1 : phi0;
      double* f = faces + (size_t)(2 * d + side) * N * N * M;
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b)
          for (int s = 0; s < M; ++s) {
            double acc = 0.0;
            for (int i = 0; i < N; ++i) {
              int z, y, x;
              if (d == 0) { z = a; y = b; x = i; }
              else if (d == 1) { z = a; y = i; x = b; }
              else { z = i; y = a; x = b; }
              acc += phi[i] * avg[NODE(z, y, x) * M + s];
            }
            f[(a * N + b) * M + s] = acc;
          }
    }
}

/*
 * The STP over E independent elements. K = number of Taylor terms (N+1 by
 * default reading). Returns 0, -1 on bad arguments, -2 on allocation failure.
 * Elements are distributed over OpenMP threads when compiled with OpenMP;
 * each element's arithmetic is the same either way.
 */
int oracle_stp_nodes(int nodes, int N, int K, int64_t E, double h, double dt, const double* q,
                     const double* params, double* avg, double* faces, double* terms) {
  if (N < 1 || N > 16 || K < 1 || E < 0 || !(h > 0.0)) return -1;
  double D[16 * 16], phi0[16], phi1[16];
  if (oracle_tables_nodes(nodes, N, NULL, D, phi0, phi1) != 0) return -1;
  const size_t n3m = (size_t)N * N * N * M;
  int err = 0;
#pragma omp parallel
  {
    double* work = (double*)malloc(sizeof(double) * 3 * n3m);
    if (!work) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 4)
    for (int64_t e = 0; e < E; ++e) {
      if (!work) continue;
      stp_element(N, K, h, dt, D, phi0, phi1, q + e * n3m,
                  params + e * (n3m / M) * 3, NULL, NULL, avg + e * n3m,
                  faces + e * (size_t)6 * N * N * M,
                  terms ? terms + e * (size_t)K * n3m : NULL, work, work + n3m,
                  work + 2 * n3m);
    }
    free(work);
  }
  return err ? -2 : 0;
}

/*
 * The STP with point sources (the source term of the linear PDE, Sec. II-A,
 * whose time derivatives enter every CK order in the generic STP figure). A
 * source is a Dirac delta at reference position pos (in [0,1]^3) of element
 * elem, times a vector amp over the 9 quantities, times a time function whose
 * derivatives f^(k)(t_n), k = 0..K-2, are given in der[K-1]. Projected onto
 * the nodal basis with the diagonal (quadrature) mass matrix, it adds
 *   s^(k)_node = phi_node(pos) / (w_node h^3) * amp * f^(k)
 * to every CK term: q^(k+1) = L q^(k) + s^(k), node weight w_node the product
 * of the 1-D quadrature weights on [0,1], phi_node the product of the 1-D
 * Lagrange polynomials. Sources in one element add up. Arrays: elem[nsrc],
 * pos[nsrc][3] (x, y, z), amp[nsrc][9], der[nsrc][K-1].
 */
/* determinant of a 3x3 row-major matrix (rule of Sarrus) */
static double det3(const double* a) {
  return a[0] * a[4] * a[8] + a[1] * a[5] * a[6] + a[2] * a[3] * a[7] -
         a[2] * a[4] * a[6] - a[0] * a[5] * a[7] - a[1] * a[3] * a[8];
}

/* Point sources on cubes of side h (metric NULL) or on curvilinear elements
 * (metric as in oracle_stp_curvilinear; h unused). The node's volume in the
 * diagonal mass matrix is w_node h^3 on a cube and w_node |det J_node| on a
 * curvilinear element, J = dx/dxi = G^-1, so |det J| = 1 / |det G|. */
static int stp_sources(int nodes, int N, int K, int64_t E, double h, double dt, const double* q,
                       const double* params, const double* metric, int nsrc, const int64_t* elem,
                       const double* pos, const double* amp, const double* der, double* avg,
                       double* faces, double* terms) {
  if (N < 1 || N > 16 || K < 1 || E < 0 || (!metric && !(h > 0.0)) || nsrc < 0) return -1;
  double xi[16], w[16], D[16 * 16], phi0[16], phi1[16];
  if (oracle_tables_nodes(nodes, N, xi, D, phi0, phi1) != 0) return -1;
  if ((nodes == 0 ? oracle_gl_nodes(N, xi, w) : oracle_gll_nodes(N, xi, w)) != 0) return -1;
  const size_t n3 = (size_t)N * N * N, n3m = n3 * M;
  /* elements with sources, their projected source terms [K-1][N^3][9] */
  double** src = (double**)calloc((size_t)(E > 0 ? E : 1), sizeof(double*));
  if (!src) return -2;
  int err = 0;
  for (int i = 0; i < nsrc && !err; ++i) {
    const int64_t e = elem[i];
    if (e < 0 || e >= E) { err = -1; break; }
    if (!src[e] && !(src[e] = (double*)calloc((size_t)(K > 1 ? K - 1 : 1) * n3m, sizeof(double)))) {
      err = -2;
      break;
    }
    for (int z = 0; z < N; ++z)
      for (int y = 0; y < N; ++y)
        for (int x = 0; x < N; ++x) {
          const double vol = metric ? 1.0 / fabs(det3(metric + ((size_t)e * n3 + NODE(z, y, x)) * 9))
                                    : h * h * h;
          const double proj = lagrange(N, xi, x, pos[3 * i]) * lagrange(N, xi, y, pos[3 * i + 1]) *
                               lagrange(N, xi, z, pos[3 * i + 2]) / (w[x] * w[y] * w[z] * vol);
          for (int k = 0; k + 1 < K; ++k)
            for (int s = 0; s < M; ++s)
              src[e][(size_t)k * n3m + (size_t)NODE(z, y, x) * M + s] +=
                  proj * amp[9 * i + s] * der[(size_t)i * (K - 1) + k];
        }
  }
  if (!err) {
#pragma omp parallel
    {
      double* work = (double*)malloc(sizeof(double) * 3 * n3m);
      if (!work) {
#pragma omp atomic write
        err = -2;
      }
#pragma omp for schedule(dynamic, 4)
      for (int64_t e = 0; e < E; ++e) {
        if (!work) continue;
        stp_element(N, K, metric ? 1.0 : h, dt, D, phi0, phi1, q + e * n3m, params + e * n3 * 3,
                    metric ? metric + e * n3 * 9 : NULL, src[e], avg + e * n3m,
                    faces + e * (size_t)6 * N * N * M,
                    terms ? terms + e * (size_t)K * n3m : NULL, work, work + n3m, work + 2 * n3m);
      }
      free(work);
    }
  }
  for (int64_t e = 0; e < E; ++e) free(src[e]);
  free(src);
  return err;
}

int oracle_stp_sources(int nodes, int N, int K, int64_t E, double h, double dt, const double* q,
                       const double* params, int nsrc, const int64_t* elem, const double* pos,
                       const double* amp, const double* der, double* avg, double* faces,
                       double* terms) {
  return stp_sources(nodes, N, K, E, h, dt, q, params, NULL, nsrc, elem, pos, amp, der, avg, faces,
                     terms);
}

/* Point sources on curvilinear elements (see stp_sources and
 * oracle_stp_curvilinear). */
int oracle_stp_sources_curvilinear(int nodes, int N, int K, int64_t E, double dt, const double* q,
                                   const double* params, const double* metric, int nsrc,
                                   const int64_t* elem, const double* pos, const double* amp,
                                   const double* der, double* avg, double* faces, double* terms) {
  if (!metric) return -1;
  return stp_sources(nodes, N, K, E, 1.0, dt, q, params, metric, nsrc, elem, pos, amp, der, avg,
                     faces, terms);
}

/*
 * The STP on curvilinear elements. The paper's benchmark runs on curvilinear
 * boundary-fitted meshes and stores 9 geometry parameters at every node beside
 * the 3 material parameters (Sec. VI). Read here as the inverse Jacobian of
 * the element map from the reference cube [0,1]^3 to physical space:
 * metric[E][N][N][N][9] holds G[d][j] = dxi_d/dx_j at index 3d + j, where
 * xi_1, xi_2, xi_3 run along the element's x, y, z node indices. The chain
 * rule d/dx_j = sum_d G[d][j] d/dxi_d turns one CK step into
 *   q^(k+1) = - sum_d (sum_j G[d][j] B_j) (D_d q^(k)),
 * D applied along reference direction d with no 1/h (G carries the scale). A
 * cube of side h has G = I/h and gives the Cartesian result. Faces are the
 * reference faces xi_d = 0, 1.
 */
int oracle_stp_curvilinear(int nodes, int N, int K, int64_t E, double dt, const double* q,
                           const double* params, const double* metric, double* avg,
                           double* faces, double* terms) {
  if (N < 1 || N > 16 || K < 1 || E < 0 || !metric) return -1;
  double D[16 * 16], phi0[16], phi1[16];
  if (oracle_tables_nodes(nodes, N, NULL, D, phi0, phi1) != 0) return -1;
  const size_t n3 = (size_t)N * N * N, n3m = n3 * M;
  int err = 0;
#pragma omp parallel
  {
    double* work = (double*)malloc(sizeof(double) * 3 * n3m);
    if (!work) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 4)
    for (int64_t e = 0; e < E; ++e) {
      if (!work) continue;
      stp_element(N, K, 1.0, dt, D, phi0, phi1, q + e * n3m, params + e * n3 * 3,
                  metric + e * n3 * 9, NULL, avg + e * n3m, faces + e * (size_t)6 * N * N * M,
                  terms ? terms + e * (size_t)K * n3m : NULL, work, work + n3m, work + 2 * n3m);
    }
    free(work);
  }
  return err ? -2 : 0;
}

/* The STP on Gauss-Legendre nodes (the default node family). */
int oracle_stp(int N, int K, int64_t E, double h, double dt, const double* q,
               const double* params, double* avg, double* faces, double* terms) {
  return oracle_stp_nodes(0, N, K, E, h, dt, q, params, avg, faces, terms);
}

/* number of OpenMP threads the oracle runs on (1 without OpenMP) */
int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
