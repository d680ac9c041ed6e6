/*
 * Plain FP64 CPU oracle of the corrector of the linear ADER-DG scheme.
 *
 * TEST INFRASTRUCTURE ONLY, like stp_oracle.c (compiled into the same
 * library): only the tests, the smoke check and the benchmark's CPU baseline
 * use it, and it shares nothing with the CUDA library.
 *
 * What it computes (Gallard et al., arXiv 2003.12787, Sec. II-A): the
 * corrector step that follows the predictor,
 *   q(t_{n+1}) = q(t_n) + V qbar + sum over the element's faces of the
 *                numerical flux of the time-integrated face values,
 * which the paper writes for a flux that is linear in its arguments, so that
 * it acts on the predictor's time-integrated face projections directly. Here
 * qbar = dt * avg (the predictor outputs the time average avg).
 *
 * Readings (the paper leaves the flux and the mesh open):
 *   - Strong nodal DG form (the paper integrates the flux terms by parts twice)
 *     on the same nodes as the predictor, with the diagonal mass matrix of the
 *     nodal quadrature (weights w on [0,1], node volume w_x w_y w_z h^3). The
 *     semi-discrete update of node (i along d, a, b) is
 *       dq/dt = - sum_d B_d (D_d q) / h
 *               - sum_{faces f=(d,side)} phi_i(side) / (w_i h) * F_f[a][b]
 *     where F_f is the numerical fluctuation on face f.
 *   - Fluctuation: the Rusanov (local Lax-Friedrichs) form for a linear
 *     non-conservative system, F = 1/2 (Bn - s I)(q+ - q-), with q- the
 *     element's own face value, q+ the neighbour's on the same face, n the
 *     outward normal (Bn = +B_d on the side-1 face, -B_d on the side-0 face),
 *     Bn the mean of the two sides' matrices and s = max(|cp-|, |cp+|).
 *   - Material on a face: the face projection phi(side)^T of the per-node
 *     material (rho, cp, cs) of each side. In the paper's code the material
 *     parameters are stored inside q and projected to the faces with the
 *     state; the material itself does not evolve and receives no flux.
 *   - Mesh: a structured grid of gx * gy * gz cubes of side h, periodic in all
 *     three directions; element e = (ez * gy + ey) * gx + ex. Face f = 2d +
 *     side of element e meets face 2d + (1 - side) of its neighbour, with the
 *     same in-plane indices (x-faces [z][y], y-faces [z][x], z-faces [y][x]).
 *   - By linearity the time integral of the semi-discrete update is the same
 *     update applied to the predictor's outputs:
 *       q_out = q + dt * ( -sum_d B_d (D_d avg) / h - lift(F(faces)) ).
 *
 * Layouts as in stp_oracle.c; face_params: [E][6][N][N][3].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define M 9

int oracle_gl_nodes(int N, double* xi, double* w);
int oracle_gll_nodes(int N, double* xi, double* w);
int oracle_tables_nodes(int nodes, int N, double* xi_out, double* D, double* phi0, double* phi1);
void oracle_elastic_B(int d, double rho, double cp, double cs, double* B);

/* node (z,y,x) of element-local index */
static int node_index(int N, int z, int y, int x) { return (z * N + y) * N + x; }

/* the node at position i along direction d on the line through the face
   point (a,b) of a d-face */
static int line_node(int N, int d, int a, int b, int i) {
  if (d == 0) return node_index(N, a, b, i); /* x-faces: (a,b) = (z,y) */
  if (d == 1) return node_index(N, a, i, b); /* y-faces: (a,b) = (z,x) */
  return node_index(N, i, a, b);             /* z-faces: (a,b) = (y,x) */
}

/* periodic neighbour of element e one cell along direction d (step +1 or -1) */
static int64_t neighbour(int gx, int gy, int gz, int64_t e, int d, int step) {
  int64_t ex = e % gx, ey = (e / gx) % gy, ez = e / ((int64_t)gx * gy);
  if (d == 0) ex = (ex + step + gx) % gx;
  if (d == 1) ey = (ey + step + gy) % gy;
  if (d == 2) ez = (ez + step + gz) % gz;
  return (ez * gy + ey) * gx + ex;
}

static int node_weights(int nodes, int N, double* w) {
  double xi[64];
  if (nodes == 0) return oracle_gl_nodes(N, xi, w);
  if (nodes == 1) return oracle_gll_nodes(N, xi, w);
  return -1;
}

/* Face projection of the material: out[e][2d+side][a][b][c] =
   sum_i phi_i(side) params[e][line node i][c]. Returns 0 or -1. */
int oracle_face_params(int nodes, int N, int64_t E, const double* params, double* out) {
  if (N < 1 || N > 16 || E < 0) return -1;
  double phi0[16], phi1[16];
  if (oracle_tables_nodes(nodes, N, NULL, NULL, phi0, phi1) != 0) return -1;
  const size_t n3 = (size_t)N * N * N;
  for (int64_t e = 0; e < E; ++e)
    for (int d = 0; d < 3; ++d)
      for (int side = 0; side < 2; ++side) {
        const double* phi = side ? phi1 : phi0;
        for (int a = 0; a < N; ++a)
          for (int b = 0; b < N; ++b)
            for (int c = 0; c < 3; ++c) {
              double acc = 0.0;
              for (int i = 0; i < N; ++i)
                acc += phi[i] * params[((size_t)e * n3 + line_node(N, d, a, b, i)) * 3 + c];
              out[((((size_t)e * 6 + 2 * d + side) * N + a) * N + b) * 3 + c] = acc;
            }
      }
  return 0;
}

/*
 * One corrector step on the periodic grid. q, avg: [E][N][N][N][9];
 * params: [E][N][N][N][3]; faces: [E][6][N][N][9] (the predictor's face
 * projections of avg); q_out: [E][N][N][N][9] (may not alias the inputs).
 * Returns 0, -1 on bad arguments, -2 on allocation failure.
 */
int oracle_correct(int nodes, int N, int gx, int gy, int gz, double h, double dt, const double* q,
                   const double* params, const double* avg, const double* faces, double* q_out) {
  if (N < 1 || N > 16 || gx < 1 || gy < 1 || gz < 1 || !(h > 0.0)) return -1;
  double D[16 * 16], phi0[16], phi1[16], w[16];
  if (oracle_tables_nodes(nodes, N, NULL, D, phi0, phi1) != 0) return -1;
  if (node_weights(nodes, N, w) != 0) return -1;
  const int64_t E = (int64_t)gx * gy * gz;
  const size_t n3 = (size_t)N * N * N, n3m = n3 * M, n2 = (size_t)N * N;
  double* fp = (double*)malloc(sizeof(double) * (size_t)E * 6 * n2 * 3);
  double* rate = (double*)malloc(sizeof(double) * n3m);
  if (!fp || !rate) {
    free(fp);
    free(rate);
    return -2;
  }
  oracle_face_params(nodes, N, E, params, fp);
  for (int64_t e = 0; e < E; ++e) {
    const double* qa = avg + e * n3m;
    const double* pe = params + e * n3 * 3;
    /* volume term: rate = - sum_d B_d (D_d avg) / h, every quantity, dense B */
    memset(rate, 0, sizeof(double) * n3m);
    for (int d = 0; d < 3; ++d)
      for (int z = 0; z < N; ++z)
        for (int y = 0; y < N; ++y)
          for (int x = 0; x < N; ++x) {
            const int n = node_index(N, z, y, x);
            const int i = (d == 0) ? x : (d == 1) ? y : z;
            double g[M];
            for (int s = 0; s < M; ++s) {
              double acc = 0.0;
              for (int l = 0; l < N; ++l) {
                const int zz = (d == 2) ? l : z, yy = (d == 1) ? l : y, xx = (d == 0) ? l : x;
                acc += D[i * N + l] * qa[(size_t)node_index(N, zz, yy, xx) * M + s];
              }
              g[s] = acc / h;
            }
            double B[M * M];
            oracle_elastic_B(d, pe[n * 3 + 0], pe[n * 3 + 1], pe[n * 3 + 2], B);
            for (int r = 0; r < M; ++r) {
              double acc = 0.0;
              for (int s = 0; s < M; ++s) acc += B[r * M + s] * g[s];
              rate[(size_t)n * M + r] -= acc;
            }
          }
    /* face terms: Rusanov fluctuation of the time-averaged face values */
    for (int d = 0; d < 3; ++d)
      for (int side = 0; side < 2; ++side) {
        const int f = 2 * d + side, fo = 2 * d + (1 - side);
        const int64_t en = neighbour(gx, gy, gz, e, d, side ? 1 : -1);
        const double sign = side ? 1.0 : -1.0; /* outward normal along d */
        const double* phi = side ? phi1 : phi0;
        for (int a = 0; a < N; ++a)
          for (int b = 0; b < N; ++b) {
            const double* qm = faces + (((size_t)e * 6 + f) * n2 + (size_t)a * N + b) * M;
            const double* qp = faces + (((size_t)en * 6 + fo) * n2 + (size_t)a * N + b) * M;
            const double* mm = fp + (((size_t)e * 6 + f) * n2 + (size_t)a * N + b) * 3;
            const double* mp = fp + (((size_t)en * 6 + fo) * n2 + (size_t)a * N + b) * 3;
            double Bm[M * M], Bp[M * M];
            oracle_elastic_B(d, mm[0], mm[1], mm[2], Bm);
            oracle_elastic_B(d, mp[0], mp[1], mp[2], Bp);
            const double smax = fmax(fabs(mm[1]), fabs(mp[1]));
            double F[M];
            for (int r = 0; r < M; ++r) {
              double acc = 0.0;
              for (int s = 0; s < M; ++s) {
                const double bn = sign * 0.5 * (Bm[r * M + s] + Bp[r * M + s]);
                acc += (bn - (r == s ? smax : 0.0)) * (qp[s] - qm[s]);
              }
              F[r] = 0.5 * acc;
            }
            for (int i = 0; i < N; ++i) {
              const int n = line_node(N, d, a, b, i);
              const double lift = phi[i] / (w[i] * h);
              for (int r = 0; r < M; ++r) rate[(size_t)n * M + r] -= lift * F[r];
            }
          }
      }
    for (size_t t = 0; t < n3m; ++t) q_out[e * n3m + t] = q[e * n3m + t] + dt * rate[t];
  }
  free(fp);
  free(rate);
  return 0;
}
