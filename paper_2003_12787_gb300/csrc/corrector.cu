// Corrector of the linear ADER-DG scheme in FP64 (Sec. II-A): the step that
// turns the predictor's time-averaged state and face projections into the
// state at t_{n+1},
//   q(t_{n+1}) = q(t_n) + V qbar + sum over faces of the numerical flux of
//                the time-integrated face values,
// on a structured grid of gx * gy * gz cubes of side dx, periodic in every
// direction (element e = (ez * gy + ey) * gx + ex).
//
// Strong nodal DG form on the predictor's nodes with the diagonal mass matrix
// of the nodal quadrature. With the predictor's average avg (qbar = dt avg)
// and its face projections, node (i along d, a, b) of an element gets
//   q_out = q + dt ( A.(D avg)/dx  -  sum_faces phi_i(side)/(w_i dx) F_f[a][b] )
// where A.(D avg) is the elastic update of the Cauchy-Kowalewsky step (the
// same node code as the predictor) and F_f the Rusanov fluctuation of face f,
//   F = 1/2 (Bn (q+ - q-) - s (q+ - q-)),  Bn = +-1/2 (B(m-) + B(m+)),
// q- the element's own face value, q+ the neighbour's on the same face, the
// sign that of the outward normal along d, m-/m+ the two sides' face
// projections of the material (rho, cp, cs) and s = max(|cp-|, |cp+|).
//
// One CTA per element: the average goes to shared memory (AoS -> SoA), the
// 6 N^2 face fluctuations are formed from the face arrays of the element and
// its six neighbours (coalesced 72-byte node records) into shared memory,
// then every thread forms the update of its nodes and the result is written
// back coalesced as q + update (q_out may be q itself).
#include <algorithm>

#include "ck_fp64.cuh"
#include "stp_internal.h"

namespace stp {
namespace {

// Lift coefficients phi_i(side) / w_i * dt / dx and the derivative scale.
struct CorrectorCoef {
  double c0[kMaxNodes];
  double c1[kMaxNodes];
  double dscale;  // dt / dx
};

template <int N>
struct CorrShape {
  static constexpr int N3 = N * N * N;
  static constexpr int S = N3 | 1;   // odd stride between quantities
  static constexpr int LDD = N | 1;  // odd row stride of D
  static constexpr int NODES = (N3 + 511) / 512;  // nodes per thread
  static constexpr int NT = ((N3 + NODES - 1) / NODES + 31) / 32 * 32;
  static constexpr int F = 6 * N * N * kQuantities;
  static constexpr size_t SMEM = sizeof(double) * (size_t)(N * LDD + 2 * N + kQuantities * S + F);
};

// out = A_d j for direction d with the elastic coefficients (1/rho, lambda,
// mu) of q_t = sum_d A_d dq/dx_d: v_i <- (1/rho) j[s_{i d}], s_ii <- lambda
// j[v_d] (+ 2 mu j[v_d] for i = d), s_ij <- mu (delta_jd j[v_i] + delta_id j[v_j]).
__device__ __forceinline__ void apply_A(int d, double invrho, double lam, double mu,
                                        const double j[9], double out[9]) {
  const double vd = j[d];
  if (d == 0) {
    out[kV1] = invrho * j[kS11];
    out[kV2] = invrho * j[kS12];
    out[kV3] = invrho * j[kS13];
    out[kS11] = fma(2.0 * mu, vd, lam * vd);
    out[kS22] = lam * vd;
    out[kS33] = lam * vd;
    out[kS12] = mu * j[kV2];
    out[kS13] = mu * j[kV3];
    out[kS23] = 0.0;
  } else if (d == 1) {
    out[kV1] = invrho * j[kS12];
    out[kV2] = invrho * j[kS22];
    out[kV3] = invrho * j[kS23];
    out[kS11] = lam * vd;
    out[kS22] = fma(2.0 * mu, vd, lam * vd);
    out[kS33] = lam * vd;
    out[kS12] = mu * j[kV1];
    out[kS13] = 0.0;
    out[kS23] = mu * j[kV3];
  } else {
    out[kV1] = invrho * j[kS13];
    out[kV2] = invrho * j[kS23];
    out[kV3] = invrho * j[kS33];
    out[kS11] = lam * vd;
    out[kS22] = lam * vd;
    out[kS33] = fma(2.0 * mu, vd, lam * vd);
    out[kS12] = 0.0;
    out[kS13] = mu * j[kV1];
    out[kS23] = mu * j[kV2];
  }
}

template <int N>
__global__ void __launch_bounds__(CorrShape<N>::NT)
corrector_kernel(const __grid_constant__ CorrectorCoef cc, int gx, int gy, int gz,
                 const double* __restrict__ tables, const double* q,
                 const double* __restrict__ params, const double* __restrict__ face_params,
                 const double* __restrict__ avg, const double* __restrict__ faces,
                 double* q_out) {
  using Sh = CorrShape<N>;
  constexpr int N3 = Sh::N3, S = Sh::S, LDD = Sh::LDD, NODES = Sh::NODES, NT = Sh::NT;
  constexpr int M = kQuantities, N2 = N * N;
  extern __shared__ double smem[];
  double* sD = smem;              // D * dt/dx, [N][LDD]
  double* sC = sD + N * LDD;      // c0[N], c1[N]
  double* sP = sC + 2 * N;        // avg, [9][S]; the update at the end
  double* sF = sP + M * S;        // fluctuations [6][N][N][9]
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  const int64_t gxy = (int64_t)gx * gy;
  const int ex = (int)(e % gx), ey = (int)((e / gx) % gy), ez = (int)(e / gxy);

  const double* Dref = tables + (N * N * N + 2 * N);  // the unscaled D after the step tables and phi
  for (int i = tid; i < N * N; i += NT) sD[(i / N) * LDD + i % N] = Dref[i] * cc.dscale;
  for (int i = tid; i < N; i += NT) {
    sC[i] = cc.c0[i];
    sC[N + i] = cc.c1[i];
  }
  const double* ae = avg + e * (int64_t)(M * N3);
  for (int f = tid; f < M * N3; f += NT) {  // coalesced AoS read, SoA scatter
    const int n = f / M, s = f - n * M;
    sP[s * S + n] = __ldg(ae + f);
  }
  // face fluctuations
  for (int t = tid; t < 6 * N2; t += NT) {
    const int f = t / N2, ab = t - f * N2, d = f >> 1, side = f & 1;
    int c[3] = {ex, ey, ez};
    const int g[3] = {gx, gy, gz};
    c[d] += side ? 1 : -1;
    if (c[d] < 0) c[d] += g[d];
    if (c[d] >= g[d]) c[d] -= g[d];
    const int64_t en = ((int64_t)c[2] * gy + c[1]) * gx + c[0];
    const int fo = f ^ 1;  // the neighbour's face on the other side
    const double* qm = faces + ((e * 6 + f) * N2 + ab) * M;
    const double* qp = faces + ((en * 6 + fo) * N2 + ab) * M;
    const double* mm = face_params + ((e * 6 + f) * N2 + ab) * 3;
    const double* mp = face_params + ((en * 6 + fo) * N2 + ab) * 3;
    double jmp[9];
#pragma unroll
    for (int s = 0; s < M; ++s) jmp[s] = __ldg(qp + s) - __ldg(qm + s);
    double ir0, l0, m0, m20, ir1, l1, m1, m21;
    const double rho0 = __ldg(mm), cp0 = __ldg(mm + 1), rho1 = __ldg(mp), cp1 = __ldg(mp + 1);
    elastic_coefficients(rho0, cp0, __ldg(mm + 2), &ir0, &l0, &m0, &m20);
    elastic_coefficients(rho1, cp1, __ldg(mp + 2), &ir1, &l1, &m1, &m21);
    double aj[9];
    apply_A(d, 0.5 * (ir0 + ir1), 0.5 * (l0 + l1), 0.5 * (m0 + m1), jmp, aj);
    const double smax = fmax(fabs(cp0), fabs(cp1));
    // Bn = -sign * mean(A); F = 1/2 (Bn j - s j)
    const double sg = side ? -1.0 : 1.0;
#pragma unroll
    for (int s = 0; s < M; ++s) sF[t * M + s] = 0.5 * fma(sg, aj[s], -smax * jmp[s]);
  }
  double cf[NODES][4];
  const double* pe = params + e * (int64_t)(kParams * N3);
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * NT;
    if (n < N3)
      elastic_coefficients(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2),
                           &cf[j][0], &cf[j][1], &cf[j][2], &cf[j][3]);
  }
  __syncthreads();

  double r[NODES][9];
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * NT;
    if (n >= N3) continue;
    const int x = n % N, y = (n / N) % N, z = n / N2;
    ck_node_fp64<N, S, LDD>(sP, sD, x, y, z, cf[j][0], cf[j][1], cf[j][2], cf[j][3], r[j]);
    const double* Fx0 = sF + (0 * N2 + z * N + y) * M;
    const double* Fx1 = sF + (1 * N2 + z * N + y) * M;
    const double* Fy0 = sF + (2 * N2 + z * N + x) * M;
    const double* Fy1 = sF + (3 * N2 + z * N + x) * M;
    const double* Fz0 = sF + (4 * N2 + y * N + x) * M;
    const double* Fz1 = sF + (5 * N2 + y * N + x) * M;
    const double ax0 = sC[x], ax1 = sC[N + x], ay0 = sC[y], ay1 = sC[N + y];
    const double az0 = sC[z], az1 = sC[N + z];
#pragma unroll
    for (int s = 0; s < M; ++s) {
      double l = ax0 * Fx0[s];
      l = fma(ax1, Fx1[s], l);
      l = fma(ay0, Fy0[s], l);
      l = fma(ay1, Fy1[s], l);
      l = fma(az0, Fz0[s], l);
      l = fma(az1, Fz1[s], l);
      r[j][s] -= l;
    }
  }
  __syncthreads();  // every read of the average is done
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * NT;
    if (n >= N3) continue;
#pragma unroll
    for (int s = 0; s < M; ++s) sP[s * S + n] = r[j][s];
  }
  __syncthreads();
  const double* qe = q + e * (int64_t)(M * N3);
  double* oe = q_out + e * (int64_t)(M * N3);
  for (int f = tid; f < M * N3; f += NT) {
    const int n = f / M, s = f - n * M;
    oe[f] = qe[f] + sP[s * S + n];
  }
}

template <int N>
cudaError_t launch_corrector_n(const CorrectorCoef& cc, int gx, int gy, int gz,
                               const double* tables, const double* q, const double* params,
                               const double* face_params, const double* avg, const double* faces,
                               double* q_out, cudaStream_t stream) {
  using Sh = CorrShape<N>;
  cudaError_t e = cudaFuncSetAttribute(corrector_kernel<N>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
  if (e != cudaSuccess) return e;
  const int64_t E = (int64_t)gx * gy * gz;
  corrector_kernel<N><<<(unsigned)E, Sh::NT, Sh::SMEM, stream>>>(cc, gx, gy, gz, tables, q, params,
                                                                  face_params, avg, faces, q_out);
  return cudaGetLastError();
}

// Face projection of the material: out[e][f][a][b][c] = sum_i phi_i(side)
// params[e][line node i][c], one thread per output value.
template <int N>
__global__ void face_params_kernel(int64_t E, const double* __restrict__ tables,
                                   const double* __restrict__ params, double* __restrict__ out) {
  constexpr int N2 = N * N, N3 = N * N * N;
  const int64_t total = E * 6 * N2 * 3;
  const double* phi0 = tables + N3;
  const double* phi1 = phi0 + N;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(o % 3);
    int64_t rest = o / 3;
    const int b = (int)(rest % N);
    rest /= N;
    const int a = (int)(rest % N);
    rest /= N;
    const int f = (int)(rest % 6);
    const int64_t e = rest / 6;
    const int d = f >> 1;
    const double* phi = (f & 1) ? phi1 : phi0;
    int base, stride;
    if (d == 0) { base = (a * N + b) * N; stride = 1; }  // x-faces [z][y]
    else if (d == 1) { base = a * N2 + b; stride = N; }  // y-faces [z][x]
    else { base = a * N + b; stride = N2; }              // z-faces [y][x]
    const double* pe = params + e * (int64_t)(3 * N3);
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) acc = fma(phi[i], __ldg(pe + (base + i * stride) * 3 + c), acc);
    out[o] = acc;
  }
}

}  // namespace

cudaError_t launch_corrector(int N, int gx, int gy, int gz, const HostTables& t, double dx,
                             double dt, const double* tables, const double* q,
                             const double* params, const double* face_params, const double* avg,
                             const double* faces, double* q_out, cudaStream_t stream) {
  CorrectorCoef cc{};
  cc.dscale = dt / dx;
  for (int i = 0; i < N; ++i) {
    cc.c0[i] = t.phi0[i] / t.weights[i] * (dt / dx);
    cc.c1[i] = t.phi1[i] / t.weights[i] * (dt / dx);
  }
  switch (N) {
#define CASE(n) \
  case n: return launch_corrector_n<n>(cc, gx, gy, gz, tables, q, params, face_params, avg, faces, q_out, stream);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
    CASE(12)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_face_params(int N, int64_t E, const double* tables, const double* params,
                               double* out, cudaStream_t stream) {
  const int64_t total = E * 6 * (int64_t)N * N * 3;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 152 * 16);
  switch (N) {
#define CASE(n) \
  case n: face_params_kernel<n><<<(unsigned)blocks, threads, 0, stream>>>(E, tables, params, out); break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11)
    CASE(12)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace stp
