// FP64 Space-Time Predictor on one curvilinear element (device code shared
// by the curvilinear kernel and the batched persistent kernel).
//
// The paper's benchmark runs the elastic wave equation on curvilinear,
// boundary-fitted meshes and stores 9 geometry parameters at every node beside
// the 3 material parameters (Sec. VI). Here they are the inverse Jacobian
// G[d][j] = dxi_d/dx_j of the element's map from the unit reference cube
// (xi_1, xi_2, xi_3 along the x, y, z node indices) to physical space, so the
// physical derivative is d/dx_j = sum_d G[d][j] d/dxi_d and one
// Cauchy-Kowalewsky step reads
//   q^(k+1) = sum_j A_j dq^(k)/dx_j = sum_d (sum_j G[d][j] A_j) (D_d q^(k)),
// the Cartesian step with every reference direction coupling all three
// physical ones (a cube of side h has G = I/h).
//
// The elastic sparsity of the Cartesian kernels (6 of 9 quantities per
// direction) is lost: every quantity is differentiated along every reference
// direction, 27 line derivatives per node and step instead of 18. Per
// direction, a line pass writes the reference derivatives of the 9 quantities
// (at N = 12: 5, then 4, to fit shared memory) with the even-odd contraction of
// the Cartesian kernels; a pointwise pass multiplies them by the node's metric
// row (G[d][0..2], read through L1) and adds them into nine per-node partial
// sums kept in registers,
//   div_i = sum_j dsigma_ij/dx_j,  dv_i/dx_i,  dv_i/dx_j + dv_j/dx_i (i < j),
// from which the last pass of the step forms r_{k+1} with the node's elastic
// coefficients. Taylor bookkeeping as in the Cartesian kernels: the step
// tables hold D dt/((k+2) dx), so the coefficients are multiplied by dx once.
#pragma once
#include <type_traits>

#include "ck_curv.cuh"
#include "stp_internal.h"

namespace stp {

template <int N, int A, bool DB>
struct CurvShape {
  static constexpr int N3 = N * N * N;
  static constexpr int RX = N | 1;  // x rows padded to an odd length
  static constexpr int PLANE = N * RX;
  static constexpr int S = (N * PLANE) | 1;
  static constexpr int H = N / 2;
  static constexpr bool ODD = (N & 1) != 0;
  // per step: E[H][H], O[H][H], middle column (odd N), middle row odd part (odd N)
  static constexpr int STEP_TABLE = 2 * H * H + (ODD ? 2 * H : 0);
  static constexpr int TABLE = N * STEP_TABLE + 2 * N;
  static constexpr int SUBS = (kQuantities + A - 1) / A;  // line passes per direction
  static constexpr size_t SMEM =
      sizeof(double) * (size_t)(TABLE + (kQuantities + (DB ? 2 : 1) * A) * S);
};

// Launch shapes of the curvilinear kernels per N (its own kernel and the
// batched plan's): threads, nodes per thread, quantities per line pass,
// lean register state, metric in registers, double buffer (measured on GB300 among 2-6
// candidates per N; from N = 7 on, enough threads that the 9 N^2 line tasks of
// a pass take one or two even rounds).
#define STP_CURV_SHAPES(X)                                                                     \
  X(1, 32, 1, 9, false, false, false) X(2, 32, 1, 9, false, false, false)                       \
  X(3, 32, 1, 9, false, false, false) X(4, 64, 1, 9, false, false, false)                       \
  X(5, 128, 1, 9, false, false, false) X(6, 224, 1, 9, false, false, false)                     \
  X(7, 448, 1, 9, false, true, true) X(8, 576, 1, 9, false, false, true)                        \
  X(9, 384, 2, 9, false, true, true) X(10, 512, 2, 9, true, true, false)                        \
  X(11, 448, 3, 9, true, false, false) X(12, 448, 4, 5, true, false, false)

// Curvilinear element shapes in the allocation-free kernel's 512-thread CTAs:
// (N, nodes per thread, quantities per line pass, lean register state). The
// quantities per pass follow the curvilinear kernel's own shapes; as the
// arithmetic does not depend on the thread layout, a set gives the same bits
// in a persistent launch as alone.
#define STP_CURV512_SHAPES(X)                                                                  \
  X(1, 1, 9, false) X(2, 1, 9, false) X(3, 1, 9, false) X(4, 1, 9, false) X(5, 1, 9, false)    \
  X(6, 1, 9, false) X(7, 1, 9, false) X(8, 1, 9, false) X(9, 2, 9, false) X(10, 2, 9, true)    \
  X(11, 3, 9, true) X(12, 4, 5, true)

// One element (index e, by a CTA of NT threads; the caller guarantees
// e < E); thread t owns nodes t, t + NT, ...
// (NODES of them). LEAN keeps only the partial sums in registers: the running
// average accumulates in the output buffer and the coefficients are derived
// from params at every step (large N, where registers are short). GREG keeps
// the owned nodes' metric in registers instead of reading it through L1. DB
// double-buffers the reference derivatives (A = 9 only).
template <int N, int NT, int NODES, int A, bool LEAN, bool GREG, bool DB>
__device__ __forceinline__ void curv_element(double* smem, const double* __restrict__ q,
                                             const double* __restrict__ params,
                                             const double* __restrict__ metric,
                                             double* __restrict__ out_avg,
                                             double* __restrict__ out_faces,
                                             const double* __restrict__ tables, double dx,
                                             int64_t e) {
  using Sh = CurvShape<N, A, DB>;
  constexpr int N3 = Sh::N3, S = Sh::S, H = Sh::H, M = kQuantities;
  constexpr int RX = Sh::RX, PLANE = Sh::PLANE, SUBS = Sh::SUBS;
  constexpr bool ODD = Sh::ODD;
  constexpr int mid = H;
  static_assert(NODES * NT >= N3, "every node needs an owner");
  static_assert(SUBS <= 2 && (!DB || SUBS == 1), "one or two line passes per direction");
  auto pad = [](int n) { return (n / (N * N)) * PLANE + ((n / N) % N) * RX + n % N; };
  double* sT = smem;                       // [N steps][STEP_TABLE]
  double* sPhi = sT + N * Sh::STEP_TABLE;  // phi0[N], phi1[N]
  double* sp = sPhi + 2 * N;               // current term r_k [9][S]; the average at the end
  double* sacc = sp + M * S;               // reference derivatives of a pass [DB ? 2 : 1][A][S]
  const int tid = threadIdx.x;
  double* gavg = out_avg + e * (int64_t)(M * N3);
  const double* ge = metric + e * (int64_t)(9 * N3);
  const double* pe = params + e * (int64_t)(kParams * N3);

  // even/odd tables of every step from the scaled D_k (tables[k*N*N + i*N + l])
  if constexpr (H > 0)
  for (int idx = tid; idx < N * Sh::STEP_TABLE; idx += NT) {
    const int k = idx / Sh::STEP_TABLE, r = idx - k * Sh::STEP_TABLE;
    const double* Dk = tables + k * N * N;
    double v;
    if (r < 2 * H * H) {
      const int which = r / (H * H), i = (r / H) % H, l = r % H;
      const double a = Dk[i * N + l], b = Dk[i * N + (N - 1 - l)];
      v = which == 0 ? 0.5 * (a + b) : 0.5 * (a - b);
    } else {
      const int rr = r - 2 * H * H;  // odd N only
      if (rr < H) v = Dk[rr * N + mid];
      else {
        const int l = rr - H;
        v = 0.5 * (Dk[mid * N + l] - Dk[mid * N + (N - 1 - l)]);
      }
    }
    sT[idx] = v;
  }
  for (int i = tid; i < 2 * N; i += NT) sPhi[i] = tables[N * N * N + i];

  const double* qe = q + e * (int64_t)(M * N3);
  for (int f = tid; f < M * N3; f += NT) {  // coalesced AoS read, SoA scatter
    const int n = f / M, s = f - n * M;
    const double v = __ldg(qe + f);
    sp[s * S + pad(n)] = v;
    if constexpr (LEAN) gavg[f] = v;  // the average starts at r_0 = q
  }
  constexpr int KEEP = LEAN ? 1 : NODES;  // nodes whose coefficients and average stay in registers
  double cf[KEEP][4];
  double avg[KEEP][M];
  double gm[GREG ? NODES : 1][9];
  if constexpr (GREG) {
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
      const int n = tid + j * NT;
#pragma unroll
      for (int c = 0; c < 9; ++c) gm[j][c] = n < N3 ? __ldg(ge + 9 * n + c) : 0.0;
    }
  }
  if constexpr (!LEAN) {
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
      const int n = tid + j * NT;
      cf[j][0] = cf[j][1] = cf[j][2] = cf[j][3] = 0.0;
      if (n < N3) {
        elastic_coefficients(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2),
                             &cf[j][0], &cf[j][1], &cf[j][2], &cf[j][3]);
#pragma unroll
        for (int c = 0; c < 4; ++c) cf[j][c] *= dx;
      }
    }
  }
  __syncthreads();
  if constexpr (!LEAN) {
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
      const int n = tid + j * NT;
#pragma unroll
      for (int s = 0; s < M; ++s) avg[j][s] = n < N3 ? sp[s * S + pad(n)] : 0.0;
    }
  }

  double part[NODES][9];

  // Line pass of direction d: reference derivatives of quantities
  // sub*A .. sub*A+nq-1 of the current term into dst[A][S].
  auto line_pass = [&](int k, int d, int sub, double* dst_base) {
    const double* Et = sT + k * Sh::STEP_TABLE;
    const double* Ot = Et + H * H;
    const double* Dm = Ot + H * H;  // odd N: middle column (rows < h)
    const double* Om = Dm + H;      // odd N: middle row odd part
    const int nq = (M - sub * A) < A ? (M - sub * A) : A;
    for (int task = tid; task < nq * N * N; task += NT) {
      const int ql = task / (N * N);
      const int a = (task / N) % N, b = task % N;  // line position (slower, faster)
      int base, stride;
      if (d == 0) { base = a * PLANE + b * RX; stride = 1; }   // (z, y), along x
      else if (d == 1) { base = a * PLANE + b; stride = RX; }  // (z, x), along y
      else { base = a * RX + b; stride = PLANE; }              // (y, x), along z
      const double* u = sp + (sub * A + ql) * S + base;
      double ev[H > 0 ? H : 1], od[H > 0 ? H : 1];
#pragma unroll
      for (int l = 0; l < H; ++l) {
        const double lo = u[l * stride], hi = u[(N - 1 - l) * stride];
        ev[l] = lo + hi;
        od[l] = lo - hi;
      }
      double out[N];
#pragma unroll
      for (int i = 0; i < H; ++i) {
        double P = 0.0, Q = 0.0;
#pragma unroll
        for (int l = 0; l < H; ++l) {
          P = fma(Et[i * H + l], ev[l], P);
          Q = fma(Ot[i * H + l], od[l], Q);
        }
        if (ODD) P = fma(Dm[i], u[mid * stride], P);
        out[i] = P + Q;
        out[N - 1 - i] = Q - P;
      }
      if (ODD) {
        double Q = 0.0;
#pragma unroll
        for (int l = 0; l < H; ++l) Q = fma(Om[l], od[l], Q);
        out[mid] = Q;
      }
      double* dst = dst_base + ql * S + base;
#pragma unroll
      for (int i = 0; i < N; ++i) dst[i * stride] = out[i];
    }
  };

  // Pointwise pass of direction d: metric row d times the reference
  // derivatives in src[A][S], into the partial sums; the last pass of a step
  // forms r_{k+1}, adds it to the average and stores it as the next term.
  auto pointwise = [&](int k, int d, auto SUB, const double* src, bool last) {
    constexpr int sub = decltype(SUB)::value;
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
      const int n = tid + j * NT;
      if (n >= N3) continue;
      const int pn = pad(n);
      double g0, g1, g2;
      if constexpr (GREG) {
        g0 = d == 0 ? gm[j][0] : d == 1 ? gm[j][3] : gm[j][6];
        g1 = d == 0 ? gm[j][1] : d == 1 ? gm[j][4] : gm[j][7];
        g2 = d == 0 ? gm[j][2] : d == 1 ? gm[j][5] : gm[j][8];
      } else {
        g0 = __ldg(ge + 9 * n + 3 * d);
        g1 = __ldg(ge + 9 * n + 3 * d + 1);
        g2 = __ldg(ge + 9 * n + 3 * d + 2);
      }
#pragma unroll
      for (int ql = 0; ql < A; ++ql) {
        constexpr int s0 = sub * A;
        if (s0 + ql < M) curv_add(s0 + ql, src[ql * S + pn], g0, g1, g2, part[j]);
      }
      if (!last) continue;
      double invrho, lam, mu, mu2;
      if constexpr (LEAN) {
        elastic_coefficients(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2),
                             &invrho, &lam, &mu, &mu2);
        invrho *= dx; lam *= dx; mu *= dx; mu2 *= dx;
      } else {
        invrho = cf[j][0]; lam = cf[j][1]; mu = cf[j][2]; mu2 = cf[j][3];
      }
      const double* pj = part[j];
      const double ltr = __dmul_rn(lam, (pj[kS11] + pj[kS22]) + pj[kS33]);
      double r[9];
      r[kV1] = __dmul_rn(invrho, pj[kV1]);
      r[kV2] = __dmul_rn(invrho, pj[kV2]);
      r[kV3] = __dmul_rn(invrho, pj[kV3]);
      r[kS11] = fma(mu2, pj[kS11], ltr);
      r[kS22] = fma(mu2, pj[kS22], ltr);
      r[kS33] = fma(mu2, pj[kS33], ltr);
      r[kS12] = __dmul_rn(mu, pj[kS12]);
      r[kS13] = __dmul_rn(mu, pj[kS13]);
      r[kS23] = __dmul_rn(mu, pj[kS23]);
#pragma unroll
      for (int s = 0; s < M; ++s) {
        if constexpr (LEAN) {
          const double v = __dadd_rn(gavg[n * M + s], r[s]);  // never fused with r's product
          if (k + 1 < N) {
            gavg[n * M + s] = v;
            sp[s * S + pn] = r[s];
          } else {
            sp[s * S + pn] = v;  // final average, staged for the store
          }
        } else {
          avg[j][s] = __dadd_rn(avg[j][s], r[s]);
          if (k + 1 < N) sp[s * S + pn] = r[s];
        }
      }
    }
  };

  for (int k = 0; k < N; ++k) {
#pragma unroll
    for (int j = 0; j < NODES; ++j)
#pragma unroll
      for (int c = 0; c < 9; ++c) part[j][c] = 0.0;
    if constexpr (DB) {
      // double-buffered: the pointwise pass of direction d and the line pass
      // of direction d+1 share a phase (4 barriers per step instead of 6)
      line_pass(k, 0, 0, sacc);
      __syncthreads();
#pragma unroll 1
      for (int d = 0; d < 3; ++d) {
        if (d < 2) line_pass(k, d + 1, 0, sacc + ((d + 1) & 1) * (A * S));
        pointwise(k, d, std::integral_constant<int, 0>{}, sacc + (d & 1) * (A * S), d == 2);
        __syncthreads();
      }
    } else {
#pragma unroll 1
      for (int d = 0; d < 3; ++d) {
        line_pass(k, d, 0, sacc);
        __syncthreads();
        pointwise(k, d, std::integral_constant<int, 0>{}, sacc, SUBS == 1 && d == 2);
        __syncthreads();
        if constexpr (SUBS > 1) {
          line_pass(k, d, 1, sacc);
          __syncthreads();
          pointwise(k, d, std::integral_constant<int, 1>{}, sacc, d == 2);
          __syncthreads();
        }
      }
    }
  }

  if constexpr (!LEAN) {
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
      const int n = tid + j * NT;
      if (n >= N3) continue;
      const int pn = pad(n);
#pragma unroll
      for (int s = 0; s < M; ++s) sp[s * S + pn] = avg[j][s];
    }
  }
  __syncthreads();
  for (int f = tid; f < M * N3; f += NT) {
    const int n = f / M, s = f - n * M;
    gavg[f] = sp[s * S + pad(n)];
  }
  double* fe = out_faces + e * (int64_t)(6 * N * N * M);
  for (int o = tid; o < 6 * N * N * M; o += NT) {
    const int s = o % M;
    int rest = o / M;
    const int bb = rest % N;
    rest /= N;
    const int aa = rest % N;
    const int f = rest / N;
    const int dd = f >> 1;
    const double* phi = sPhi + (f & 1) * N;
    int base, stride;
    if (dd == 0) { base = aa * PLANE + bb * RX; stride = 1; }
    else if (dd == 1) { base = aa * PLANE + bb; stride = RX; }
    else { base = aa * RX + bb; stride = PLANE; }
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) acc = fma(phi[i], sp[s * S + base + i * stride], acc);
    fe[o] = acc;
  }
}

}  // namespace stp
