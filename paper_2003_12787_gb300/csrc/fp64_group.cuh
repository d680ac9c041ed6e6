// FP64 STP over one group of elements (device code shared by the
// single-workload kernel and the batched persistent kernel).
//
// One CTA owns EPC whole elements. The element's current Taylor term lives in
// shared memory in structure-of-arrays layout p[quantity][node]; every thread
// owns NPT nodes and, per Cauchy-Kowalewsky step, forms the 18 directional
// derivatives its node needs straight from shared memory, combines them with
// the node's elastic coefficients and adds the new term to the running time
// average. This is the sum-factorised, dimension-by-dimension scheme of
// Sec. IV (SplitCK) with the time average accumulated on the fly, mapped onto
// one SM: the O(N^3 m) live set sits in shared memory, the per-node result in
// registers.
//
// Taylor bookkeeping: r_k = dt^k/(k+1)! q^(k) satisfies r_0 = q,
// r_{k+1} = dt/(k+2) * L r_k with L q = -sum_d B_d (D_d q)/dx, and the time
// average of Eq. (exahypeTimeAverage) divided by dt is sum_{k=0..N} r_k.
#pragma once
#include "ck_fp64.cuh"
#include "stp_internal.h"

namespace stp {

constexpr int ceil_div(int a, int b) { return (a + b - 1) / b; }

template <int N, int NPT, int EPC, bool AVG_SMEM>
struct Fp64Shape {
  static constexpr int N3 = N * N * N;
  static constexpr int T = ceil_div(N3, NPT);       // threads per element
  static constexpr int BLOCK = T * EPC;
  static constexpr int S = N3 | 1;                  // odd row stride: no bank aliasing across quantities
  static constexpr int LDD = N | 1;                 // odd row stride of D: distinct banks per row
  static constexpr int SLOT = (kQuantities + 4 + (AVG_SMEM ? kQuantities : 0)) * S;
  static constexpr int TABLE = N * N * LDD + 2 * N;
  static constexpr size_t SMEM = sizeof(double) * (size_t)(TABLE + EPC * SLOT);
  static constexpr int MINB_SMEM = (int)((232448 - 1024) / SMEM);
  static constexpr int MINB_THR = 2048 / BLOCK;
  static constexpr int MINB = MINB_SMEM < 1 ? 1 : (MINB_SMEM < MINB_THR ? MINB_SMEM : MINB_THR);
};

// Elements [e0, e0 + EPC) of one set, clipped to E, by the calling CTA
// (NTHREADS threads, NTHREADS >= EPC * T). Starts and ends with a barrier
// free of pending shared-memory reads, so a CTA may call it repeatedly.
// R_GLOBAL: the new term of the owned nodes is parked in rbuf (global memory,
// 9*S doubles per element of the group, private to the calling CTA) instead
// of registers until every thread has read the old one; used for shapes with
// many nodes per thread, which would not fit in registers.
template <int N, int NPT, int EPC, bool AVG_SMEM, int NTHREADS, bool R_GLOBAL = false>
__device__ __forceinline__ void fp64_group(double* smem, const double* __restrict__ q,
                                           const double* __restrict__ params,
                                           double* __restrict__ out_avg,
                                           double* __restrict__ out_faces,
                                           const double* __restrict__ tables, int64_t e0,
                                           int64_t E, double* __restrict__ rbuf = nullptr) {
  using Sh = Fp64Shape<N, NPT, EPC, AVG_SMEM>;
  static_assert(Sh::BLOCK <= NTHREADS, "group needs more threads than the CTA has");
  constexpr int N3 = Sh::N3, T = Sh::T, S = Sh::S, LDD = Sh::LDD;
  constexpr int M = kQuantities;
  double* sD = smem;                     // [N steps][N rows][LDD]
  double* sPhi = sD + N * N * LDD;       // phi0[N], phi1[N]
  const int tid = threadIdx.x;
  const int el = tid / T;
  const int lt = tid - el * T;
  const int64_t e = e0 + el;
  const bool active = (el < EPC) && (e < E);
  double* sp = sPhi + 2 * N + (el < EPC ? el : 0) * Sh::SLOT;  // p[M][S]: current term r_k
  double* sc = sp + M * S;                     // coef[4][S]: 1/rho, lambda, mu, 2 mu
  double* sa = sc + 4 * S;                     // avg[M][S] when AVG_SMEM
  double* gavg = out_avg + e * (int64_t)(M * N3);

  for (int i = tid; i < N * N * N; i += NTHREADS) {
    const int row = i / N, col = i - row * N;  // row = k*N + r
    sD[row * LDD + col] = tables[i];
  }
  for (int i = tid; i < 2 * N; i += NTHREADS) sPhi[i] = tables[N3 + i];

  if (active) {
    const double* qe = q + e * (int64_t)(M * N3);
    for (int f = lt; f < M * N3; f += T) {  // coalesced AoS read, SoA scatter
      const int n = f / M, s = f - n * M;
      const double v = __ldg(qe + f);
      sp[s * S + n] = v;
      if (AVG_SMEM) sa[s * S + n] = v; else gavg[f] = v;
    }
    const double* pe = params + e * (int64_t)(kParams * N3);
    for (int n = lt; n < N3; n += T) {
      const double rho = __ldg(pe + 3 * n), cp = __ldg(pe + 3 * n + 1), cs = __ldg(pe + 3 * n + 2);
      elastic_coefficients(rho, cp, cs, &sc[n], &sc[S + n], &sc[2 * S + n], &sc[3 * S + n]);
    }
  }
  __syncthreads();

  double* rb = R_GLOBAL ? rbuf + (el < EPC ? el : 0) * (M * S) : nullptr;
  for (int k = 0; k < N; ++k) {
    const double* Dk = sD + k * N * LDD;
    double r[R_GLOBAL ? 1 : NPT][M];
#pragma unroll(R_GLOBAL ? 1 : NPT)
    for (int j = 0; j < NPT; ++j) {
      const int n = lt + j * T;
      if (!active || n >= N3) continue;
      const int x = n % N, y = (n / N) % N, z = n / (N * N);
      double* rj = r[R_GLOBAL ? 0 : j];
      ck_node_fp64<N, S, LDD>(sp, Dk, x, y, z, sc[n], sc[S + n], sc[2 * S + n], sc[3 * S + n], rj);
      if (AVG_SMEM) {
#pragma unroll
        for (int s = 0; s < M; ++s) sa[s * S + n] += rj[s];
      } else {
#pragma unroll
        for (int s = 0; s < M; ++s) gavg[n * M + s] += rj[s];
      }
      if (R_GLOBAL && k + 1 < N) {
#pragma unroll
        for (int s = 0; s < M; ++s) rb[s * S + n] = rj[s];
      }
    }
    __syncthreads();  // every thread has read r_k
    if (k + 1 < N) {
#pragma unroll
      for (int j = 0; j < NPT; ++j) {
        const int n = lt + j * T;
        if (!active || n >= N3) continue;
#pragma unroll
        for (int s = 0; s < M; ++s) sp[s * S + n] = R_GLOBAL ? rb[s * S + n] : r[j][s];
      }
      __syncthreads();  // r_{k+1} visible
    }
  }

  if (active) {
    if (AVG_SMEM) {
      for (int f = lt; f < M * N3; f += T) {
        const int n = f / M, s = f - n * M;
        gavg[f] = sa[s * S + n];
      }
    }
    // Face projections of the time average (Sec. II-B): one phi contraction per face.
    double* fe = out_faces + e * (int64_t)(6 * N * N * M);
    for (int o = lt; o < 6 * N * N * M; o += T) {
      const int s = o % M;
      int rest = o / M;
      const int bb = rest % N;
      rest /= N;
      const int aa = rest % N;
      const int f = rest / N;
      const int d = f >> 1;
      const double* phi = sPhi + (f & 1) * N;
      int base, stride;
      if (d == 0) { base = (aa * N + bb) * N; stride = 1; }
      else if (d == 1) { base = aa * N * N + bb; stride = N; }
      else { base = aa * N + bb; stride = N * N; }
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int node = base + i * stride;
        const double v = AVG_SMEM ? sa[s * S + node] : gavg[node * M + s];
        acc = fma(phi[i], v, acc);
      }
      fe[o] = acc;
    }
  }
  __syncthreads();  // shared memory may be reused by the next group
}

}  // namespace stp
