// FP64 STP over one element with even-odd derivative contractions (device
// code). Same result as fp64_group (up to rounding order), fewer FP64
// instructions for N >= 6.
//
// Gauss-Legendre nodes are symmetric about 1/2, so the derivative matrix is
// centro-antisymmetric: D[N-1-i][N-1-l] = -D[i][l]. For a line u of N values,
// with h = floor(N/2), e_l = u_l + u_{N-1-l}, o_l = u_l - u_{N-1-l} (l < h),
//   E[i][l] = (D[i][l] + D[i][N-1-l]) / 2,  O[i][l] = (D[i][l] - D[i][N-1-l]) / 2,
//   P_i = sum_l E[i][l] e_l (+ D[i][m] u_m for odd N, m = h),  Q_i = sum_l O[i][l] o_l,
//   (D u)_i = P_i + Q_i,  (D u)_{N-1-i} = Q_i - P_i  (i < h),
//   (D u)_m = sum_l O[m][l] o_l  (odd N).
// A line's N outputs cost about N^2/2 + 2N FP64 operations instead of N^2.
//
// The contractions therefore run line by line, one direction at a time (the
// dimension splitting of Sec. IV, SplitCK): a pass over the 6 quantities each
// direction couples writes or adds every line's derivatives into nine per-node
// accumulators in shared memory; a pointwise pass then forms the new term
// r_{k+1} from the accumulators and the node's elastic coefficients, adds it
// to the time average (kept in the output buffer) and overwrites p.
#pragma once
#include "fp64_group.cuh"

namespace stp {

template <int N>
struct EoShape {
  static constexpr int N3 = N * N * N;
  // x rows padded to an odd length: x-lines handled by consecutive lanes start
  // RX doubles apart and fall into different shared-memory banks
  static constexpr int RX = N | 1;
  static constexpr int PLANE = N * RX;
  static constexpr int S = (N * PLANE) | 1;
  static constexpr int H = N / 2;
  static constexpr bool ODD = (N & 1) != 0;
  // per step: E[H][H], O[H][H], middle column Dm[H] (odd), middle row Om[H] (odd)
  static constexpr int STEP_TABLE = 2 * H * H + (ODD ? 2 * H : 0);
  static constexpr int TABLE = N * STEP_TABLE + 2 * N;  // + phi0, phi1
  // p[9][S], acc[9][S]; the owned nodes' coefficients and average live in registers
  static constexpr int SLOT = 18 * S;
  static constexpr size_t SMEM = sizeof(double) * (size_t)(TABLE + SLOT);
};

// Accumulator slots: 0..2 velocity sums, 3 s12, 4 s13, 5 s23, 6 dv1/dx,
// 7 dv2/dy, 8 dv3/dz. Quantity q6 of pass d (x, y, z) and its accumulator:
__device__ __forceinline__ int eo_qty(int pass, int q6) {
  if (q6 >= 3) return q6 - 3;  // v1, v2, v3
  // stresses sigma_{pass, j}, j = x, y, z
  return pass == 0 ? (q6 == 0 ? kS11 : q6 == 1 ? kS12 : kS13)
       : pass == 1 ? (q6 == 0 ? kS12 : q6 == 1 ? kS22 : kS23)
                   : (q6 == 0 ? kS13 : q6 == 1 ? kS23 : kS33);
}
__device__ __forceinline__ int eo_acc(int pass, int q6) {
  if (q6 < 3) return q6;
  return pass == 0 ? (q6 == 3 ? 6 : q6 == 4 ? 3 : 4)
       : pass == 1 ? (q6 == 3 ? 3 : q6 == 4 ? 7 : 5)
                   : (q6 == 3 ? 4 : q6 == 4 ? 5 : 8);
}
// whether the pass writes (first contribution) or adds into the accumulator
__device__ __forceinline__ bool eo_first(int pass, int acc) {
  if (acc <= 2) return pass == 0;      // velocities: x, y, z
  if (acc == 3 || acc == 4) return pass == 0;  // s12: x, y; s13: x, z
  if (acc == 5) return pass == 1;      // s23: y, z
  return true;                          // dv1/dx, dv2/dy, dv3/dz: one pass each
}

// One element by a CTA of NTHREADS threads, of which the first USE do the
// work (USE chosen so the 6N^2 line tasks and N^3 nodes spread evenly). Thread
// t < USE owns nodes t, t + USE, ... (NODES of them): their elastic
// coefficients and running average stay in its registers. The caller
// guarantees e < E. Ends with a barrier.
template <int N, int NTHREADS, int USE = NTHREADS>
__device__ __forceinline__ void fp64_element_eo(double* smem, const double* __restrict__ q,
                                                const double* __restrict__ params,
                                                double* __restrict__ out_avg,
                                                double* __restrict__ out_faces,
                                                const double* __restrict__ tables, int64_t e) {
  using Sh = EoShape<N>;
  constexpr int N3 = Sh::N3, S = Sh::S, H = Sh::H, M = kQuantities;
  constexpr int RX = Sh::RX, PLANE = Sh::PLANE;
  constexpr bool ODD = Sh::ODD;
  constexpr int mid = H;
  constexpr int NODES = (N3 + USE - 1) / USE;
  // shared-memory index of node n = (z*N + y)*N + x
  auto pad = [](int n) { return (n / (N * N)) * PLANE + ((n / N) % N) * RX + n % N; };
  double* sT = smem;                                  // [N steps][STEP_TABLE]
  double* sPhi = sT + N * Sh::STEP_TABLE;             // phi0[N], phi1[N]
  double* sp = sPhi + 2 * N;                          // p[9][S]
  double* sacc = sp + M * S;                          // acc[9][S]; avg at the end
  const int tid = threadIdx.x;
  double* gavg = out_avg + e * (int64_t)(M * N3);

  // even/odd tables of every step from the scaled D_k (tables[k*N*N + i*N + l])
  for (int idx = tid; idx < N * Sh::STEP_TABLE; idx += NTHREADS) {
    const int k = idx / Sh::STEP_TABLE, r = idx - k * Sh::STEP_TABLE;
    const double* Dk = tables + k * N * N;
    double v;
    if (r < 2 * H * H) {
      const int which = r / (H * H), i = (r / H) % H, l = r % H;
      const double a = Dk[i * N + l], b = Dk[i * N + (N - 1 - l)];
      v = which == 0 ? 0.5 * (a + b) : 0.5 * (a - b);
    } else {
      const int rr = r - 2 * H * H;  // odd N only
      if (rr < H) v = Dk[rr * N + mid];                     // middle column, rows i < h
      else {
        const int l = rr - H;                                // middle row, odd part
        v = 0.5 * (Dk[mid * N + l] - Dk[mid * N + (N - 1 - l)]);
      }
    }
    sT[idx] = v;
  }
  for (int i = tid; i < 2 * N; i += NTHREADS) sPhi[i] = tables[N * N * N + i];

  const double* qe = q + e * (int64_t)(M * N3);
  for (int f = tid; f < M * N3; f += NTHREADS) {  // coalesced AoS read, SoA scatter
    const int n = f / M, s = f - n * M;
    sp[s * S + pad(n)] = __ldg(qe + f);
  }
  double cf[NODES][4], avg[NODES][M];
  const double* pe = params + e * (int64_t)(kParams * N3);
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * USE;
    if (tid < USE && n < N3)
      elastic_coefficients(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2), &cf[j][0],
                           &cf[j][1], &cf[j][2], &cf[j][3]);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * USE;
#pragma unroll
    for (int s = 0; s < M; ++s) avg[j][s] = (tid < USE && n < N3) ? sp[s * S + pad(n)] : 0.0;
  }

  for (int k = 0; k < N; ++k) {
    const double* E = sT + k * Sh::STEP_TABLE;
    const double* O = E + H * H;
    const double* Dm = O + H * H;  // odd N: middle column (rows < h)
    const double* Om = Dm + H;     // odd N: middle row odd part
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
      for (int task = tid; task < (tid < USE ? 6 * N * N : 0); task += USE) {
        const int q6 = task / (N * N);
        const int a = (task / N) % N, b = task % N;  // line position (slower, faster)
        const int s = eo_qty(pass, q6), acc = eo_acc(pass, q6);
        int base, stride;
        if (pass == 0) { base = a * PLANE + b * RX; stride = 1; }     // (z, y), along x
        else if (pass == 1) { base = a * PLANE + b; stride = RX; }    // (z, x), along y
        else { base = a * RX + b; stride = PLANE; }                   // (y, x), along z
        const double* u = sp + s * S + base;
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
            P = fma(E[i * H + l], ev[l], P);
            Q = fma(O[i * H + l], od[l], Q);
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
        double* dst = sacc + acc * S + base;
        if (eo_first(pass, acc)) {
#pragma unroll
          for (int i = 0; i < N; ++i) dst[i * stride] = out[i];
        } else {
#pragma unroll
          for (int i = 0; i < N; ++i) dst[i * stride] += out[i];
        }
      }
      __syncthreads();
    }
    // pointwise: new term of the owned nodes, average, overwrite p (all reads
    // of p are done)
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
      const int n = tid + j * USE;
      if (tid >= USE || n >= N3) continue;
      const int pn = pad(n);
      double g[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) g[c] = sacc[c * S + pn];
      const double invrho = cf[j][0], lam = cf[j][1], mu = cf[j][2], mu2 = cf[j][3];
      const double ltr = __dmul_rn(lam, (g[6] + g[7]) + g[8]);
      double r[9];
      r[kV1] = __dmul_rn(invrho, g[0]);
      r[kV2] = __dmul_rn(invrho, g[1]);
      r[kV3] = __dmul_rn(invrho, g[2]);
      r[kS11] = fma(mu2, g[6], ltr);
      r[kS22] = fma(mu2, g[7], ltr);
      r[kS33] = fma(mu2, g[8], ltr);
      r[kS12] = __dmul_rn(mu, g[3]);
      r[kS13] = __dmul_rn(mu, g[4]);
      r[kS23] = __dmul_rn(mu, g[5]);
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        avg[j][s] += r[s];
        if (k + 1 < N) sp[s * S + pn] = r[s];
      }
    }
    __syncthreads();
  }

  // the average goes through the accumulator area (AoS order, coalesced store)
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * USE;
    if (tid >= USE || n >= N3) continue;
    const int pn = pad(n);
#pragma unroll
    for (int s = 0; s < M; ++s) sacc[s * S + pn] = avg[j][s];
  }
  __syncthreads();
  for (int f = tid; f < M * N3; f += NTHREADS) {
    const int n = f / M, s = f - n * M;
    gavg[f] = sacc[s * S + pad(n)];
  }
  // faces from the average in shared memory
  double* fe = out_faces + e * (int64_t)(6 * N * N * M);
  for (int o = tid; o < 6 * N * N * M; o += NTHREADS) {
    const int s = o % M;
    int rest = o / M;
    const int bb = rest % N;
    rest /= N;
    const int aa = rest % N;
    const int f = rest / N;
    const int d = f >> 1;
    const double* phi = sPhi + (f & 1) * N;
    int base, stride;
    if (d == 0) { base = aa * PLANE + bb * RX; stride = 1; }
    else if (d == 1) { base = aa * PLANE + bb; stride = RX; }
    else { base = aa * RX + bb; stride = PLANE; }
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) acc = fma(phi[i], sacc[s * S + base + i * stride], acc);
    fe[o] = acc;
  }
  __syncthreads();
}

}  // namespace stp

namespace stp {

// ---- even-odd with 16 reusable slots (N = 12) --------------------------------
//
// p (9 arrays) plus the nine accumulators do not fit in shared memory at
// N = 12, but never more than 16 arrays are live at once: s11 is last read in
// the x pass, s12 and s22 in the y pass, and the pointwise pass can write the
// new term in place over the accumulators of the same node. Every thread
// derives the same slot map each step:
//   step start: state in slots st[0..8], the other 7 free (ascending f0..f6)
//   x pass: acc v1,v2,v3 -> f0,f1,f2; dv1/dx -> f3; s12 -> f4; s13 -> f5
//   y pass: dv2/dy -> f6; s23 -> st[s11]
//   z pass: dv3/dz -> st[s12]
//   new state: v1,v2,v3 <- the velocity sums, s12,s13,s23 <- the shear sums,
//              s11,s22,s33 <- dv1/dx, dv2/dy, dv3/dz slots
// The average is accumulated in the output buffer.
template <int N>
struct EoSlotShape {
  static constexpr int N3 = N * N * N;
  static constexpr int S = N3 | 1;
  static constexpr int H = N / 2;
  static constexpr bool ODD = (N & 1) != 0;
  static constexpr int STEP_TABLE = 2 * H * H + (ODD ? 2 * H : 0);
  static constexpr int TABLE = N * STEP_TABLE + 2 * N;
  static constexpr size_t SMEM = sizeof(double) * (size_t)(TABLE + 16 * S);
};

__device__ __forceinline__ int pick9(const int* v, int i) {
  int r = v[0];
#pragma unroll
  for (int j = 1; j < 9; ++j) r = (i == j) ? v[j] : r;
  return r;
}

template <int N, int NTHREADS, int USE = NTHREADS>
__device__ __forceinline__ void fp64_element_eo_slots(double* smem, const double* __restrict__ q,
                                                      const double* __restrict__ params,
                                                      double* __restrict__ out_avg,
                                                      double* __restrict__ out_faces,
                                                      const double* __restrict__ tables, int64_t e) {
  using Sh = EoSlotShape<N>;
  constexpr int N3 = Sh::N3, S = Sh::S, H = Sh::H, M = kQuantities;
  constexpr bool ODD = Sh::ODD;
  constexpr int mid = H;
  constexpr int NODES = (N3 + USE - 1) / USE;
  double* sT = smem;
  double* sPhi = sT + N * Sh::STEP_TABLE;
  double* slot = sPhi + 2 * N;  // [16][S]
  const int tid = threadIdx.x;
  double* gavg = out_avg + e * (int64_t)(M * N3);

  for (int idx = tid; idx < N * Sh::STEP_TABLE; idx += NTHREADS) {
    const int k = idx / Sh::STEP_TABLE, r = idx - k * Sh::STEP_TABLE;
    const double* Dk = tables + k * N * N;
    double v;
    if (r < 2 * H * H) {
      const int which = r / (H * H), i = (r / H) % H, l = r % H;
      const double a = Dk[i * N + l], b = Dk[i * N + (N - 1 - l)];
      v = which == 0 ? 0.5 * (a + b) : 0.5 * (a - b);
    } else {
      const int rr = r - 2 * H * H;
      if (rr < H) v = Dk[rr * N + mid];
      else {
        const int l = rr - H;
        v = 0.5 * (Dk[mid * N + l] - Dk[mid * N + (N - 1 - l)]);
      }
    }
    sT[idx] = v;
  }
  for (int i = tid; i < 2 * N; i += NTHREADS) sPhi[i] = tables[N * N * N + i];

  int st[9];  // slot of each state quantity
#pragma unroll
  for (int s = 0; s < 9; ++s) st[s] = s;
  const double* qe = q + e * (int64_t)(M * N3);
  for (int f = tid; f < M * N3; f += NTHREADS) {
    const int n = f / M, s = f - n * M;
    const double v = __ldg(qe + f);
    slot[s * S + n] = v;  // st[s] == s at the start
    gavg[f] = v;
  }
  double cf[NODES][4];
  const double* pe = params + e * (int64_t)(kParams * N3);
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * USE;
    if (tid < USE && n < N3)
      elastic_coefficients(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2), &cf[j][0],
                           &cf[j][1], &cf[j][2], &cf[j][3]);
  }
  __syncthreads();

  for (int k = 0; k < N; ++k) {
    // slot map of this step
    int fr[7] = {0, 0, 0, 0, 0, 0, 0};
    {
      unsigned used = 0u;
#pragma unroll
      for (int s = 0; s < 9; ++s) used |= 1u << st[s];
      int c = 0;
#pragma unroll
      for (int sl = 0; sl < 16; ++sl) {
        const bool f = !((used >> sl) & 1u);
#pragma unroll
        for (int t = 0; t < 7; ++t) fr[t] = (f && c == t) ? sl : fr[t];
        c += f ? 1 : 0;
      }
    }
    int ac[9];  // slot of each accumulator
    ac[0] = fr[0]; ac[1] = fr[1]; ac[2] = fr[2]; ac[6] = fr[3]; ac[3] = fr[4]; ac[4] = fr[5];
    ac[7] = fr[6]; ac[5] = st[kS11]; ac[8] = st[kS12];

    const double* E = sT + k * Sh::STEP_TABLE;
    const double* O = E + H * H;
    const double* Dm = O + H * H;
    const double* Om = Dm + H;
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
      for (int task = tid; task < (tid < USE ? 6 * N * N : 0); task += USE) {
        const int q6 = task / (N * N);
        const int a = (task / N) % N, b = task % N;
        const int s = eo_qty(pass, q6), acc = eo_acc(pass, q6);
        int base, stride;
        if (pass == 0) { base = (a * N + b) * N; stride = 1; }
        else if (pass == 1) { base = a * N * N + b; stride = N; }
        else { base = a * N + b; stride = N * N; }
        const double* u = slot + pick9(st, s) * S + base;
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
            P = fma(E[i * H + l], ev[l], P);
            Q = fma(O[i * H + l], od[l], Q);
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
        double* dst = slot + pick9(ac, acc) * S + base;
        if (eo_first(pass, acc)) {
#pragma unroll
          for (int i = 0; i < N; ++i) dst[i * stride] = out[i];
        } else {
#pragma unroll
          for (int i = 0; i < N; ++i) dst[i * stride] += out[i];
        }
      }
      __syncthreads();
    }
    // pointwise: new term in place over the accumulators, average in the output
    int nst[9];
    nst[kV1] = ac[0]; nst[kV2] = ac[1]; nst[kV3] = ac[2];
    nst[kS12] = ac[3]; nst[kS13] = ac[4]; nst[kS23] = ac[5];
    nst[kS11] = ac[6]; nst[kS22] = ac[7]; nst[kS33] = ac[8];
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
      const int n = tid + j * USE;
      if (tid >= USE || n >= N3) continue;
      double g[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) g[c] = slot[ac[c] * S + n];
      const double invrho = cf[j][0], lam = cf[j][1], mu = cf[j][2], mu2 = cf[j][3];
      const double ltr = __dmul_rn(lam, (g[6] + g[7]) + g[8]);
      double r[9];
      r[kV1] = __dmul_rn(invrho, g[0]);
      r[kV2] = __dmul_rn(invrho, g[1]);
      r[kV3] = __dmul_rn(invrho, g[2]);
      r[kS11] = fma(mu2, g[6], ltr);
      r[kS22] = fma(mu2, g[7], ltr);
      r[kS33] = fma(mu2, g[8], ltr);
      r[kS12] = __dmul_rn(mu, g[3]);
      r[kS13] = __dmul_rn(mu, g[4]);
      r[kS23] = __dmul_rn(mu, g[5]);
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        gavg[n * M + s] += r[s];
        if (k + 1 < N) slot[nst[s] * S + n] = r[s];
      }
    }
#pragma unroll
    for (int s = 0; s < 9; ++s) st[s] = nst[s];
    __syncthreads();
  }

  double* fe = out_faces + e * (int64_t)(6 * N * N * M);
  for (int o = tid; o < 6 * N * N * M; o += NTHREADS) {
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
    for (int i = 0; i < N; ++i) acc = fma(phi[i], gavg[(base + i * stride) * M + s], acc);
    fe[o] = acc;
  }
  __syncthreads();
}

}  // namespace stp
