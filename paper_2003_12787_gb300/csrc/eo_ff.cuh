// Even-odd line contractions in float-float arithmetic (device code shared by
// the FP32 and float-float variants of the Space-Time Predictor).
//
// Layout of one element in shared memory: p[quantity][node] with x rows padded
// to an odd length RX and the quantity stride S odd (bank spread). D is
// centro-antisymmetric on symmetric nodes (Gauss-Legendre, Gauss-Lobatto), so with
// h = floor(N/2), e_l = u_l + u_{N-1-l}, o_l = u_l - u_{N-1-l} (l < h),
// E[i][l] = (D[i][l] + D[i][N-1-l]) / 2 and O[i][l] = (D[i][l] - D[i][N-1-l]) / 2,
// the derivative of a line is (D u)_i = P_i + Q_i and (D u)_{N-1-i} = Q_i - P_i
// with P_i = sum_l E[i][l] e_l (+ D[i][h] u_h for odd N), Q_i = sum_l O[i][l] o_l,
// and (D u)_h = sum_l O[h][l] o_l for odd N. Each direction pass (Sec. IV,
// SplitCK) contracts the lines of the six quantities it couples and adds
// them into nine per-node accumulators; the pointwise update then forms the
// new term from the accumulators and the node's elastic coefficients.
#pragma once
#include "bulk.cuh"
#include "fp64_eo.cuh"
#include "ff32.cuh"

namespace stp {

// Shared-memory layout of one element. PERNODE0: the first step runs node by
// node from p alone (no accumulators), for N where they do not fit.
template <int N, bool PERNODE0 = false>
struct EoFfShape {
  static constexpr int N3 = N * N * N;
  static constexpr int RX = N | 1;  // x rows padded to an odd length (banks)
  static constexpr int PLANE = N * RX;
  static constexpr int S = (N * PLANE) | 1;
  static constexpr int H = N / 2;
  static constexpr bool ODD = (N & 1) != 0;
  // per step: E[H][H], O[H][H], middle column (rows < H) and middle-row odd part (odd N)
  static constexpr int STEP_TABLE = 2 * H * H + (ODD ? 2 * H : 0);
  // FP32 tables: the same with rows padded to a multiple of 4 (16-byte loads)
  static constexpr int HP = (H + 3) & ~3;
  static constexpr int STEP32 = 2 * H * HP + (ODD ? 2 * HP : 0);
  // floats first: FP32 tables of steps 0..N-1 (row 0 unused); then 8-byte
  // float-float entries: step-0 table, phi0, phi1, and an area of 18 S
  // entries holding p[9][S] and acc[9][S] in float-float for step 0, then
  // p[9][S] and 18 partial-derivative arrays [18][S] in FP32, then the
  // average in float-float
  // With PERNODE0, step 0 runs node by node from p alone (no accumulators):
  // the step-0 table is the full N x LDD matrix and the area only needs
  // max(9 S pairs, 27 S floats).
  static constexpr int LDD = N | 1;
  static constexpr int TABLE0 = PERNODE0 ? N * LDD : STEP_TABLE;
  static constexpr int AREA = PERNODE0 ? (27 * S + 1) / 2 : 18 * S;
  static constexpr int PAIRS = TABLE0 + 2 * N + AREA;
  static constexpr size_t SMEM = sizeof(float) * (size_t)(N * STEP32) + sizeof(float2) * (size_t)PAIRS;
  static_assert((N * STEP32) % 4 == 0, "FP32 tables keep the doubles 16-byte aligned");
};

// Entry r of the even-odd table of one step matrix Dk (N x N, row-major), in FP64.
template <int N>
__device__ __forceinline__ double eo_table_entry(const double* __restrict__ Dk, int r) {
  constexpr int H = N / 2, mid = H;
  if (r < 2 * H * H) {
    const int which = r / (H * H), i = (r / H) % H, l = r % H;
    const double a = Dk[i * N + l], b = Dk[i * N + (N - 1 - l)];
    return which == 0 ? 0.5 * (a + b) : 0.5 * (a - b);
  }
  const int rr = r - 2 * H * H;  // odd N only
  if (rr < H) return Dk[rr * N + mid];
  const int l = rr - H;
  return 0.5 * (Dk[mid * N + l] - Dk[mid * N + (N - 1 - l)]);
}

// One direction pass in float-float over the 6 N^2 lines of the
// quantities it couples (threads tid < use); the first contribution to an
// accumulator is written, later ones added.
template <int N>
__device__ __forceinline__ void eo_pass_ff(const float2* __restrict__ sp, float2* __restrict__ sacc,
                                           const float2* __restrict__ T, int pass, int tid, int use) {
  using Sh = EoFfShape<N>;
  constexpr int S = Sh::S, H = Sh::H, RX = Sh::RX, PLANE = Sh::PLANE, mid = H;
  constexpr bool ODD = Sh::ODD;
  const float2* E = T;
  const float2* O = E + H * H;
  const float2* Dm = O + H * H;
  const float2* Om = Dm + H;
  for (int task = tid; task < (tid < use ? 6 * N * N : 0); task += use) {
    const int q6 = task / (N * N);
    const int a = (task / N) % N, b = task % N;
    const int s = eo_qty(pass, q6), acc = eo_acc(pass, q6);
    int base, stride;
    if (pass == 0) { base = a * PLANE + b * RX; stride = 1; }
    else if (pass == 1) { base = a * PLANE + b; stride = RX; }
    else { base = a * RX + b; stride = PLANE; }
    const float2* u = sp + s * S + base;
    float2 ev[H > 0 ? H : 1], od[H > 0 ? H : 1];
#pragma unroll
    for (int l = 0; l < H; ++l) {
      const float2 lo = u[l * stride], hi = u[(N - 1 - l) * stride];
      ev[l] = ff::add(lo, hi);
      od[l] = ff::sub(lo, hi);
    }
    float2 out[N];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      ff::Dot P, Q;
#pragma unroll
      for (int l = 0; l < H; ++l) {
        P.fma(E[i * H + l], ev[l]);
        Q.fma(O[i * H + l], od[l]);
      }
      if (ODD) P.fma(Dm[i], u[mid * stride]);
      const float2 pv = P.value_lazy(), qv = Q.value_lazy();
      out[i] = ff::add_lazy(pv, qv);
      out[N - 1 - i] = ff::sub_lazy(qv, pv);
    }
    if (ODD) {
      ff::Dot Q;
#pragma unroll
      for (int l = 0; l < H; ++l) Q.fma(Om[l], od[l]);
      out[mid] = Q.value_lazy();
    }
    float2* dst = sacc + acc * S + base;
    if (eo_first(pass, acc)) {
#pragma unroll
      for (int i = 0; i < N; ++i) dst[i * stride] = out[i];
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) dst[i * stride] = ff::add_lazy(dst[i * stride], out[i]);
    }
  }
}

// New term of one node in float-float.
__device__ __forceinline__ void eo_pointwise_ff(const float2 g[9], float2 invrho, float2 lam,
                                                float2 mu, float2 mu2, float2 r[9]) {
  const float2 ltr = ff::mul(lam, ff::add(ff::add(g[6], g[7]), g[8]));
  r[kV1] = ff::mul(invrho, g[0]);
  r[kV2] = ff::mul(invrho, g[1]);
  r[kV3] = ff::mul(invrho, g[2]);
  r[kS11] = ff::add(ff::mul(mu2, g[6]), ltr);
  r[kS22] = ff::add(ff::mul(mu2, g[7]), ltr);
  r[kS33] = ff::add(ff::mul(mu2, g[8]), ltr);
  r[kS12] = ff::mul(mu, g[3]);
  r[kS13] = ff::mul(mu, g[4]);
  r[kS23] = ff::mul(mu, g[5]);
}

// Lame coefficients (1/rho, lambda, mu, 2 mu) in float-float from FP64
// (rho, cp, cs); 1/rho is the FP32 reciprocal refined by one Newton step.
__device__ __forceinline__ void elastic_coefficients_ff(double rho, double cp, double cs, float2 c[4]) {
  const float2 r = ff::split(rho), p = ff::split(cp), v = ff::split(cs);
  const float2 cs2 = ff::mul(v, v);
  const float2 m = ff::mul(r, cs2);
  const float2 y0 = make_float2(1.0f / r.x, 0.f);
  const float2 res = ff::sub(make_float2(1.f, 0.f), ff::mul(r, y0));
  c[0] = ff::add(y0, ff::mul(y0, res));
  c[1] = ff::mul(r, ff::sub(ff::mul(p, p), make_float2(2.f * cs2.x, 2.f * cs2.y)));
  c[2] = m;
  c[3] = make_float2(2.f * m.x, 2.f * m.y);
}

// One CK step of one node in float-float (same contraction pattern as the
// FP64 per-node step): dimension-split derivatives of the owned node from
// the x-, y- and z-lines through it, combined with the node's coefficients.
template <int N>
__device__ __forceinline__ void ck_node_ff(const float2* __restrict__ p, const float2* __restrict__ D0,
                                           int x, int y, int z, const float2 c[4], float2 r[9]) {
  using Sh = EoFfShape<N, true>;
  constexpr int S = Sh::S, RX = Sh::RX, PLANE = Sh::PLANE, LDD = Sh::LDD;
  const float2* Dx = D0 + x * LDD;
  const float2* Dy = D0 + y * LDD;
  const float2* Dz = D0 + z * LDD;
  const float2* px = p + z * PLANE + y * RX;
  const float2* py = p + z * PLANE + x;
  const float2* pz = p + y * RX + x;
  ff::Dot v1, v2, v3, s12a, s12b, s13a, s13b, s23a, s23b, a, b, cc;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const float2 d = Dx[l];
    v1.fma(d, px[kS11 * S + l]);
    v2.fma(d, px[kS12 * S + l]);
    v3.fma(d, px[kS13 * S + l]);
    a.fma(d, px[kV1 * S + l]);
    s12a.fma(d, px[kV2 * S + l]);
    s13a.fma(d, px[kV3 * S + l]);
  }
  ff::Dot v1y, v2y, v3y;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const float2 d = Dy[l];
    const int o = l * RX;
    v1y.fma(d, py[kS12 * S + o]);
    v2y.fma(d, py[kS22 * S + o]);
    v3y.fma(d, py[kS23 * S + o]);
    s12b.fma(d, py[kV1 * S + o]);
    b.fma(d, py[kV2 * S + o]);
    s23a.fma(d, py[kV3 * S + o]);
  }
  ff::Dot v1z, v2z, v3z;
#pragma unroll
  for (int l = 0; l < N; ++l) {
    const float2 d = Dz[l];
    const int o = l * PLANE;
    v1z.fma(d, pz[kS13 * S + o]);
    v2z.fma(d, pz[kS23 * S + o]);
    v3z.fma(d, pz[kS33 * S + o]);
    s13b.fma(d, pz[kV1 * S + o]);
    s23b.fma(d, pz[kV2 * S + o]);
    cc.fma(d, pz[kV3 * S + o]);
  }
  float2 g[9];
  g[0] = ff::add(ff::add(v1.value(), v1y.value()), v1z.value());
  g[1] = ff::add(ff::add(v2.value(), v2y.value()), v2z.value());
  g[2] = ff::add(ff::add(v3.value(), v3y.value()), v3z.value());
  g[3] = ff::add(s12a.value(), s12b.value());
  g[4] = ff::add(s13a.value(), s13b.value());
  g[5] = ff::add(s23a.value(), s23b.value());
  g[6] = a.value();
  g[7] = b.value();
  g[8] = cc.value();
  eo_pointwise_ff(g, c[0], c[1], c[2], c[3], r);
}

// Loads element state q_e (AoS doubles, node-major) into sp[s * S + pad(n)]
// as float-float scaled by 2^-sc, where sc makes the element's largest finite
// magnitude lie in [1, 2) (L is linear, so the scale carries through every
// step and is undone when the results are converted back). Called by all NT
// threads (NT a multiple of 32); returns sc; ends with a barrier.
// (load_state_ff_layout: the same for any quantity stride S and row/plane
// strides RX, PLANE.)
template <int N, int NT, int S, int RX, int PLANE>
__device__ __forceinline__ int load_state_ff_layout(const double* __restrict__ qe, float2* sp) {
  constexpr int N3 = N * N * N, M = kQuantities;
  static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
  __shared__ int s_field[32];
  double* spd = reinterpret_cast<double*>(sp);  // the same bytes, first as doubles
  int lmax = 0;
  // coalesced AoS read, SoA scatter; loads issued in batches of eight so that
  // eight of them are in flight per thread instead of one
  constexpr int TOTAL = M * N3, ITER = (TOTAL + NT - 1) / NT, BATCH = 8;
#pragma unroll 1
  for (int i0 = 0; i0 < ITER; i0 += BATCH) {
    double v[BATCH];
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const int f = threadIdx.x + (i0 + u) * NT;
      v[u] = (i0 + u < ITER && f < TOTAL) ? __ldg(qe + f) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < BATCH; ++u) {
      const int f = threadIdx.x + (i0 + u) * NT;
      if (i0 + u >= ITER || f >= TOTAL) continue;
      const int n = f / M, s = f - n * M;
      const int pn = (n / (N * N)) * PLANE + ((n / N) % N) * RX + n % N;
      spd[s * S + pn] = v[u];
      const int fld = ff::exponent_field(v[u]);
      if (fld != 0x7ff) lmax = max(lmax, fld);
    }
  }
  lmax = __reduce_max_sync(0xffffffffu, lmax);
  if ((threadIdx.x & 31) == 0) s_field[threadIdx.x >> 5] = lmax;
  __syncthreads();
  int field = 0;
#pragma unroll 1
  for (int w = 0; w < NT / 32; ++w) field = max(field, s_field[w]);
  const int sc = ff::scale_from_field(field);
  for (int f = threadIdx.x; f < M * N3; f += NT) {  // same thread, same entries
    const int n = f / M, s = f - n * M;
    const int pn = (n / (N * N)) * PLANE + ((n / N) % N) * RX + n % N;
    sp[s * S + pn] = ff::split(spd[s * S + pn], sc);
  }
  __syncthreads();
  return sc;
}

// The same, with the element's AoS block first copied in one bulk copy into
// `stage` (shared, 16-byte aligned, at least 72 N^3 bytes, not overlapping
// sp) when q_e allows it (16-byte aligned, 72 N^3 a multiple of 16, so even
// N); otherwise the batched loads above. bar: an initialised mbarrier of the
// CTA, parity: its next phase parity (advanced when used). A wait that gives
// up sets bit 0 of *status (the results are then not to be trusted).
template <int N, int NT, int S, int RX, int PLANE>
__device__ __forceinline__ int load_state_ff_bulk(const double* __restrict__ qe, float2* sp, double* stage,
                                                  uint64_t* bar, uint32_t& parity, unsigned* status) {
  constexpr int N3 = N * N * N, M = kQuantities, TOTAL = M * N3;
  constexpr uint32_t BYTES = 8u * TOTAL;
  if (!bulk::can_copy(qe, BYTES)) return load_state_ff_layout<N, NT, S, RX, PLANE>(qe, sp);
  if (threadIdx.x == 0) bulk::start(stage, qe, BYTES, bar);
  const bool ok = bulk::wait(bar, parity);
  parity ^= 1u;
  if (!ok && threadIdx.x == 0) atomicOr(status, 1u);
  __shared__ int s_field[32];
  int lmax = 0;
  for (int f = threadIdx.x; f < TOTAL; f += NT) {
    const int fld = ff::exponent_field(stage[f]);
    if (fld != 0x7ff) lmax = max(lmax, fld);
  }
  lmax = __reduce_max_sync(0xffffffffu, lmax);
  if ((threadIdx.x & 31) == 0) s_field[threadIdx.x >> 5] = lmax;
  __syncthreads();
  int field = 0;
#pragma unroll 1
  for (int w = 0; w < NT / 32; ++w) field = max(field, s_field[w]);
  const int sc = ff::scale_from_field(field);
  for (int f = threadIdx.x; f < TOTAL; f += NT) {  // SoA scatter from the AoS copy
    const int n = f / M, s = f - n * M;
    const int pn = (n / (N * N)) * PLANE + ((n / N) % N) * RX + n % N;
    sp[s * S + pn] = ff::split(stage[f], sc);
  }
  __syncthreads();
  return sc;
}

template <int N, int NT, bool PERNODE0 = false>
__device__ __forceinline__ int load_state_ff(const double* __restrict__ qe, float2* sp) {
  using Sh = EoFfShape<N, PERNODE0>;
  return load_state_ff_layout<N, NT, Sh::S, Sh::RX, Sh::PLANE>(qe, sp);
}

// The nine accumulator values of node pn from the 18 partial arrays (slot
// order of eo_acc; passes added in x, y, z order).
__device__ __forceinline__ void eo32_gather(const float* __restrict__ spart, int S, int pn, float g[9]) {
  auto P = [&](int pass, int q6) { return spart[(pass * 6 + q6) * S + pn]; };
#pragma unroll
  for (int j = 0; j < 3; ++j) g[j] = (P(0, j) + P(1, j)) + P(2, j);
  g[3] = P(0, 4) + P(1, 3);
  g[4] = P(0, 5) + P(2, 3);
  g[5] = P(1, 5) + P(2, 4);
  g[6] = P(0, 3);
  g[7] = P(1, 4);
  g[8] = P(2, 5);
}

// New term of one node in FP32 from its nine accumulators (slot order of
// eo_acc).
__device__ __forceinline__ void eo_pointwise32(const float g[9], float invrho, float lam, float mu,
                                               float mu2, float r[9]) {
  const float ltr = lam * ((g[6] + g[7]) + g[8]);
  r[kV1] = invrho * g[0];
  r[kV2] = invrho * g[1];
  r[kV3] = invrho * g[2];
  r[kS11] = fmaf(mu2, g[6], ltr);
  r[kS22] = fmaf(mu2, g[7], ltr);
  r[kS33] = fmaf(mu2, g[8], ltr);
  r[kS12] = mu * g[3];
  r[kS13] = mu * g[4];
  r[kS23] = mu * g[5];
}

}  // namespace stp
