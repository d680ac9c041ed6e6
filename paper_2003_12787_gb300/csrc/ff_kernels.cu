// Float-float variant of the Space-Time Predictor (precision STP_PRECISION_FF).
//
// Same Taylor bookkeeping as the FP64 kernels: r_0 = q,
// r_{k+1} = dt/(k+2) * L r_k with L q = -sum_d B_d (D_d q)/dx, and the time
// average of Eq. (exahypeTimeAverage) divided by dt is sum_{k=0..N} r_k, with
// the face projections of Sec. II-B. Every step runs in float-float
// arithmetic (ff32.cuh: about 48 significant bits, error-free TwoSum /
// TwoProduct transformations and Dot2 dot products) on the FP32 pipes; FP64
// instructions remain only in the one addition per output value that turns a
// float-float result into a double. On GB300 one FP64 instruction takes the
// issue capacity of about 64 FP32 ones, so emulating the extra precision
// costs less than running the contractions in FP64. The paper's kernels are
// FP64 throughout; this variant is an addition.
//
// Structure (eo_ff.cuh): one CTA per element, the element's current term in
// shared memory as float-float p[quantity][node]; per step three even-odd
// direction passes (Sec. IV, SplitCK) add each line's derivatives into nine
// per-node accumulators, then a pointwise pass forms the new term, adds it to
// the node's running average (registers, or the output buffer as scratch)
// and overwrites p.
#include "eo_ff.cuh"
#include "stp_internal.h"

namespace stp {
namespace {

template <int N, int NT, int USE, int MINB, bool AVG_REG>
__global__ void __launch_bounds__(NT, MINB)
ff_eo_kernel(const double* __restrict__ q, const double* __restrict__ params,
             double* __restrict__ out_avg, double* __restrict__ out_faces,
             const double* __restrict__ tables, int64_t E) {
  using Sh = EoFfShape<N>;
  constexpr int N3 = Sh::N3, S = Sh::S, RX = Sh::RX, PLANE = Sh::PLANE, ST = Sh::STEP_TABLE;
  constexpr int M = kQuantities;
  constexpr int NODES = (N3 + USE - 1) / USE;
  auto pad = [](int n) { return (n / (N * N)) * PLANE + ((n / N) % N) * RX + n % N; };
  extern __shared__ float2 smem_ff[];
  float2* sT = smem_ff;            // [N][ST] even-odd tables of every step
  float2* sPhi = sT + N * ST;      // phi0[N], phi1[N]
  float2* sp = sPhi + 2 * N;       // p[9][S]; the average at the end
  float2* sacc = sp + M * S;       // acc[9][S]
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  double* gavg = out_avg + e * (int64_t)(M * N3);
  float2* gpark = reinterpret_cast<float2*>(gavg);  // running average when not in registers

  for (int i = tid; i < N * ST; i += NT) {
    const int k = i / ST;
    sT[i] = ff::split(eo_table_entry<N>(tables + k * N * N, i - k * ST));
  }
  for (int i = tid; i < 2 * N; i += NT) sPhi[i] = ff::split(tables[N3 + i]);
  const int sc = load_state_ff<N, NT>(q + e * (int64_t)(M * N3), sp);

  float2 cf[NODES][4], avg[AVG_REG ? NODES : 1][M];
  const double* pe = params + e * (int64_t)(kParams * N3);
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * USE;
    if (tid >= USE || n >= N3) continue;
    elastic_coefficients_ff(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2), cf[j]);
    const int pn = pad(n);
#pragma unroll
    for (int s = 0; s < M; ++s) {
      if (AVG_REG) avg[j][s] = sp[s * S + pn];
      else gpark[n * M + s] = sp[s * S + pn];
    }
  }

  for (int k = 0; k < N; ++k) {
    const float2* T = sT + k * ST;
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
      eo_pass_ff<N>(sp, sacc, T, pass, tid, USE);
      __syncthreads();
    }
    // pointwise: new term of the owned nodes, running average, overwrite p
    // (every read of p in this step is done)
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
      const int n = tid + j * USE;
      if (tid >= USE || n >= N3) continue;
      const int pn = pad(n);
      float2 g[9], r[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) g[c] = sacc[c * S + pn];
      eo_pointwise_ff(g, cf[j][0], cf[j][1], cf[j][2], cf[j][3], r);
#pragma unroll
      for (int s = 0; s < M; ++s) {
        if (AVG_REG) avg[j][s] = ff::add(avg[j][s], r[s]);
        else gpark[n * M + s] = ff::add(gpark[n * M + s], r[s]);
        if (k + 1 < N) sp[s * S + pn] = r[s];
      }
    }
    __syncthreads();
  }

  // time average to the output (FP64) and into shared memory for the faces
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * USE;
    if (tid >= USE || n >= N3) continue;
    const int pn = pad(n);
#pragma unroll
    for (int s = 0; s < M; ++s) {
      const float2 v = AVG_REG ? avg[j][s] : gpark[n * M + s];
      sp[s * S + pn] = v;
      gavg[n * M + s] = ff::to_double(v, sc);
    }
  }
  __syncthreads();
  double* fe = out_faces + e * (int64_t)(6 * N * N * M);
  for (int o = tid; o < 6 * N * N * M; o += NT) {
    const int s = o % M;
    int rest = o / M;
    const int bb = rest % N;
    rest /= N;
    const int aa = rest % N;
    const int f = rest / N;
    const int d = f >> 1;
    const float2* phi = sPhi + (f & 1) * N;
    int base, stride;
    if (d == 0) { base = aa * PLANE + bb * RX; stride = 1; }
    else if (d == 1) { base = aa * PLANE + bb; stride = RX; }
    else { base = aa * RX + bb; stride = PLANE; }
    ff::Dot a;
#pragma unroll
    for (int i = 0; i < N; ++i) a.fma(phi[i], sp[s * S + base + i * stride]);
    fe[o] = ff::to_double(a.value(), sc);
  }
}

template <int N, int NT, int USE, int MINB, bool AVG_REG>
cudaError_t launch_ff_eo(int64_t E, const double* q, const double* params, double* out_avg,
                         double* out_faces, const double* tables, cudaStream_t stream) {
  using Sh = EoFfShape<N>;
  constexpr size_t smem = sizeof(float2) * (size_t)(N * Sh::STEP_TABLE + 2 * N + 18 * Sh::S);
  static_assert(smem <= 232448, "shared memory budget of one CTA exceeded");
  static_assert(USE <= NT && NT <= 1024, "bad thread counts");
  auto kern = ff_eo_kernel<N, NT, USE, MINB, AVG_REG>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (E > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (E == 0) return cudaSuccess;
  kern<<<(unsigned)E, NT, smem, stream>>>(q, params, out_avg, out_faces, tables, E);
  return cudaGetLastError();
}

// ---- N = 12: slot-reusing body ------------------------------------------------
//
// p and the nine accumulators (18 arrays of pairs) do not fit in shared memory
// at N = 12, but at most 16 arrays are live at once; this body uses the slot
// map of the FP64 slot-reusing body (fp64_eo.cuh): every step, the accumulators
// take the 7 free slots and two dead state slots (sigma11 after the x pass,
// sigma12 after the y pass), and the pointwise pass writes the new term in
// place over the node's accumulators. Rows are not padded (no room), the
// running average stays in the output buffer as pairs.
template <int N>
struct FfSlotShape {
  static constexpr int N3 = N * N * N;
  static constexpr int S = N3 | 1;
  static constexpr int H = N / 2;
  static constexpr bool ODD = (N & 1) != 0;
  static constexpr int STEP_TABLE = 2 * H * H + (ODD ? 2 * H : 0);
  static constexpr size_t SMEM = sizeof(float2) * (size_t)(N * STEP_TABLE + 2 * N + 16 * S);
};

template <int N, int NT, int USE>
__global__ void __launch_bounds__(NT, 1)
ff_slots_kernel(const double* __restrict__ q, const double* __restrict__ params,
                double* __restrict__ out_avg, double* __restrict__ out_faces,
                const double* __restrict__ tables, int64_t E) {
  using Sh = FfSlotShape<N>;
  constexpr int N3 = Sh::N3, S = Sh::S, H = Sh::H, ST = Sh::STEP_TABLE, M = kQuantities;
  constexpr bool ODD = Sh::ODD;
  constexpr int mid = H;
  constexpr int NODES = (N3 + USE - 1) / USE;
  extern __shared__ float2 smem_ff[];
  float2* sT = smem_ff;
  float2* sPhi = sT + N * ST;
  float2* slot = sPhi + 2 * N;  // [16][S]
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  double* gavg = out_avg + e * (int64_t)(M * N3);
  float2* gpark = reinterpret_cast<float2*>(gavg);  // running average (pairs)

  for (int i = tid; i < N * ST; i += NT) {
    const int k = i / ST;
    sT[i] = ff::split(eo_table_entry<N>(tables + k * N * N, i - k * ST));
  }
  for (int i = tid; i < 2 * N; i += NT) sPhi[i] = ff::split(tables[N3 + i]);
  // state in slots 0..8 (st[s] == s at the start)
  const int sc = load_state_ff_layout<N, NT, S, N, N * N>(q + e * (int64_t)(M * N3), slot);
  int st[9];
#pragma unroll
  for (int s = 0; s < 9; ++s) st[s] = s;

  float2 cf[NODES][4];
  const double* pe = params + e * (int64_t)(kParams * N3);
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * USE;
    if (tid >= USE || n >= N3) continue;
    elastic_coefficients_ff(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2), cf[j]);
#pragma unroll
    for (int s = 0; s < M; ++s) gpark[n * M + s] = slot[s * S + n];
  }

  for (int k = 0; k < N; ++k) {
    int fr[7] = {0, 0, 0, 0, 0, 0, 0};  // free slots, ascending
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

    const float2* Et = sT + k * ST;
    const float2* Ot = Et + H * H;
    const float2* Dm = Ot + H * H;
    const float2* Om = Dm + H;
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
        const float2* u = slot + pick9(st, s) * S + base;
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
            P.fma(Et[i * H + l], ev[l]);
            Q.fma(Ot[i * H + l], od[l]);
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
        float2* dst = slot + pick9(ac, acc) * S + base;
        if (eo_first(pass, acc)) {
#pragma unroll
          for (int i = 0; i < N; ++i) dst[i * stride] = out[i];
        } else {
#pragma unroll
          for (int i = 0; i < N; ++i) dst[i * stride] = ff::add_lazy(dst[i * stride], out[i]);
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
      float2 g[9], r[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) g[c] = slot[ac[c] * S + n];
      eo_pointwise_ff(g, cf[j][0], cf[j][1], cf[j][2], cf[j][3], r);
#pragma unroll
      for (int s = 0; s < M; ++s) {
        gpark[n * M + s] = ff::add(gpark[n * M + s], r[s]);
        if (k + 1 < N) slot[nst[s] * S + n] = r[s];
      }
    }
#pragma unroll
    for (int s = 0; s < 9; ++s) st[s] = nst[s];
    __syncthreads();
  }

  // time average to the output (FP64) and into slots 0..8 for the faces
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * USE;
    if (tid >= USE || n >= N3) continue;
#pragma unroll
    for (int s = 0; s < M; ++s) {
      const float2 v = gpark[n * M + s];
      slot[s * S + n] = v;
      gavg[n * M + s] = ff::to_double(v, sc);
    }
  }
  __syncthreads();
  double* fe = out_faces + e * (int64_t)(6 * N * N * M);
  for (int o = tid; o < 6 * N * N * M; o += NT) {
    const int s = o % M;
    int rest = o / M;
    const int bb = rest % N;
    rest /= N;
    const int aa = rest % N;
    const int f = rest / N;
    const int d = f >> 1;
    const float2* phi = sPhi + (f & 1) * N;
    int base, stride;
    if (d == 0) { base = (aa * N + bb) * N; stride = 1; }
    else if (d == 1) { base = aa * N * N + bb; stride = N; }
    else { base = aa * N + bb; stride = N * N; }
    ff::Dot a;
#pragma unroll
    for (int i = 0; i < N; ++i) a.fma(phi[i], slot[s * S + base + i * stride]);
    fe[o] = ff::to_double(a.value(), sc);
  }
}

template <int N, int NT, int USE>
cudaError_t launch_ff_slots(int64_t E, const double* q, const double* params, double* out_avg,
                            double* out_faces, const double* tables, cudaStream_t stream) {
  constexpr size_t smem = FfSlotShape<N>::SMEM;
  static_assert(smem + 128 <= 232448, "shared memory budget of one CTA exceeded");
  static_assert(USE <= NT && NT <= 1024, "bad thread counts");
  auto kern = ff_slots_kernel<N, NT, USE>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (E > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (E == 0) return cudaSuccess;
  kern<<<(unsigned)E, NT, smem, stream>>>(q, params, out_avg, out_faces, tables, E);
  return cudaGetLastError();
}

}  // namespace

// Launch shape per N: (N, threads, working threads, CTAs per SM the registers
// are sized for, running average in registers).
#define STP_FF_SHAPES(X)                                                                       \
  X(2, 32, 24, 16, true) X(3, 32, 27, 16, true) X(4, 96, 96, 8, true) X(5, 160, 150, 4, true) \
  X(6, 256, 216, 1, true) X(7, 352, 343, 2, true) X(8, 384, 384, 2, true)                     \
  X(9, 768, 729, 1, true) X(10, 640, 600, 1, true) X(11, 736, 726, 1, false)

// N = 12: the slot-reusing body (threads, working threads).
#define STP_FF_SLOT_SHAPE(X) X(12, 448, 432)

bool ff_supported(int N) {
  switch (N) {
#define X(n, nt, use, minb, ar) case n: return true;
    STP_FF_SHAPES(X)
#undef X
#define X(n, nt, use) case n: return true;
    STP_FF_SLOT_SHAPE(X)
#undef X
    default: return false;
  }
}

cudaError_t launch_ff(int N, int64_t E, const double* q, const double* params, double* out_avg,
                      double* out_faces, const double* tables, cudaStream_t stream) {
  switch (N) {
#define X(n, nt, use, minb, ar) \
  case n: return launch_ff_eo<n, nt, use, minb, ar>(E, q, params, out_avg, out_faces, tables, stream);
    STP_FF_SHAPES(X)
#undef X
#define X(n, nt, use) \
  case n: return launch_ff_slots<n, nt, use>(E, q, params, out_avg, out_faces, tables, stream);
    STP_FF_SLOT_SHAPE(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stp
