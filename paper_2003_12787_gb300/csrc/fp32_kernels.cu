// FP32 variant of the Space-Time Predictor on the CUDA cores (precision
// STP_PRECISION_FP32).
//
// Same Taylor bookkeeping as the FP64 kernels: r_0 = q,
// r_{k+1} = dt/(k+2) * L r_k with L q = -sum_d B_d (D_d q)/dx, and the time
// average of Eq. (exahypeTimeAverage) divided by dt is sum_{k=0..N} r_k.
// The paper's kernels are FP64 throughout; this variant splits the arithmetic
// like the library's tensor-core variants, with FP32 in place of the
// BF16/FP16 slices, and without FP64 instructions on the hot path:
//   * r_1 = dt/2 L q, r_0 + r_1, the time average and the face projections
//     of Sec. II-B in float-float arithmetic (about 48 significant bits,
//     ff32.cuh) on the FP32 pipes;
//   * r_2 .. r_N in FP32 (state, step matrices and coefficients rounded to
//     FP32), their sum accumulated in FP32 and added to r_0 + r_1 at the end.
// On GB300 one FP64 instruction, and likewise one float<->double conversion,
// takes the issue capacity of about 64 FP32 instructions; the only FP64
// operations left are one addition per output value (float-float -> double).
// The contractions are K = N long, too short to feed the tensor cores
// efficiently once slice conversions and the scatter of results back to the
// nodes are paid.
//
// The derivative contractions are the dimension-split scheme of Sec. IV
// (SplitCK) with the even-odd decomposition of the FP64 kernels (D is
// centro-antisymmetric on symmetric nodes, Gauss-Legendre or Gauss-Lobatto, so a line of N
// outputs costs about N^2/2 + 2N operations). One CTA owns one element; the
// element's current term lives in shared memory as p[quantity][node].
#include "eo_ff.cuh"

namespace stp {
namespace {

// Entry r of the padded FP32 table of one step (zeros in the padding).
template <int N>
__device__ __forceinline__ float eo_table_entry32(const double* __restrict__ Dk, int r) {
  using Sh = EoFfShape<N>;
  constexpr int H = Sh::H, HP = Sh::HP;
  int row, col, src;
  if (r < 2 * H * HP) {
    const int which = r / (H * HP);
    row = (r / HP) % H;
    col = r % HP;
    src = which * H * H + row * H + col;
  } else {
    const int rr = r - 2 * H * HP;  // odd N only
    col = rr % HP;
    src = 2 * H * H + (rr / HP) * H + col;
  }
  return col < H ? __double2float_rn(eo_table_entry<N>(Dk, src)) : 0.f;
}

// All three direction passes of one FP32 step at once: every (pass, group of
// QPT quantities, line position) task contracts QPT lines and writes their
// derivatives to partial array pass * 6 + q6 (no read-modify-write, so the
// passes need no barrier between them). Threads tid < use.
template <int N, int QPT>
__device__ __forceinline__ void eo32_passes(const float* __restrict__ sp, float* __restrict__ spart,
                                            const float* __restrict__ T, int tid, int use) {
  using Sh = EoFfShape<N>;
  constexpr int S = Sh::S, H = Sh::H, HP = Sh::HP, RX = Sh::RX, PLANE = Sh::PLANE, mid = H;
  constexpr bool ODD = Sh::ODD;
  constexpr int G = 6 / QPT;
  static_assert(G * QPT == 6, "QPT divides 6");
  constexpr int TASKS = 3 * G * N * N;
  const float4* E4 = reinterpret_cast<const float4*>(T);
  const float4* O4 = reinterpret_cast<const float4*>(T + H * HP);
  const float* Dm = T + 2 * H * HP;
  const float4* Om4 = reinterpret_cast<const float4*>(Dm + HP);
  for (int task = tid; task < (tid < use ? TASKS : 0); task += use) {
    const int pass = task / (G * N * N);
    const int rem = task - pass * (G * N * N);
    const int grp = rem / (N * N);
    const int a = (rem / N) % N, b = rem % N;
    int base, stride;
    if (pass == 0) { base = a * PLANE + b * RX; stride = 1; }
    else if (pass == 1) { base = a * PLANE + b; stride = RX; }
    else { base = a * RX + b; stride = PLANE; }
    float ev[QPT][HP], od[QPT][HP], um[QPT];
#pragma unroll
    for (int qi = 0; qi < QPT; ++qi) {
      const float* u = sp + eo_qty(pass, grp * QPT + qi) * S + base;
#pragma unroll
      for (int l = 0; l < HP; ++l) {
        if (l < H) {
          const float lo = u[l * stride], hi = u[(N - 1 - l) * stride];
          ev[qi][l] = lo + hi;
          od[qi][l] = lo - hi;
        } else {
          ev[qi][l] = 0.f;
          od[qi][l] = 0.f;
        }
      }
      um[qi] = ODD ? u[mid * stride] : 0.f;
    }
    float out[QPT][N];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      float er[HP], orow[HP];
#pragma unroll
      for (int v = 0; v < HP / 4; ++v) {
        const float4 x = E4[i * (HP / 4) + v], y = O4[i * (HP / 4) + v];
        er[4 * v] = x.x; er[4 * v + 1] = x.y; er[4 * v + 2] = x.z; er[4 * v + 3] = x.w;
        orow[4 * v] = y.x; orow[4 * v + 1] = y.y; orow[4 * v + 2] = y.z; orow[4 * v + 3] = y.w;
      }
#pragma unroll
      for (int qi = 0; qi < QPT; ++qi) {
        float P = 0.f, Q = 0.f;
#pragma unroll
        for (int l = 0; l < H; ++l) {
          P = fmaf(er[l], ev[qi][l], P);
          Q = fmaf(orow[l], od[qi][l], Q);
        }
        if (ODD) P = fmaf(Dm[i], um[qi], P);
        out[qi][i] = P + Q;
        out[qi][N - 1 - i] = Q - P;
      }
    }
    if (ODD) {
      float om[HP];
#pragma unroll
      for (int v = 0; v < HP / 4; ++v) {
        const float4 x = Om4[v];
        om[4 * v] = x.x; om[4 * v + 1] = x.y; om[4 * v + 2] = x.z; om[4 * v + 3] = x.w;
      }
#pragma unroll
      for (int qi = 0; qi < QPT; ++qi) {
        float Q = 0.f;
#pragma unroll
        for (int l = 0; l < H; ++l) Q = fmaf(om[l], od[qi][l], Q);
        out[qi][mid] = Q;
      }
    }
#pragma unroll
    for (int qi = 0; qi < QPT; ++qi) {
      float* dst = spart + (pass * 6 + grp * QPT + qi) * S + base;
#pragma unroll
      for (int i = 0; i < N; ++i) dst[i * stride] = out[qi][i];
    }
  }
}

// One element (e < E) by a CTA of NT threads, the first USE doing the work;
// thread t < USE owns nodes t, t + USE, ...
template <int N, int NT, int USE, int QPT, int MINB, bool PERNODE0>
__global__ void __launch_bounds__(NT, MINB)
fp32_eo_kernel(const double* __restrict__ q, const double* __restrict__ params,
               double* __restrict__ out_avg, double* __restrict__ out_faces,
               const double* __restrict__ tables, int64_t E, unsigned int* __restrict__ status) {
  using Sh = EoFfShape<N, PERNODE0>;
  constexpr int N3 = Sh::N3, S = Sh::S, RX = Sh::RX, PLANE = Sh::PLANE, ST = Sh::STEP_TABLE;
  constexpr int ST32 = Sh::STEP32;
  constexpr int M = kQuantities;
  constexpr int NODES = (N3 + USE - 1) / USE;
  auto pad = [](int n) { return (n / (N * N)) * PLANE + ((n / N) % N) * RX + n % N; };
  extern __shared__ double smem[];
  float* sTf = reinterpret_cast<float*>(smem);  // [N][ST32] FP32 tables (16-byte rows)
  float2* sT0 = reinterpret_cast<float2*>(sTf + N * ST32);  // step-0 even-odd table (float-float)
  float2* sPhi = sT0 + Sh::TABLE0;          // phi0[N], phi1[N] (float-float)
  float2* sp = sPhi + 2 * N;                // p[9][S] (float-float, step 0); the average at the end
  float2* sacc = sp + M * S;                // acc[9][S] (float-float, step 0)
  float* spf = reinterpret_cast<float*>(sp);  // p[9][S] (FP32, later steps)
  float* spart = spf + M * S;                 // partial derivatives [18][S] (FP32)
  const int tid = threadIdx.x;
  const int64_t e = blockIdx.x;
  // r_0 + r_1 of the owned nodes is parked in the output average as float-float
  double* gavg = out_avg + e * (int64_t)(M * N3);
  float2* gpark = reinterpret_cast<float2*>(gavg);

  if (PERNODE0) {
    for (int i = tid; i < N * N; i += NT) {
      const int row = i / N, col = i - row * N;
      sT0[row * Sh::LDD + col] = ff::split(tables[i]);
    }
  } else {
    for (int i = tid; i < ST; i += NT) sT0[i] = ff::split(eo_table_entry<N>(tables, i));
  }
  for (int i = ST32 + tid; i < N * ST32; i += NT) {
    const int k = i / ST32;
    sTf[i] = eo_table_entry32<N>(tables + k * N * N, i - k * ST32);
  }
  for (int i = tid; i < 2 * N; i += NT) sPhi[i] = ff::split(tables[N3 + i]);
  // bulk copies (state in, parked average back) land in the accumulator half
  // of the area, 16-byte aligned (its 72 S bytes hold 72 N^3 + 8 for even N)
  __shared__ uint64_t s_bar;
  uint32_t bparity = 0u;
  double* stage = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(sacc) + 15) & ~(uintptr_t)15);
  if (tid == 0) bulk::init(&s_bar);
  __syncthreads();
  int sc;
  if constexpr (PERNODE0)
    sc = load_state_ff<N, NT, PERNODE0>(q + e * (int64_t)(M * N3), sp);
  else
    sc = load_state_ff_bulk<N, NT, S, RX, PLANE>(q + e * (int64_t)(M * N3), sp, stage, &s_bar, bparity, status);

  // step 0 in float-float
  if (!PERNODE0) {
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
      eo_pass_ff<N>(sp, sacc, sT0, pass, tid, USE);
      __syncthreads();
    }
  }
  float r[NODES][M], cf[NODES][4];
  const double* pe = params + e * (int64_t)(kParams * N3);
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * USE;
#pragma unroll
    for (int c = 0; c < 4; ++c) cf[j][c] = 0.f;
    if (tid >= USE || n >= N3) continue;
    float2 c2[4];
    elastic_coefficients_ff(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2), c2);
#pragma unroll
    for (int c = 0; c < 4; ++c) cf[j][c] = c2[c].x;
    const int pn = pad(n);
    float2 r1[9];
    if (PERNODE0) {
      ck_node_ff<N>(sp, sT0, n % N, (n / N) % N, n / (N * N), c2, r1);
    } else {
      float2 g[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) g[c] = sacc[c * S + pn];
      eo_pointwise_ff(g, c2[0], c2[1], c2[2], c2[3], r1);
    }
#pragma unroll
    for (int s = 0; s < M; ++s) {
      gpark[n * M + s] = ff::add(sp[s * S + pn], r1[s]);  // r_0 + r_1
      r[j][s] = r1[s].x;
    }
  }
  bulk::fence_global_writes();  // the parked values are read back by a bulk copy
  __syncthreads();  // every float-float read is done
  float acc[NODES][M];
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * USE;
#pragma unroll
    for (int s = 0; s < M; ++s) acc[j][s] = 0.f;
    if (tid >= USE || n >= N3) continue;
    const int pn = pad(n);
#pragma unroll
    for (int s = 0; s < M; ++s) spf[s * S + pn] = r[j][s];
  }
  __syncthreads();

  // steps 1 .. N-1 in FP32
  for (int k = 1; k < N; ++k) {
    eo32_passes<N, QPT>(spf, spart, sTf + k * ST32, tid, USE);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
      const int n = tid + j * USE;
      if (tid >= USE || n >= N3) continue;
      const int pn = pad(n);
      float g[9], rn[9];
      eo32_gather(spart, S, pn, g);
      eo_pointwise32(g, cf[j][0], cf[j][1], cf[j][2], cf[j][3], rn);
#pragma unroll
      for (int s = 0; s < M; ++s) {
        acc[j][s] += rn[s];
        if (k + 1 < N) spf[s * S + pn] = rn[s];
      }
    }
    __syncthreads();
  }

  // time average (r_0 + r_1 plus the FP32 tail) in float-float, then the
  // faces; the parked r_0 + r_1 comes back in one bulk copy into the
  // accumulator half (the partial arrays there are dead; sp is not touched)
  const float2* park = gpark;
  if (!PERNODE0 && bulk::can_copy(gpark, 8u * M * N3)) {
    bulk::fence_shared();
    __syncthreads();
    if (tid == 0) bulk::start(stage, gpark, 8u * M * N3, &s_bar);
    if (!bulk::wait(&s_bar, bparity) && tid == 0) atomicOr(status, 1u);
    bparity ^= 1u;
    park = reinterpret_cast<const float2*>(stage);
  }
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * USE;
    if (tid >= USE || n >= N3) continue;
    const int pn = pad(n);
    float2 pk[M];  // the parked r_0 + r_1 first (all loads in flight), then the sums
#pragma unroll
    for (int s = 0; s < M; ++s) pk[s] = park[n * M + s];
#pragma unroll
    for (int s = 0; s < M; ++s) {
      const float2 v = ff::add(pk[s], make_float2(acc[j][s], 0.f));
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

template <int N, int NT, int USE, int QPT, int MINB, bool PERNODE0>
cudaError_t launch_fp32_eo(int64_t E, const double* q, const double* params, double* out_avg,
                           double* out_faces, const double* tables, unsigned int* status,
                           cudaStream_t stream) {
  constexpr size_t smem = EoFfShape<N, PERNODE0>::SMEM;
  static_assert(smem <= 232448, "shared memory budget of one CTA exceeded");
  static_assert(USE <= NT && NT <= 1024, "bad thread counts");
  auto kern = fp32_eo_kernel<N, NT, USE, QPT, MINB, PERNODE0>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (E > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (E == 0) return cudaSuccess;
  kern<<<(unsigned)E, NT, smem, stream>>>(q, params, out_avg, out_faces, tables, E, status);
  return cudaGetLastError();
}

}  // namespace

// Launch shape per N: (N, threads, working threads, quantities per FP32 line
// task, CTAs per SM the registers are sized for, step 0 node by node).
#define STP_FP32_SHAPES(X)                                                                        \
  X(2, 32, 24, 1, 16, false) X(3, 32, 27, 2, 16, false) X(4, 96, 96, 1, 8, false)                \
  X(5, 160, 150, 1, 6, false) X(6, 256, 216, 1, 1, false) X(7, 160, 147, 2, 4, false)            \
  X(8, 384, 384, 1, 2, false) X(9, 768, 729, 1, 1, false) X(10, 1024, 1000, 2, 1, false)         \
  X(11, 384, 363, 2, 1, false) X(12, 448, 432, 2, 1, true)

cudaError_t launch_fp32(int N, int64_t E, const double* q, const double* params, double* out_avg,
                        double* out_faces, const double* tables, unsigned int* status,
                        cudaStream_t stream) {
  switch (N) {
#define X(n, nt, use, qpt, minb, pn0) \
  case n: return launch_fp32_eo<n, nt, use, qpt, minb, pn0>(E, q, params, out_avg, out_faces, tables, status, stream);
    STP_FP32_SHAPES(X)
#undef X
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace stp
