// Space-Time Predictor with the derivative contractions of the later Taylor
// terms on the tensor cores (tcgen05.mma, accumulators in TMEM); precisions
// STP_PRECISION_FP16X2/X3 and BF16X2/X3, 2 <= N <= 10.
//
// Taylor bookkeeping as in the other kernels: r_0 = q, r_{k+1} = dt/(k+2) L r_k,
// avg = sum_{k=0..N} r_k (Eq. (exahypeTimeAverage) divided by dt).
//
//   * r_1 = dt/2 L q, r_0 + r_1, the time average and the face projections
//     of Sec. II-B in float-float (ff32.cuh) on the CUDA cores, as in the FP32
//     variant: the first term carries the state's full precision.
//   * r_2 .. r_N: the three directional contractions of each step run on the
//     tensor cores as exact integer products. Each quantity of r_k is written
//     in fixed point relative to its largest magnitude and cut into balanced
//     base-2^W digits A_0 + A_1 2^-W + ... (W = 10 for FP16, 8 for BF16;
//     |A_s| <= 2^(W-1), integers, so every digit is an exact 16-bit value);
//     D is cut the same way on the host (make_tc_tiles). A product of two
//     digits is exact in FP32 and so is the whole level-0 sum A_0 B_0 over
//     K <= 16 (|sum| < 2^24): that block of TMEM columns (L0) is exact. The
//     products of the lower levels, scaled by powers of two so that every
//     operand stays a normal 16-bit number, accumulate in FP32 in a second
//     block (h). The step uses the T digits with s + t < T; T is chosen per
//     element and step from rho_k = max|r_k| / max|r_0 + r_1| (r_k already
//     carries dt^k/(k+1)!, so rho_k is the weight of the term's error in the
//     average): more digits while the term is large, one when it is tiny.
//     The pointwise elastic update and the running sum of these terms are
//     FP32.
//
// One CTA per element. Each thread owns an x-adjacent node pair: one packed
// conversion gives the 32-bit word of the pair's digit, stored into the
// operand tile of every pass that differentiates the quantity, digit s at
// k = N s + (position along the line):
//   pass x: A[row = (q6, z, y)][k = N s + x]  K-major
//   pass y: A[row = (q6, z, x)][k = N s + y]  MN-major
//   pass z: A[row = (q6, y, x)][k = N s + z]  MN-major
// (rows padded to 8 per quantity, 128-row x 32-K tiles, no swizzle). So one
// chain of ceil(N T / 16) MMAs per (pass, tile) contracts every digit at
// once against the operand of D for T digits, whose three column blocks of
// N outputs collect L0 = A_0 B_0 (exact), X = the level-1 products and Y =
// the level-2 products (M = 128, N = 16 or 32 columns). Two issuing threads
// in warps of their own take alternate (pass, tile) pairs. The results are
// read from TMEM by lane (= line), combined as L0 + (X + Y) 2^-(W+c) and
// scaled, and stored to 18 partial-derivative arrays (pass, quantity), which
// the pointwise update gathers per node. All mbarrier waits are bounded; a
// wait that gives up sets bit 0 of the status word, and bit 2 when the
// tensor cores were still not drained at the end (results of the context
// are then not to be trusted).
//
// The contraction-as-small-GEMM view is the paper's loop-over-GEMM (Sec. III)
// with the dimension splitting and on-the-fly time integration of SplitCK
// (Sec. IV); the transposition of the element on entry and exit follows
// Sec. V-B. Splitting operands into exactly multiplied integer digits is
// the error-free matrix product of Ozaki, Ogita, Oishi and Rump (2012).
#pragma once
#include "eo_ff.cuh"
#include "mixed_kernels.cuh"

namespace stp {
namespace tc {

using mixed::fence_async_smem;
using mixed::mbar_init;
using mixed::mbar_wait;
using mixed::smem_u32;
using mixed::tc_fence_after;
using mixed::tc_fence_before;
using mixed::tmem_alloc;
using mixed::tmem_dealloc;
using mixed::tmem_ld16;
using mixed::umma_commit;
using mixed::umma_desc;
using mixed::umma_f16;

// Digit type: W bits per digit, c = power-of-two shift of the X and Y
// operands (keeps FP16 values normal), instruction-descriptor format code,
// and the term ratios above which T = 3 and 2 digits are used.
// Float-float steps while max|r_k| > kRhoFF max|r_0 + r_1| (always the first).
constexpr float kRhoFF = 1e-3f;

template <bool BF16>
struct Digits;
template <>
struct Digits<false> {
  static constexpr int W = 10, C = 6;
  static constexpr uint32_t FMT = 0;
  static constexpr float RHO3 = 1e-6f, RHO2 = 1e-9f;
};
template <>
struct Digits<true> {
  static constexpr int W = 8, C = 0;
  static constexpr uint32_t FMT = 1;
  static constexpr float RHO3 = 1e-8f, RHO2 = 1e-10f;
};

// 8-row groups of a digit tile are kGroupBytes apart (see a_offset).
constexpr int kGroupBytes = 528, kTileBytes = 16 * kGroupBytes;

template <int N>
struct TcShape {
  using Ff = EoFfShape<N>;
  static constexpr int N3 = N * N * N, S = Ff::S, RX = Ff::RX, PLANE = Ff::PLANE;
  static constexpr int ST0 = Ff::STEP_TABLE;
  static constexpr int HP2 = (N + 1) / 2;          // node pairs per x line
  static constexpr int PAIRS = N * N * HP2;
  static constexpr int OWN = (PAIRS + 31) & ~31;   // threads of the pair-owning warps
  static constexpr int NT = (OWN + 64 + 127) & ~127;  // + two issuing warps, whole warpgroups
  static constexpr int ISS0 = OWN, ISS1 = OWN + 32;
  static constexpr int CW = 3 * N <= 16 ? 16 : 32;  // TMEM columns of a (pass, tile): [L0 | X | Y]
  static constexpr int RQ = (N * N + 7) & ~7;      // rows of one quantity (multiple of 8)
  static constexpr int TILES = (6 * RQ + 127) / 128;
  static constexpr int COMBOS = 3 * TILES;         // (pass, tile) pairs
  static constexpr int DIG_BYTES = COMBOS * kTileBytes;  // 128 rows x 32 K digits per pair
  static constexpr int TMEM_USED = COMBOS * CW;
  static constexpr int TMEM_COLS = TMEM_USED <= 32 ? 32 : TMEM_USED <= 64 ? 64 : TMEM_USED <= 128 ? 128
                                 : TMEM_USED <= 256 ? 256 : 512;
  // area shared by the phases: float-float p and accumulators of the first
  // step, then the digit tiles and 18 FP32 partial arrays, then the average
  static constexpr size_t FF_BYTES = sizeof(float2) * (size_t)18 * S;
  static constexpr size_t TC_BYTES = (size_t)DIG_BYTES + sizeof(float) * (size_t)18 * S;
  static constexpr size_t AREA = ((FF_BYTES > TC_BYTES ? FF_BYTES : TC_BYTES) + 1023) & ~(size_t)1023;
  static constexpr size_t PART_OFF = (size_t)DIG_BYTES;
  static constexpr size_t TILE_OFF = AREA;         // operands of D for T = 1, 2, 3
  static constexpr size_t T0_OFF = TILE_OFF + (size_t)3 * kTcOperandBytes;
  static constexpr size_t PHI_OFF = T0_OFF + sizeof(float2) * ST0;
  static constexpr size_t MAX_OFF = PHI_OFF + sizeof(float2) * 2 * N;
  static constexpr size_t FAC_OFF = MAX_OFF + sizeof(unsigned) * 20;  // maxima [2][9], amax
  static constexpr size_t BAR_OFF = (FAC_OFF + sizeof(float) * 18 + 15) & ~(size_t)15;
  static constexpr size_t TADDR_OFF = BAR_OFF + 8 * 3;  // one mbarrier per issuer, one for bulk copies
  static constexpr size_t SMEM = TADDR_OFF + 16 + 1024;  // + slack to align the base to 1 KB
  static_assert(SMEM <= 232448, "shared memory budget of one CTA exceeded");
  static_assert(COMBOS >= 2, "one (pass, tile) pair per issuer at least");
  static_assert(3 * N <= 32 && N <= 10, "three digits of a line fit in K = 32");
  static_assert(sizeof(float2) * (size_t)9 * S <= PART_OFF, "the average and the partial area are disjoint");
  static_assert(OWN >= PAIRS && NT <= 1024, "bad thread counts");
};

// Byte offset of (row, k) of pass p in its tile set: tiles of 128 rows x 32
// K; core matrices of 8 x 16 bytes, K groups of 8 128 bytes apart, 8-row
// groups kGroupBytes = 528 bytes apart (512 + 16: consecutive row groups then
// start four banks apart, so the stores of a warp that spans several row
// groups at one k do not collide), so tile m = row / 128 starts at
// kTileBytes m. Pass 0 is K-major (16 bytes hold 8 consecutive k of a row),
// passes 1, 2 MN-major (16 bytes hold 8 consecutive rows of one k). The MMA
// of K chunk c (k = 16 c .. 16 c + 15) starts 256 c bytes into the tile.
__device__ __forceinline__ int a_offset(int pass, int row, int k) {
  const int base = (row >> 3) * kGroupBytes + (k >> 3) * 128;
  return pass == 0 ? base + (row & 7) * 16 + (k & 7) * 2 : base + (k & 7) * 16 + (row & 7) * 2;
}

// Nearest integer of |x| < 2^22, ties to even (two FP32 additions).
__device__ __forceinline__ float round_int(float x) {
  return __fsub_rn(__fadd_rn(x, 12582912.0f), 12582912.0f);  // 1.5 2^23
}

// Row-quantity index of quantity s in pass `pass` (inverse of eo_qty; -1:
// the pass does not differentiate s).
__host__ __device__ constexpr int q6_of(int pass, int s) {
  return s < 3 ? 3 + s
       : pass == 0 ? (s == kS11 ? 0 : s == kS12 ? 1 : s == kS13 ? 2 : -1)
       : pass == 1 ? (s == kS12 ? 0 : s == kS22 ? 1 : s == kS23 ? 2 : -1)
                   : (s == kS13 ? 0 : s == kS23 ? 1 : s == kS33 ? 2 : -1);
}

// Instruction descriptor, kind::f16: D = F32, A = B = fmt, M = 128, N = n,
// A MN-major when mn (bit 15), B K-major.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, uint32_t n, bool mn) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (mn ? (1u << 15) : 0u) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

// Two digits as the packed 16-bit word (lo in the low half); exact.
template <bool BF16>
__device__ __forceinline__ uint32_t pack_digits(float lo, float hi) {
  if (BF16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}

// Binary exponent e of a nonnegative float m (m = f 2^e, f in [0.5, 1)),
// kept >= -100 so the digit scale 2^(W-1-e) stays a normal FP32 number.
__device__ __forceinline__ int max_exponent(float m) {
  const int bits = __float_as_int(m);
  const int e = bits == 0 ? 0 : ((bits >> 23) & 0xff) - 126;
  return e < -100 ? -100 : e;
}

template <int N, bool BF16, int TMAX>
__global__ void __launch_bounds__(TcShape<N>::NT, 1)
tc_stp_kernel(const double* __restrict__ q, const double* __restrict__ params,
              double* __restrict__ out_avg, double* __restrict__ out_faces,
              const double* __restrict__ tables, const unsigned char* __restrict__ tiles,
              float dt_over_dx, int eD, int64_t E, unsigned int* __restrict__ status) {
  using Sh = TcShape<N>;
  using Dg = Digits<BF16>;
  static_assert(TMAX >= 1 && TMAX <= 3, "one to three digits (operands of D exist for T <= 3)");
  constexpr int NT = Sh::NT, N3 = Sh::N3, S = Sh::S, RX = Sh::RX, PLANE = Sh::PLANE;
  constexpr int M = kQuantities, TILES = Sh::TILES, RQ = Sh::RQ, HP2 = Sh::HP2, CW = Sh::CW;
  constexpr int PAIRS = Sh::PAIRS, COMBOS = Sh::COMBOS, W = Dg::W;

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float2* sp = reinterpret_cast<float2*>(smem);    // first step: p[9][S]; the average at the end
  float2* sacc = sp + M * S;                       // first step: accumulators [9][S]
  unsigned char* dig = smem;                       // later steps: digit tiles [COMBOS][kTileBytes]
  float* spart = reinterpret_cast<float*>(smem + Sh::PART_OFF);  // [18][S]
  unsigned char* stile = smem + Sh::TILE_OFF;      // operands of D [T - 1][2 chunks][1024]
  float2* sT0 = reinterpret_cast<float2*>(smem + Sh::T0_OFF);
  float2* sPhi = reinterpret_cast<float2*>(smem + Sh::PHI_OFF);
  unsigned* smax = reinterpret_cast<unsigned*>(smem + Sh::MAX_OFF);  // [2][9] float bits, then amax
  float* sfac = reinterpret_cast<float*>(smem + Sh::FAC_OFF);        // [18] readback factors
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Sh::BAR_OFF);   // [issuer], then bulk copies
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(smem + Sh::TADDR_OFF);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t e = blockIdx.x;
  if (e >= E) return;  // the grid is exactly E blocks; kept as a guard
  const int iss = tid == Sh::ISS0 ? 0 : tid == Sh::ISS1 ? 1 : -1;

  if (warp == 0) {
    tmem_alloc(taddr_s, Sh::TMEM_COLS);
    tc_fence_before();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    bulk::init(bar + 2);  // (fences the three initialisations)
  }
  __syncthreads();  // barriers initialised before the bulk load waits on one
  {  // operands of D for this digit type
    const uint4* gt = reinterpret_cast<const uint4*>(tiles + (BF16 ? 3 * kTcOperandBytes : 0));
    uint4* st = reinterpret_cast<uint4*>(stile);
    for (int i = tid; i < 3 * kTcOperandBytes / 16; i += NT) st[i] = __ldg(gt + i);
  }
  for (int i = tid; i < Sh::ST0; i += NT) sT0[i] = ff::split(eo_table_entry<N>(tables, i));
  for (int i = tid; i < 2 * N; i += NT) sPhi[i] = ff::split(tables[N3 + i]);
  if (tid < 19) smax[tid] = 0u;
  uint32_t bparity = 0u;  // next phase of the bulk-copy barrier
  // the element's AoS state in one bulk copy into the accumulator area (16-byte aligned start)
  double* stage = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(sacc) + 15) & ~(uintptr_t)15);
  const int sc = load_state_ff_bulk<N, NT, S, RX, PLANE>(q + e * (int64_t)(M * N3), sp, stage, bar + 2,
                                                         bparity, status);  // ends with a barrier
  tc_fence_after();
  const uint32_t tmem = *taddr_s;
  double* gavg = out_avg + e * (int64_t)(M * N3);
  float2* gpark = reinterpret_cast<float2*>(gavg);  // r_0 + r_1 in float-float until the end
  const double* pe = params + e * (int64_t)(kParams * N3);

  // ---- float-float steps on the CUDA cores: r_1 always, then while the
  // term is large (rho_k > kRhoFF), where FP32 state and pointwise rounding
  // would show in the average ----
  const int p = tid;  // the thread's node pair (z, y, x0 .. x0 + 1)
  const bool has_pair = p < PAIRS;
  const int pz = p / (N * HP2), py = (p / HP2) % N, px = 2 * (p % HP2);
  float r[2][9], cf[2][4], tail[2][9];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int s = 0; s < M; ++s) {
      r[h][s] = 0.f;
      tail[h][s] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) cf[h][c] = 0.f;
  }
  int k = 0;
#pragma unroll 1
  for (; k < N; ++k) {
    if (k >= 1) {  // the same decision in every thread (shared values)
      float m = 0.f;
#pragma unroll
      for (int s = 0; s < M; ++s) m = fmaxf(m, __uint_as_float(smax[9 * (k & 1) + s]));
      if (!(m > kRhoFF * __uint_as_float(smax[18]))) break;
      for (int i = tid; i < Sh::ST0; i += NT) sT0[i] = ff::split(eo_table_entry<N>(tables + k * N * N, i));
      __syncthreads();
    }
    if (tid < 9) smax[9 * ((k + 1) & 1) + tid] = 0u;  // no reader left of that half
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
      eo_pass_ff<N>(sp, sacc, sT0, pass, tid, NT);
      __syncthreads();
    }
    float lm[9], am = 0.f;
#pragma unroll
    for (int s = 0; s < M; ++s) lm[s] = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int x = px + h;
      if (!has_pair || x >= N) continue;
      const int n = (pz * N + py) * N + x, pn = pz * PLANE + py * RX + x;
      float2 c2[4], g[9], r1[9];
      elastic_coefficients_ff(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2), c2);
#pragma unroll
      for (int c = 0; c < 4; ++c) cf[h][c] = c2[c].x;
#pragma unroll
      for (int c = 0; c < 9; ++c) g[c] = sacc[c * S + pn];
      eo_pointwise_ff(g, c2[0], c2[1], c2[2], c2[3], r1);
#pragma unroll
      for (int s = 0; s < M; ++s) {
        // the average's float-float part, read back by a bulk copy at the end (fence below)
        const float2 v = ff::add(k == 0 ? sp[s * S + pn] : gpark[n * M + s], r1[s]);
        gpark[n * M + s] = v;
        am = fmaxf(am, fabsf(v.x));
        r[h][s] = r1[s].x;
        lm[s] = fmaxf(lm[s], fabsf(r1[s].x));
        sp[s * S + pn] = r1[s];  // every read of p is done (barrier after the z pass)
      }
    }
    // maxima (nonnegative floats compare as their bits): max|r_{k+1}| per
    // quantity, and max|r_0 + r_1| after the first step
#pragma unroll
    for (int s = 0; s < M; ++s) {
      const unsigned v = __reduce_max_sync(0xffffffffu, __float_as_uint(lm[s]));
      if (lane == 0 && v) atomicMax(smax + 9 * ((k + 1) & 1) + s, v);
    }
    if (k == 0) {
      const unsigned va = __reduce_max_sync(0xffffffffu, __float_as_uint(am));
      if (lane == 0 && va) atomicMax(smax + 18, va);
    }
    bulk::fence_global_writes();
    __syncthreads();
  }
  const bool park_bulk = bulk::can_copy(gpark, 8u * M * N3);
  __syncthreads();  // every float-float read is done: the area becomes digit tiles
  for (int i = tid; i < (int)(Sh::PART_OFF / 16); i += NT)
    reinterpret_cast<uint4*>(dig)[i] = make_uint4(0u, 0u, 0u, 0u);  // padding reads as zero
  __syncthreads();
  const float amax = __uint_as_float(smax[18]);

  // ---- the remaining steps on the tensor cores ----
  constexpr uint32_t idK = idesc(Dg::FMT, CW, false), idMN = idesc(Dg::FMT, CW, true);
  uint32_t phase = 0u;  // issuers: parity of the next commit
  // row part of the byte offsets of the pair's word in each pass's tiles,
  // quantity block 0 (a quantity block adds q6 RQ / 8 row groups)
  const int r0row = pz * N + py, r1row = pz * N + px, r2row = py * N + px;
  // the pair is one aligned 32-bit word in pass 1 / 2 when its first row is
  // even (rows r, r + 1 then share an 8-row group)
  const bool w1 = (N & 1) == 0 || ((r1row & 1) == 0 && px + 1 < N);
  const bool w2 = (N & 1) == 0 || ((r2row & 1) == 0 && px + 1 < N);
  bool ok = true;
#pragma unroll 1
  for (; k < N; ++k) {
    float m = 0.f;
    int es[9];
#pragma unroll
    for (int s = 0; s < M; ++s) {
      const float mq = __uint_as_float(smax[9 * (k & 1) + s]);
      m = fmaxf(m, mq);
      es[s] = max_exponent(mq);
    }
    int T = m > Dg::RHO3 * amax ? 3 : m > Dg::RHO2 * amax ? 2 : 1;
    T = T > TMAX ? TMAX : T;
    // fixed point: |r 2^(W-1-e)| < 2^(W-1)
#pragma unroll
    for (int s = 0; s < M; ++s) {
      const float scl = __int_as_float((127 + W - 1 - es[s]) << 23);
      r[0][s] *= scl;
      r[1][s] *= scl;
    }
    if (tid < 18)  // factor turning a result of (pass, q6) into the step's derivative
      sfac[tid] = ldexpf(dt_over_dx / (float)(k + 2), es[eo_qty(tid / 6, tid % 6)] + eD - 2 * (W - 1));
    if (tid < 9) smax[9 * ((k + 1) & 1) + tid] = 0u;  // the other half: no reader left
    if (has_pair) {
#pragma unroll 1
      for (int sd = 0; sd < T; ++sd) {
#pragma unroll
        for (int s = 0; s < M; ++s) {
          const float d0 = round_int(r[0][s]), d1 = round_int(r[1][s]);
          r[0][s] = (r[0][s] - d0) * (float)(1 << W);  // exact: the residual has few bits
          r[1][s] = (r[1][s] - d1) * (float)(1 << W);
          const uint32_t wd = pack_digits<BF16>(d0, d1);
#pragma unroll
          for (int pass = 0; pass < 3; ++pass) {
            const int q6 = q6_of(pass, s);
            if (q6 < 0) continue;
            unsigned char* At = dig + pass * TILES * kTileBytes + q6 * (RQ / 8) * kGroupBytes;
            if (pass == 0) {
              const int kx = N * sd + px;
              if ((kx & 1) == 0) {  // an aligned word within one 8-k group
                *reinterpret_cast<uint32_t*>(At + a_offset(0, r0row, kx)) = wd;
              } else {
                *reinterpret_cast<uint16_t*>(At + a_offset(0, r0row, kx)) = (uint16_t)(wd & 0xffffu);
                *reinterpret_cast<uint16_t*>(At + a_offset(0, r0row, kx + 1)) = (uint16_t)(wd >> 16);
              }
            } else {
              const int row = pass == 1 ? r1row : r2row;
              const int kk = N * sd + (pass == 1 ? py : pz);
              if (pass == 1 ? w1 : w2) {
                *reinterpret_cast<uint32_t*>(At + a_offset(pass, row, kk)) = wd;
              } else {
                *reinterpret_cast<uint16_t*>(At + a_offset(pass, row, kk)) = (uint16_t)(wd & 0xffffu);
                if (px + 1 < N) *reinterpret_cast<uint16_t*>(At + a_offset(pass, row + 1, kk)) = (uint16_t)(wd >> 16);
              }
            }
          }
        }
      }
    }
    fence_async_smem();
    __syncthreads();
    if (iss >= 0) {
      tc_fence_after();
      // descriptors advance by (byte offset >> 4) in their 14-bit address
      // field; shared-memory addresses stay below 2^18, so no carry
      const uint64_t a0 = umma_desc(smem_u32(dig), 128, kGroupBytes);
      const uint64_t b0 = umma_desc(smem_u32(stile + (T - 1) * kTcOperandBytes), 128, 256);
      const int nch = (N * T + 15) / 16;  // K chunks holding the T digits
#pragma unroll 1
      for (int j = iss; j < COMBOS; j += 2) {
        const uint64_t ad = a0 + (uint64_t)(j * (kTileBytes >> 4));
        const uint32_t dcol = tmem + (uint32_t)(j * CW);
        const uint32_t id = j < TILES ? idK : idMN;
        umma_f16(dcol, ad, b0, id, 0u);
        if (nch > 1) umma_f16(dcol, ad + (uint64_t)(256 >> 4), b0 + (uint64_t)(kTcChunkBytes >> 4), id, 1u);
      }
      umma_commit(bar + iss);
    }
    // every MMA of the step is done when both commits have arrived
    bool okw = true;
    if (iss >= 0) {
      okw = mbar_wait(bar + iss, phase);
      phase ^= 1u;
    }
    if (!__syncthreads_and(okw ? 1 : 0)) {
      ok = false;
      break;
    }
    tc_fence_after();
    // results: warp w reads lane quarter w % 4 of the pairs w / 4, w / 4 + NT / 128, ...
    for (int j = warp >> 2; j < COMBOS; j += NT / 128) {
      const int quarter = warp & 3;
      float v[CW];
      const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(j * CW);
      tmem_ld16(ta, v);
      if (CW == 32) tmem_ld16(ta + 16, v + 16);
      const int pass = j / TILES;
      const int row = (j - pass * TILES) * 128 + quarter * 32 + lane;
      const int q6 = row / RQ, rr = row - q6 * RQ;
      if (q6 < 6 && rr < N * N) {  // a line (not padding)
        const int a = rr / N, bb = rr - a * N;
        const float f = sfac[pass * 6 + q6];
        constexpr float hs = 1.0f / (float)(1u << (W + Dg::C));
        float* dst = spart + (pass * 6 + q6) * S;
        int base, stride;
        if (pass == 0) { base = a * PLANE + bb * RX; stride = 1; }
        else if (pass == 1) { base = a * PLANE + bb; stride = RX; }
        else { base = a * RX + bb; stride = PLANE; }
#pragma unroll
        for (int i = 0; i < N; ++i) dst[base + i * stride] = f * fmaf(v[N + i] + v[2 * N + i], hs, v[i]);
      }
    }
    tc_fence_before();
    __syncthreads();
    // pointwise update of the owned nodes
    float lm[9];
#pragma unroll
    for (int s = 0; s < M; ++s) lm[s] = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int x = px + h;
      if (!has_pair || x >= N) continue;
      float g[9], rn[9];
      eo32_gather(spart, S, pz * PLANE + py * RX + x, g);
      eo_pointwise32(g, cf[h][0], cf[h][1], cf[h][2], cf[h][3], rn);
#pragma unroll
      for (int s = 0; s < M; ++s) {
        r[h][s] = rn[s];
        tail[h][s] += rn[s];
        lm[s] = fmaxf(lm[s], fabsf(rn[s]));
      }
    }
#pragma unroll
    for (int s = 0; s < M; ++s) {
      const unsigned v = __reduce_max_sync(0xffffffffu, __float_as_uint(lm[s]));
      if (lane == 0 && v) atomicMax(smax + 9 * ((k + 1) & 1) + s, v);
    }
    __syncthreads();
  }
  if (!ok && iss >= 0) {
    // a bounded wait gave up: report it, give the tensor cores one more
    // bounded wait, and flag the context if they are still not drained
    const bool drained = mbar_wait(bar + iss, phase);
    atomicOr(status, drained ? 1u : 5u);
  }
  tc_fence_before();
  fence_async_smem();  // generic accesses to the area before the bulk copy into it
  __syncthreads();  // digit tiles and partials are dead: the average goes to sp
  if (warp == 0) tmem_dealloc(tmem, Sh::TMEM_COLS);

  // ---- time average (float-float r_0 + r_1 plus the FP32 tail) and faces ----
  {
    // the parked r_0 + r_1 in one bulk copy into the partial-array area (its
    // last readers have passed the barrier above; it does not overlap sp,
    // 72 S <= the digit tiles' bytes), else from global memory
    const float2* pk = gpark;
    if (park_bulk) {
      if (tid == 0) bulk::start(spart, gpark, 8u * M * N3, bar + 2);
      if (!bulk::wait(bar + 2, bparity) && tid == 0) atomicOr(status, 1u);
      bparity ^= 1u;
      pk = reinterpret_cast<const float2*>(spart);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int x = px + h;
      if (!has_pair || x >= N) continue;
      const int n = (pz * N + py) * N + x, pn = pz * PLANE + py * RX + x;
#pragma unroll
      for (int s = 0; s < M; ++s) {
        const float2 v = ff::add(pk[n * M + s], make_float2(tail[h][s], 0.f));
        sp[s * S + pn] = v;
        gavg[n * M + s] = ff::to_double(v, sc);
      }
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
    ff::Dot acc;
#pragma unroll
    for (int i = 0; i < N; ++i) acc.fma(phi[i], sp[s * S + base + i * stride]);
    fe[o] = ff::to_double(acc.value(), sc);
  }
}

template <int N, bool BF16, int TMAX>
cudaError_t launch_tc(int64_t E, const double* q, const double* params, double* out_avg,
                      double* out_faces, const double* tables, const unsigned char* tiles,
                      double dt_over_dx, int eD, unsigned int* status, cudaStream_t stream) {
  using Sh = TcShape<N>;
  auto kern = tc_stp_kernel<N, BF16, TMAX>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
  if (err != cudaSuccess) return err;
  if (E > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (E == 0) return cudaSuccess;
  kern<<<(unsigned)E, Sh::NT, Sh::SMEM, stream>>>(q, params, out_avg, out_faces, tables, tiles,
                                                   (float)dt_over_dx, eD, E, status);
  return cudaGetLastError();
}

// Variants 1..4 = BF16x2, BF16x3, FP16x2, FP16x3: the x3 settings use up to
// three digits (10-bit FP16: stated 1e-9; 8-bit BF16: 5e-9), the x2
// settings cap the digits at two.
template <int N>
cudaError_t launch_tc_n(int variant, int64_t E, const double* q, const double* params,
                        double* out_avg, double* out_faces, const double* tables,
                        const double* Dref, double dt_over_dx, int eD, unsigned int* status,
                        cudaStream_t stream) {
  (void)Dref;
  const unsigned char* tiles = reinterpret_cast<const unsigned char*>(tables + table_offset_tc(N));
  switch (variant) {
    case 1: return launch_tc<N, true, 2>(E, q, params, out_avg, out_faces, tables, tiles, dt_over_dx, eD, status, stream);
    case 2: return launch_tc<N, true, 3>(E, q, params, out_avg, out_faces, tables, tiles, dt_over_dx, eD, status, stream);
    case 3: return launch_tc<N, false, 2>(E, q, params, out_avg, out_faces, tables, tiles, dt_over_dx, eD, status, stream);
    case 4: return launch_tc<N, false, 3>(E, q, params, out_avg, out_faces, tables, tiles, dt_over_dx, eD, status, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tc

// Per-N entry points of the tensor-core precisions, instantiated in
// mixed_n*.cu: the kernel above for N <= 10, the kernel of mixed_kernels.cuh
// for N = 11, 12.
template <int N>
cudaError_t launch_mixed_for(int variant, int64_t E, const double* q, const double* params,
                             double* out_avg, double* out_faces, const double* tables,
                             const double* Dref, double dt_over_dx, int eD, unsigned int* status,
                             cudaStream_t stream) {
  if constexpr (N <= 10)
    return tc::launch_tc_n<N>(variant, E, q, params, out_avg, out_faces, tables, Dref,
                              dt_over_dx, eD, status, stream);
  else
    return mixed::launch_mixed_n<N>(variant, E, q, params, out_avg, out_faces, tables, Dref,
                                    dt_over_dx, eD, status, stream);
}

}  // namespace stp
