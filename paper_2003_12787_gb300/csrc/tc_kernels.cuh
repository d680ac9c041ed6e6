// Space-Time Predictor with the derivative contractions on the tensor cores
// (tcgen05.mma, accumulators in TMEM) and the precision of every Taylor term
// chosen from its size (precisions STP_PRECISION_BF16X2/X3, FP16X2/X3).
//
// Taylor bookkeeping as in the other kernels: r_0 = q, r_{k+1} = dt/(k+2) L r_k,
// avg = sum_{k=0..N} r_k (Eq. (exahypeTimeAverage) divided by dt). Term r_k
// enters the average with the weight dt^k/(k+1)! already folded in, so the
// error a step may make is set by rho_k = max|r_k| / max|r_0 + r_1|: each
// derivative order is kept in range by that rescaling, and its precision is
// chosen from it, per element:
//   * float-float (about 48 bits, ff32.cuh) on the CUDA cores while
//     rho_k > 1e-3: always the first step (r_1), and the next ones on
//     coarse fields, where later terms stay large;
//   * from the first step with rho_k <= 1e-3 on, the contraction of the
//     three directions runs on the tensor cores with r_k split into T
//     BF16 or FP16 slices: T = 3 while rho_k > 1e-6, 2 while rho_k > 3e-9,
//     then 1 (the x2 variants cap T at 2); every slice product with
//     s + t < T accumulates in FP32 in TMEM; the pointwise elastic update and
//     the running sum of these terms are FP32.
// The average (float-float part plus the FP32 tail) and the face projections
// of Sec. II-B are formed in float-float and returned as doubles.
//
// Tensor-core step (one CTA per element). Each thread owns x-adjacent node
// pairs (x0 = 2j, x0 + 1), so one cvt.rn.bf16x2 of a quantity yields the
// 32-bit word of the pair for every direction that differentiates it:
//   pass x: A[row = (q6, z, y)][k = x]  K-major   (pair adjacent along K)
//   pass y: A[row = (q6, z, x)][k = y]  MN-major  (pair adjacent along M)
//   pass z: A[row = (q6, y, x)][k = z]  MN-major
// (row = q6 * RQ + line within the quantity, RQ = N^2 rounded up to 8, so
// the byte offset of a thread's word is one per-thread base per pass plus a
// constant per quantity)
// with B = the split derivative matrix (K-major, [i][l]); the 6N^2 rows of a
// pass form 128-row tiles, one M128 x N16 x K16 accumulator per tile and pass
// in TMEM (32 columns: the products with B_0, and those with B_1, B_2, which
// readback adds). Slice levels are staged into NBUF buffers; one thread issues
// the MMAs of a level for all passes and tiles - A_t against [B_0; B_1] as
// one N = 32 product where both pairs are needed - and commits them to the
// buffer's mbarrier while the next level is staged. The results are read from TMEM by
// lane (= line) and stored to 18 partial-derivative arrays (pass, quantity),
// which the pointwise update gathers per node. All mbarrier waits are bounded;
// a wait that gives up sets bit 0 of the status word, and bit 2 when the
// tensor cores were still not drained at the end (results of the context are
// then not to be trusted).
//
// The contraction-as-small-GEMM view is the paper's loop-over-GEMM (Sec. III)
// with the dimension splitting and on-the-fly time integration of SplitCK
// (Sec. IV); the transposition of the element on entry and exit follows
// Sec. V-B.
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
using mixed::tile_offset;
using mixed::tmem_alloc;
using mixed::tmem_dealloc;
using mixed::tmem_ld16;
using mixed::umma_commit;
using mixed::umma_desc;
using mixed::umma_f16;

constexpr float kRhoFF = 1e-3f;   // float-float above this term ratio
constexpr float kRho3 = 1e-6f;    // three slices above this
constexpr float kRho2 = 3e-9f;    // two slices above this, one below
constexpr int kScale = 14;        // largest scaled magnitude just below 2^14

template <int N, int TMAX, int NT, int NBUF>
struct TcShape {
  static constexpr bool PERNODE = N >= 12;  // float-float steps node by node
  using Ff = EoFfShape<N, PERNODE>;
  static constexpr int N3 = N * N * N;
  static constexpr int RX = Ff::RX, PLANE = Ff::PLANE, S = Ff::S, LDD = Ff::LDD;
  static constexpr int HP2 = (N + 1) / 2;          // node pairs per x line
  static constexpr int PAIRS = N * N * HP2;
  static constexpr int NPAIR = (PAIRS + NT - 1) / NT;
  static constexpr int NODES_FF = (N3 + NT - 1) / NT;
  // rows of one pass: six blocks of N^2 lines, each padded to a multiple of 8
  // rows so that a quantity's block starts on a core-matrix boundary
  static constexpr int RQ = (N * N + 7) & ~7;
  static constexpr int ROWS = 6 * RQ;
  static constexpr int TILES = (ROWS + 127) / 128;
  // per pass and tile 32 columns: products with B_0 in the first 16, with
  // B_1 and B_2 in the second 16 (added at readback)
  static constexpr int TMEM_USED = 3 * TILES * 32;
  static constexpr int TMEM_COLS = TMEM_USED <= 32 ? 32 : TMEM_USED <= 64 ? 64 : TMEM_USED <= 128 ? 128
                                 : TMEM_USED <= 256 ? 256 : 512;
  // float-float tables of every step: even-odd (or, node by node, N x LDD)
  static constexpr int FT = PERNODE ? N * LDD : Ff::STEP_TABLE;
  // region shared by the phases (bytes)
  static constexpr size_t FF_BYTES = sizeof(float2) * (size_t)(N * FT + (PERNODE ? 9 : 18) * S);
  static constexpr size_t LEVEL_BYTES = (size_t)3 * TILES * 4096;
  static constexpr size_t TC_BYTES = NBUF * LEVEL_BYTES + sizeof(float) * (size_t)18 * S;
  static constexpr size_t REGION = ((FF_BYTES > TC_BYTES ? FF_BYTES : TC_BYTES) + 1023) & ~(size_t)1023;
  // fixed part: B slices [TMAX][512], phi (float-float) [2N], maxima [2][9],
  // amax, readback factors [18], mbarriers [NBUF], TMEM address
  static constexpr size_t B_OFF = REGION;
  static constexpr size_t PHI_OFF = B_OFF + (size_t)TMAX * 512;
  static constexpr size_t MAX_OFF = PHI_OFF + sizeof(float2) * 2 * N;
  static constexpr size_t AMAX_OFF = MAX_OFF + sizeof(unsigned) * 18;
  static constexpr size_t SFAC_OFF = AMAX_OFF + sizeof(unsigned);
  static constexpr size_t BAR_OFF = (SFAC_OFF + sizeof(float) * 18 + 15) & ~(size_t)15;
  static constexpr size_t TADDR_OFF = BAR_OFF + 8 * NBUF;
  static constexpr size_t SMEM = TADDR_OFF + 16 + 1024;  // + slack to align the base to 1 KB
  static_assert(NBUF >= 1 && NBUF <= TMAX, "one to TMAX slice buffers");
  static_assert(SMEM <= 232448, "shared memory budget of one CTA exceeded");
};

// Packed round-to-nearest conversion of (lo, hi) to two 16-bit values: the
// 32-bit word (lo in the low half) and the two values back in FP32.
template <bool FP16>
__device__ __forceinline__ uint32_t cvt_pair(float lo, float hi, float* blo, float* bhi) {
  if (FP16) {
    const __half2 h = __floats2half2_rn(lo, hi);
    const float2 f = __half22float2(h);
    *blo = f.x;
    *bhi = f.y;
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    const float2 f = __bfloat1622float2(h);
    *blo = f.x;
    *bhi = f.y;
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}

// Byte offset of (row, k) of pass p in its tile set (tiles of 128 rows x 16
// K, 4096 B each; core matrices of 8 x 16 B, K-groups 128 B apart, row groups
// 256 B apart). Pass 0 is K-major (16 bytes hold 8 consecutive k of a row),
// passes 1, 2 MN-major (16 bytes hold 8 consecutive rows of one k).
// (tile m = row / 128 at 4096 m, so the row-group term is (row / 8) * 256.)
__device__ __forceinline__ int a_offset(int pass, int row, int k) {
  const int base = (row >> 3) * 256 + (k >> 3) * 128;
  return pass == 0 ? base + (row & 7) * 16 + (k & 7) * 2 : base + (k & 7) * 16 + (row & 7) * 2;
}

// Passes that differentiate quantity s and the row quantity index q6 it has
// there (-1: not used by that pass); q6 order of pass_qty in mixed_kernels.cuh.
__host__ __device__ constexpr int q6_of(int pass, int s) {
  return s < 3 ? 3 + s
       : pass == 0 ? (s == kS11 ? 0 : s == kS12 ? 1 : s == kS13 ? 2 : -1)
       : pass == 1 ? (s == kS12 ? 0 : s == kS22 ? 1 : s == kS23 ? 2 : -1)
                   : (s == kS13 ? 0 : s == kS23 ? 1 : s == kS33 ? 2 : -1);
}

template <int N, int TMAX, bool FP16, int NT, int NBUF, int MINB>
__global__ void __launch_bounds__(NT, MINB)
tc_stp_kernel(const double* __restrict__ q, const double* __restrict__ params,
              double* __restrict__ out_avg, double* __restrict__ out_faces,
              const double* __restrict__ tables, const double* __restrict__ Dref,
              float dt_over_dx, int eD, int64_t E, unsigned int* __restrict__ status) {
  using Sh = TcShape<N, TMAX, NT, NBUF>;
  static_assert(!Sh::PERNODE, "orders with float-float steps node by node use the other kernel");
  static_assert(NT % 128 == 0, "whole warpgroups: every TMEM lane quarter has readers");
  static_assert(Sh::NPAIR == 1, "one node pair per thread");
  static_assert(NT - 1 >= Sh::PAIRS, "the issuing thread owns no node pair");
  constexpr int ISSUER = NT - 1;  // issues and waits for the MMAs; stages nothing
  constexpr int N3 = Sh::N3, S = Sh::S, RX = Sh::RX, PLANE = Sh::PLANE, FT = Sh::FT;
  constexpr int M = kQuantities, TILES = Sh::TILES, RQ = Sh::RQ, HP2 = Sh::HP2;
  constexpr int PAIRS = Sh::PAIRS, NODES = Sh::NODES_FF;
  constexpr size_t LEVEL = Sh::LEVEL_BYTES;
  auto pad = [](int n) { return (n / (N * N)) * PLANE + ((n / N) % N) * RX + n % N; };

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float2* sTf = reinterpret_cast<float2*>(smem);   // float-float phase: [N][FT] step tables
  float2* sp = sTf + N * FT;                       //   state [9][S]; the average at the end
  float2* sacc = sp + M * S;                       //   accumulators [9][S]
  unsigned char* Abuf = smem;                      // tensor-core phase: [NBUF][3][TILES][4096]
  float* spart = reinterpret_cast<float*>(smem + NBUF * LEVEL);  // [18][S]
  unsigned char* Bt = smem + Sh::B_OFF;
  float2* sPhi = reinterpret_cast<float2*>(smem + Sh::PHI_OFF);
  unsigned* smax = reinterpret_cast<unsigned*>(smem + Sh::MAX_OFF);  // [2][9] float bits
  unsigned* samax = reinterpret_cast<unsigned*>(smem + Sh::AMAX_OFF);
  float* sfac = reinterpret_cast<float*>(smem + Sh::SFAC_OFF);  // [18] readback factors
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Sh::BAR_OFF);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(smem + Sh::TADDR_OFF);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t e = blockIdx.x;
  if (e >= E) return;  // the grid is exactly E blocks; kept as a guard

  if (warp == 0) {
    tmem_alloc(taddr_s, Sh::TMEM_COLS);
    tc_fence_before();
  }
  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < NBUF; ++b) mbar_init(bar + b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < N * FT; i += NT) {
    const int k = i / FT;
    sTf[i] = ff::split(eo_table_entry<N>(tables + k * N * N, i - k * FT));
  }
  for (int i = tid; i < 2 * N; i += NT) sPhi[i] = ff::split(tables[N3 + i]);
  if (tid < 18) smax[tid] = 0u;
  if (tid == 0) *samax = 0u;
  // B_t[i][l]: slice t of D[i][l] 2^(kScale - eD), zero padded to 16 x 16
  {
    const double sD = ldexp(1.0, kScale - eD);
    for (int i = tid; i < 256; i += NT) {
      const int n = i >> 4, l = i & 15;
      double rem = (n < N && l < N) ? Dref[n * N + l] * sD : 0.0;
#pragma unroll
      for (int t = 0; t < TMAX; ++t) {
        float back;
        const uint16_t bits = mixed::to_bits<FP16>((float)rem, &back);
        *reinterpret_cast<uint16_t*>(Bt + t * 512 + tile_offset(n, l)) = bits;
        rem -= (double)back;
      }
    }
  }
  const int sc = load_state_ff<N, NT>(q + e * (int64_t)(M * N3), sp);  // ends with a barrier
  tc_fence_after();
  const uint32_t tmem = *taddr_s;
  double* gavg = out_avg + e * (int64_t)(M * N3);
  float2* gpark = reinterpret_cast<float2*>(gavg);  // float-float partial sum of the average
  const double* pe = params + e * (int64_t)(kParams * N3);

  // ---- float-float steps: r_1 always, then while rho_k > kRhoFF ----
  float2 cf2[NODES][4];  // coefficients of the owned nodes, formed once
#pragma unroll
  for (int j = 0; j < NODES; ++j) {
    const int n = tid + j * NT;
    if (n < N3) elastic_coefficients_ff(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2), cf2[j]);
  }
  int k = 0;
  bool to_tc = false;
  for (; k < N; ++k) {
    if (k >= 1) {  // the same decision in every thread (shared values)
      float m = 0.f;
#pragma unroll
      for (int s = 0; s < M; ++s) m = fmaxf(m, __uint_as_float(smax[9 * (k & 1) + s]));
      if (!(m > kRhoFF * __uint_as_float(*samax))) {
        to_tc = true;
        break;
      }
    }
    if (tid < 9) smax[9 * ((k + 1) & 1) + tid] = 0u;
    const float2* T = sTf + k * FT;
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
      eo_pass_ff<N>(sp, sacc, T, pass, tid, NT);
      __syncthreads();
    }
    float lm[9], am = 0.f;
#pragma unroll
    for (int s = 0; s < M; ++s) lm[s] = 0.f;
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
      const int n = tid + j * NT;
      if (n >= N3) continue;
      const int pn = pad(n);
      float2 g[9], r1[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) g[c] = sacc[c * S + pn];
      eo_pointwise_ff(g, cf2[j][0], cf2[j][1], cf2[j][2], cf2[j][3], r1);
#pragma unroll
      for (int s = 0; s < M; ++s) {
        if (k == 0) {
          const float2 v = ff::add(sp[s * S + pn], r1[s]);  // r_0 + r_1
          gpark[n * M + s] = v;
          am = fmaxf(am, fabsf(v.x));
        } else {
          gpark[n * M + s] = ff::add(gpark[n * M + s], r1[s]);
        }
        lm[s] = fmaxf(lm[s], fabsf(r1[s].x));
        sp[s * S + pn] = r1[s];  // every read of p is done (barrier after the z pass)
      }
    }
    {
      // maxima of the new term (nonnegative floats compare as their bits)
#pragma unroll
      for (int s = 0; s < M; ++s) {
        const unsigned v = __reduce_max_sync(0xffffffffu, __float_as_uint(lm[s]));
        if (lane == 0) atomicMax(smax + 9 * ((k + 1) & 1) + s, v);
      }
      if (k == 0) {
        const unsigned v = __reduce_max_sync(0xffffffffu, __float_as_uint(am));
        if (lane == 0) atomicMax(samax, v);
      }
    }
    __syncthreads();
  }

  // ---- tensor-core steps ----
  const int p = tid;  // the thread's node pair (z, y, x0 .. x0 + 1)
  const bool has_pair = p < PAIRS;
  const int pz = p / (N * HP2), py = (p / HP2) % N, px = 2 * (p % HP2);
  float tail[2][9];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int s = 0; s < M; ++s) tail[h][s] = 0.f;
  if (to_tc) {
    float r[2][9], cf[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int x = px + h;
      const bool live = has_pair && x < N;
      const int n = (pz * N + py) * N + x;
      float2 c2[4];
      if (live) elastic_coefficients_ff(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2), c2);
#pragma unroll
      for (int c = 0; c < 4; ++c) cf[h][c] = live ? c2[c].x : 0.f;
#pragma unroll
      for (int s = 0; s < M; ++s) r[h][s] = live ? sp[s * S + pz * PLANE + py * RX + x].x : 0.f;
    }
    const float amax = __uint_as_float(*samax);
    __syncthreads();  // the state is in registers: the region becomes operand tiles
    for (int i = tid; i < (int)(NBUF * LEVEL / 16); i += NT)
      reinterpret_cast<uint4*>(Abuf)[i] = make_uint4(0u, 0u, 0u, 0u);  // padding reads as zero
    __syncthreads();
    constexpr uint32_t idK = mixed::umma_idesc_m128_n16(FP16 ? 0u : 1u);
    constexpr uint32_t idMN = idK | (1u << 15);  // A transposed: MN-major
    // the same with N = 32: B = [B_s; B_s+1] (consecutive 512-byte slices form
    // one 32-row K-major operand with 256-byte row groups)
    constexpr uint32_t idK32 = (idK & ~(0x3Fu << 17)) | ((32u >> 3) << 17);
    constexpr uint32_t idMN32 = idK32 | (1u << 15);
    uint32_t phase = 0u, pending = 0u;  // bit b: parity to wait for / commit outstanding on buffer b
    // byte offsets of the thread's words in the tiles of each pass (row block
    // of quantity 0; quantity q6 adds q6 * RQ / 8 row groups)
    const int off0 = a_offset(0, pz * N + py, px);
    const int off1 = a_offset(1, pz * N + px, py), off1b = a_offset(1, pz * N + px + 1, py);
    const int off2 = a_offset(2, py * N + px, pz), off2b = a_offset(2, py * N + px + 1, pz);
    bool ok = true;
    for (; k < N; ++k) {
      float mq[9], m = 0.f;
#pragma unroll
      for (int s = 0; s < M; ++s) {
        mq[s] = __uint_as_float(smax[9 * (k & 1) + s]);
        m = fmaxf(m, mq[s]);
      }
      int T = m > kRho3 * amax ? 3 : (m > kRho2 * amax ? 2 : 1);
      T = T > TMAX ? TMAX : T;
      float rem[2][9];
#pragma unroll
      for (int s = 0; s < M; ++s) {
        // binary exponent e of the maximum (max = m 2^e, m in [0.5, 1)), kept
        // >= -100 so that 2^(kScale - e) is a normal FP32 number
        const int bits = __float_as_int(mq[s]);
        int es = bits == 0 ? 0 : ((bits >> 23) & 0xff) - 126;
        es = es < -100 ? -100 : es;
        const float scl = __int_as_float((127 + kScale - es) << 23);
        rem[0][s] = r[0][s] * scl;
        rem[1][s] = r[1][s] * scl;
      }
      if (tid < 18) {  // factor turning a tensor-core result of (pass, q6) into the step's derivative
        const int bits = (int)smax[9 * (k & 1) + eo_qty(tid / 6, tid % 6)];
        int es = bits == 0 ? 0 : ((bits >> 23) & 0xff) - 126;
        es = es < -100 ? -100 : es;
        sfac[tid] = ldexpf(dt_over_dx / (float)(k + 2), es + eD - 2 * kScale);
      }
      if (tid < 9) smax[9 * ((k + 1) & 1) + tid] = 0u;  // the other buffer: no reader left
#pragma unroll 1
      for (int t = 0; t < T; ++t) {
        const int b = t % NBUF;
        if (pending & (1u << b)) {
          // the MMAs that last read this buffer must be done: one thread waits
          // (bounded), the others wait at the barrier without polling
          bool okb = true;
          if (tid == ISSUER) okb = mbar_wait(bar + b, (phase >> b) & 1u);
          if (!__syncthreads_and(okb ? 1 : 0)) {  // still pending: drained at the end
            ok = false;
            break;
          }
          phase ^= 1u << b;
          pending &= ~(1u << b);
        }
        unsigned char* Ab = Abuf + b * LEVEL;
        if (has_pair) {
#pragma unroll
          for (int s = 0; s < M; ++s) {
            float b0, b1;
            const uint32_t w = cvt_pair<FP16>(rem[0][s], rem[1][s], &b0, &b1);
            rem[0][s] -= b0;
            rem[1][s] -= b1;
#pragma unroll
            for (int pass = 0; pass < 3; ++pass) {
              const int q6 = q6_of(pass, s);
              if (q6 < 0) continue;
              unsigned char* At = Ab + pass * TILES * 4096 + q6 * (RQ / 8) * 256;
              if (pass == 0) {
                *reinterpret_cast<uint32_t*>(At + off0) = w;
              } else {
                const int o = pass == 1 ? off1 : off2, ob = pass == 1 ? off1b : off2b;
                // the pair is 4-byte aligned and in one core matrix when its
                // first row is even (always for even N)
                const int r0 = pass == 1 ? pz * N + px : py * N + px;
                if ((N & 1) == 0 || (px + 1 < N && (r0 & 1) == 0)) {
                  *reinterpret_cast<uint32_t*>(At + o) = w;
                } else {
                  *reinterpret_cast<uint16_t*>(At + o) = (uint16_t)(w & 0xffffu);
                  if (px + 1 < N) *reinterpret_cast<uint16_t*>(At + ob) = (uint16_t)(w >> 16);
                }
              }
            }
          }
        }
        fence_async_smem();
        __syncthreads();
        if (tid == ISSUER) {  // the next level is staged meanwhile by the other threads
          tc_fence_after();
          // descriptors advance by (byte offset >> 4) in their 14-bit address
          // field; shared-memory addresses stay below 2^18, so no carry
          const uint64_t a0 = umma_desc(smem_u32(Ab), 128, 256);
          const uint64_t b0 = umma_desc(smem_u32(Bt), 128, 256);
#pragma unroll
          for (int pass = 0; pass < 3; ++pass)
#pragma unroll
            for (int mt = 0; mt < TILES; ++mt) {
              const uint64_t ad = a0 + (uint64_t)((pass * TILES + mt) * (4096 >> 4));
              const uint32_t dcol = tmem + (uint32_t)((pass * TILES + mt) * 32);
              const uint32_t i16 = pass == 0 ? idK : idMN, i32 = pass == 0 ? idK32 : idMN32;
              // slice pairs (t, u) with t + u < T: columns 0..15 collect the
              // products with B_0, columns 16..31 those with B_1 and B_2
              if (T - t >= 2) {  // A_t [B_0; B_1], N = 32
                umma_f16(dcol, ad, b0, i32, t == 0 ? 0u : 1u);
                if (T - t == 3)  // A_t B_2 into the second half
                  umma_f16(dcol + 16, ad, b0 + (uint64_t)(1024 >> 4), i16, 1u);
              } else {  // A_t B_0 only
                umma_f16(dcol, ad, b0, i16, t == 0 ? 0u : 1u);
              }
            }
          umma_commit(bar + b);
        }
        pending |= 1u << b;
      }
      if (!ok) break;
      // every MMA of the step is done when the last commit has arrived; the
      // other buffers' phases are consumed too, so the parities stay in step
      bool okw = true;
#pragma unroll
      for (int b = 0; b < NBUF; ++b)
        if (tid == ISSUER && (pending & (1u << b))) okw = mbar_wait(bar + b, (phase >> b) & 1u) && okw;
      if (!__syncthreads_and(okw ? 1 : 0)) {
        ok = false;
        break;
      }
      phase ^= pending;
      pending = 0u;
      tc_fence_after();
      // results: warp w reads lane quarter w % 4 of the tiles w / 4, w / 4 + NT / 128, ...
      for (int j = warp >> 2; j < 3 * TILES; j += NT / 128) {
        const int quarter = warp & 3;
        float v[16], v1[16];
        const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(j * 32);
        tmem_ld16(ta, v);
        tmem_ld16(ta + 16, v1);
        if (T >= 2) {  // the second half holds the products with B_1, B_2
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = v1[i] + v[i];
        }
        const int pass = j / TILES;
        const int row = (j - pass * TILES) * 128 + quarter * 32 + lane;
        const int q6 = row / RQ, rr = row - q6 * RQ;
        if (q6 < 6 && rr < N * N) {  // a line (not padding)
          const int a = rr / N, bb = rr - a * N;
          const float f = sfac[pass * 6 + q6];
          float* dst = spart + (pass * 6 + q6) * S;
          int base, stride;
          if (pass == 0) { base = a * PLANE + bb * RX; stride = 1; }
          else if (pass == 1) { base = a * PLANE + bb; stride = RX; }
          else { base = a * RX + bb; stride = PLANE; }
#pragma unroll
          for (int i = 0; i < N; ++i) dst[base + i * stride] = f * v[i];
        }
      }
      tc_fence_before();
      __syncthreads();
      // pointwise update of the two owned nodes
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
        if (lane == 0) atomicMax(smax + 9 * ((k + 1) & 1) + s, v);
      }
      __syncthreads();
    }
    if (!ok) {
      // a bounded wait gave up: report it, give the tensor cores one more
      // bounded wait, and flag the context if they are still not drained
      if (tid == ISSUER) {
        bool drained = true;
#pragma unroll
        for (int b = 0; b < NBUF; ++b)
          if (pending & (1u << b)) drained = mbar_wait(bar + b, (phase >> b) & 1u) && drained;
        atomicOr(status, drained ? 1u : 5u);
      }
    }
  }
  tc_fence_before();
  __syncthreads();  // operand tiles and partials are dead: the average goes to sp
  if (warp == 0) tmem_dealloc(tmem, Sh::TMEM_COLS);

  // ---- time average (float-float part + FP32 tail) and faces ----
  if (to_tc) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int x = px + h;
      if (!has_pair || x >= N) continue;
      const int n = (pz * N + py) * N + x, pn = pz * PLANE + py * RX + x;
#pragma unroll
      for (int s = 0; s < M; ++s) {
        const float2 v = ff::add(gpark[n * M + s], make_float2(tail[h][s], 0.f));
        sp[s * S + pn] = v;
        gavg[n * M + s] = ff::to_double(v, sc);
      }
    }
  } else {
    for (int n = tid; n < N3; n += NT) {
      const int pn = pad(n);
#pragma unroll
      for (int s = 0; s < M; ++s) {
        const float2 v = gpark[n * M + s];
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

template <int N, int TMAX, bool FP16, int NT, int NBUF, int MINB>
cudaError_t launch_tc(int64_t E, const double* q, const double* params, double* out_avg,
                      double* out_faces, const double* tables, const double* Dref,
                      double dt_over_dx, int eD, unsigned int* status, cudaStream_t stream) {
  using Sh = TcShape<N, TMAX, NT, NBUF>;
  auto kern = tc_stp_kernel<N, TMAX, FP16, NT, NBUF, MINB>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
  if (err != cudaSuccess) return err;
  if (E > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (E == 0) return cudaSuccess;
  kern<<<(unsigned)E, NT, Sh::SMEM, stream>>>(q, params, out_avg, out_faces, tables, Dref,
                                              (float)dt_over_dx, eD, E, status);
  return cudaGetLastError();
}

// Launch shape per order: (N, threads, slice buffers for three slices, CTAs
// per SM the registers are sized for). Threads: at least the 6 N^2 line
// tasks of a float-float pass (one task per thread) and the N^2 ceil(N/2)
// node pairs, in whole warpgroups.
template <int N>
struct TcLaunch;
#define STP_TC_SHAPES(X) \
  X(2, 128, 3, 4) X(3, 128, 3, 4) X(4, 128, 3, 4) X(5, 256, 3, 2) X(6, 256, 3, 2) \
  X(7, 384, 3, 1) X(8, 384, 3, 1) X(9, 512, 2, 1) X(10, 640, 2, 1)
#define X(n_, nt_, nbuf_, minb_)                 \
  template <>                                   \
  struct TcLaunch<n_> {                         \
    static constexpr int NT = nt_, NBUF3 = nbuf_, MINB = minb_; \
  };
STP_TC_SHAPES(X)
#undef X

template <int N>
cudaError_t launch_tc_n(int variant, int64_t E, const double* q, const double* params,
                        double* out_avg, double* out_faces, const double* tables,
                        const double* Dref, double dt_over_dx, int eD, unsigned int* status,
                        cudaStream_t stream) {
  using L = TcLaunch<N>;
  constexpr int NB2 = L::NBUF3 < 2 ? L::NBUF3 : 2;
  switch (variant) {
    case 1: return launch_tc<N, 2, false, L::NT, NB2, L::MINB>(E, q, params, out_avg, out_faces, tables, Dref, dt_over_dx, eD, status, stream);
    case 2: return launch_tc<N, 3, false, L::NT, L::NBUF3, L::MINB>(E, q, params, out_avg, out_faces, tables, Dref, dt_over_dx, eD, status, stream);
    case 3: return launch_tc<N, 2, true, L::NT, NB2, L::MINB>(E, q, params, out_avg, out_faces, tables, Dref, dt_over_dx, eD, status, stream);
    case 4: return launch_tc<N, 3, true, L::NT, L::NBUF3, L::MINB>(E, q, params, out_avg, out_faces, tables, Dref, dt_over_dx, eD, status, stream);
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
