// Mixed-precision Space-Time Predictor for sm_103a: derivative contractions
// on the 5th-generation tensor cores (tcgen05.mma, accumulators in TMEM).
// Kernel of the orders N = 11, 12 (where one node pair per thread of the
// kernel in tc_kernels.cuh would not fit the registers); the helpers below
// (descriptors, mbarriers, TMEM) serve both kernels.
//
// Per element (one CTA):
//   1. r_0 = q; the first Cauchy-Kowalewsky term r_1 = dt/2 L q is computed in
//      FP64 with the same DFMA code as the FP64 kernel. It is the dominant
//      time-dependent term, and it is the FP64 correction pass of the series:
//      every later term only enters the average scaled by dt^k/(k+1)!.
//      avg = r_0 + r_1 is written in FP64.
//   2. r_2 .. r_N: each term r_k (FP32) is scaled per quantity by a power of
//      two (largest magnitude just below 2^14), split into T = 2 or 3 BF16 or
//      FP16 slices, and the three directional contractions run as GEMMs on the
//      tensor cores: rows = (quantity, two in-plane indices) lines of the
//      element, K = the contracted index (N padded to 16), N_gemm = the N
//      outputs of a line (padded to 16). The slice products
//      (s, t) with s + t < T accumulate in FP32 in TMEM, smallest first.
//      The pointwise elastic update runs in FP32 on the CUDA cores.
//   3. The FP32 sum of r_2..r_N is added to the FP64 average, and the six face
//      projections are computed from it in FP64.
// The derivative matrix is split the same way (in FP64, once per CTA).
//
// This follows the Taylor form of Eq. (exahypeTimeAverage) with the on-the-fly
// accumulation of Sec. IV (SplitCK); the contraction-as-small-GEMM view is the
// paper's loop-over-GEMM (Sec. III), here with the whole element's lines in
// the GEMM's M dimension.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ck_fp64.cuh"
#include "stp_internal.h"

namespace stp {
namespace mixed {

constexpr int ceil_div_c(int a, int b) { return (a + b - 1) / b; }

// ---- tcgen05 / mbarrier helpers (inline PTX) --------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes stored contiguously; lbo = byte distance between the two
// core matrices along K, sbo = byte distance between 8-row groups.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for sm_100-class tensor cores
  // base offset 0, absolute LBO mode, layout type 0 = no swizzle
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A/B = F16 (fmt 0) or BF16 (fmt 1),
// both K-major, M = 128, N = 16.
__host__ __device__ constexpr uint32_t umma_idesc_m128_n16(uint32_t fmt) {
  return (1u << 4)            // D format: F32
         | (fmt << 7)         // A format
         | (fmt << 10)        // B format
         | ((16u >> 3) << 17) // N >> 3
         | ((128u >> 4) << 24);  // M >> 4
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Bounded wait for the phase with the given parity (at most `limit` polls);
// returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = 1 << 22) {
  const uint32_t addr = smem_u32(bar);
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 lanes x 16 consecutive 32-bit columns; thread i of the warp gets lane
// (lane base of taddr) + i.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a 128 x 16 16-bit operand tile in the
// K-major no-swizzle layout with lbo = 128, sbo = 256.
__device__ __forceinline__ int tile_offset(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Two values rounded to nearest in one conversion instruction; each gets its
// 16-bit pattern and its value back in FP32 (same rounding as to_bits).
template <bool FP16>
__device__ __forceinline__ void to_bits2(float a, float b, uint16_t* ba, uint16_t* bb, float* fa,
                                         float* fb) {
  if (FP16) {
    const __half2 h = __floats2half2_rn(a, b);
    *ba = __half_as_ushort(__low2half(h));
    *bb = __half_as_ushort(__high2half(h));
    const float2 f = __half22float2(h);
    *fa = f.x;
    *fb = f.y;
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    *ba = __bfloat16_as_ushort(__low2bfloat16(h));
    *bb = __bfloat16_as_ushort(__high2bfloat16(h));
    const float2 f = __bfloat1622float2(h);
    *fa = f.x;
    *fb = f.y;
  }
}

template <bool FP16>
__device__ __forceinline__ uint16_t to_bits(float v, float* back) {
  if (FP16) {
    const __half h = __float2half_rn(v);
    *back = __half2float(h);
    return __half_as_ushort(h);
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    *back = __bfloat162float(h);
    return __bfloat16_as_ushort(h);
  }
}

// Quantities each pass differentiates and the accumulator each result feeds:
// accumulators 0..2 velocities, 3 s12, 4 s13, 5 s23, 6 dv1/dx, 7 dv2/dy, 8 dv3/dz.
// (functions, so that unrolled loops fold them to constants)
__host__ __device__ constexpr int pass_qty(int pass, int q6) {
  // q6 0..2: the stress components sigma_{d,j} (j = x, y, z); 3..5: v1, v2, v3
  return q6 >= 3 ? (q6 - 3)
       : pass == 0 ? (q6 == 0 ? kS11 : q6 == 1 ? kS12 : kS13)
       : pass == 1 ? (q6 == 0 ? kS12 : q6 == 1 ? kS22 : kS23)
                   : (q6 == 0 ? kS13 : q6 == 1 ? kS23 : kS33);
}
// value of quantity pass_qty(pass, q6) from a 9-vector, by selects only
__device__ __forceinline__ float pick_pass(const float* v, int pass, int q6) {
  if (q6 >= 3) return v[q6 - 3];
  const float x = v[q6 == 0 ? kS11 : q6 == 1 ? kS12 : kS13];
  const float y = v[q6 == 0 ? kS12 : q6 == 1 ? kS22 : kS23];
  const float z = v[q6 == 0 ? kS13 : q6 == 1 ? kS23 : kS33];
  return pass == 0 ? x : (pass == 1 ? y : z);
}

__host__ __device__ constexpr int pass_acc(int pass, int q6) {
  // stresses feed the velocity accumulators 0..2; d v_i / d x_pass feeds
  // dv1/dx (6), dv2/dy (7), dv3/dz (8) or the shear sums s12 (3), s13 (4), s23 (5)
  return q6 < 3 ? q6
       : pass == 0 ? (q6 == 3 ? 6 : q6 == 4 ? 3 : 4)
       : pass == 1 ? (q6 == 3 ? 3 : q6 == 4 ? 7 : 5)
                   : (q6 == 3 ? 4 : q6 == 4 ? 5 : 8);
}

constexpr int kScaleExp = 14;  // largest scaled magnitude just below 2^14

template <int N, int T, bool FP16>
struct MixedShape {
  static constexpr int N3 = N * N * N;
  static constexpr int THREADS = N <= 10 ? 256 : 512;
  static constexpr int NPT = ceil_div_c(N3, THREADS);
  static constexpr int S = N3 | 1;
  static constexpr int LDD = N | 1;
  static constexpr int ROWS = 6 * N * N;           // lines per pass
  static constexpr int TILES = ceil_div_c(ROWS, 128);
  static constexpr int TMEM_COLS = TILES * 16 <= 32 ? 32 : (TILES * 16 <= 64 ? 64 : 128);
  // phase 1 (FP64 step): p64[9][S] + coef64[4][S]
  static constexpr size_t PH1 = sizeof(double) * (size_t)(13 * S);
  // phase 2 (mixed steps): A tiles [T][TILES][4096 B] + gacc[9][S] float
  static constexpr size_t A_BYTES = (size_t)T * TILES * 4096;
  static constexpr size_t PH2 = A_BYTES + sizeof(float) * (size_t)(9 * S);
  static constexpr size_t REGION = PH1 > PH2 ? PH1 : PH2;
  // fixed part: B tiles [T][512 B], D0 [N][LDD] double, phi [2N] double,
  // scale maxima [2][9] uint, mbarrier, TMEM address
  static constexpr size_t B_OFF = (REGION + 1023) & ~(size_t)1023;
  static constexpr size_t D0_OFF = B_OFF + (size_t)T * 512;
  static constexpr size_t PHI_OFF = D0_OFF + sizeof(double) * N * LDD;
  static constexpr size_t MAX_OFF = PHI_OFF + sizeof(double) * 2 * N;
  static constexpr size_t FAC_OFF = MAX_OFF + 2 * 9 * 4;  // float [3][6]
  static constexpr size_t BAR_OFF = (FAC_OFF + 18 * 4 + 15) & ~(size_t)15;
  static constexpr size_t TADDR_OFF = BAR_OFF + 8;
  static constexpr size_t SMEM = TADDR_OFF + 16 + 1024;  // + slack to align the base to 1 KB
  static constexpr int MINB = (2 * (SMEM + 1024) <= 233472 && THREADS <= 512) ? 2 : 1;
};

template <int N, int T, bool FP16>
__global__ void __launch_bounds__(MixedShape<N, T, FP16>::THREADS, MixedShape<N, T, FP16>::MINB)
mixed_stp_kernel(const double* __restrict__ q, const double* __restrict__ params,
                 double* __restrict__ out_avg, double* __restrict__ out_faces,
                 const double* __restrict__ tables, const double* __restrict__ Dref,
                 float dt_over_dx, int eD, int64_t E, unsigned int* __restrict__ status) {
  using Sh = MixedShape<N, T, FP16>;
  constexpr int N3 = Sh::N3, S = Sh::S, LDD = Sh::LDD, NPT = Sh::NPT, THREADS = Sh::THREADS;
  constexpr int TILES = Sh::TILES, ROWS = Sh::ROWS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  double* p64 = reinterpret_cast<double*>(smem);     // phase 1
  double* coef = p64 + 9 * S;                          // phase 1
  unsigned char* A = smem;                             // phase 2
  float* gacc = reinterpret_cast<float*>(smem + Sh::A_BYTES);  // phase 2
  unsigned char* Bt = smem + Sh::B_OFF;
  double* D0 = reinterpret_cast<double*>(smem + Sh::D0_OFF);
  double* phi = reinterpret_cast<double*>(smem + Sh::PHI_OFF);
  unsigned int* smax = reinterpret_cast<unsigned int*>(smem + Sh::MAX_OFF);
  float* sfac = reinterpret_cast<float*>(smem + Sh::FAC_OFF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Sh::BAR_OFF);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(smem + Sh::TADDR_OFF);

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int64_t e = blockIdx.x;
  if (e >= E) return;  // grid is exactly E blocks; kept as a guard

  if (warp == 0) {
    tmem_alloc(taddr_s, Sh::TMEM_COLS);
    tc_fence_before();
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // tables: first step matrix (k = 0) and face vectors; scale maxima cleared
  for (int i = tid; i < N * N; i += THREADS) D0[(i / N) * LDD + (i % N)] = tables[i];
  for (int i = tid; i < 2 * N; i += THREADS) phi[i] = tables[N3 + i];
  if (tid < 18) smax[tid] = 0u;
  // split derivative matrix: B_t[n=i][k=l] = slice t of D[i][l] * 2^sD (zero padded)
  const double sD = ldexp(1.0, kScaleExp - eD);  // eD: exponent of max |D| (host)
  for (int i = tid; i < 16 * 16; i += THREADS) {
    const int n = i >> 4, k = i & 15;
    double rem = (n < N && k < N) ? Dref[n * N + k] * sD : 0.0;
#pragma unroll
    for (int t = 0; t < T; ++t) {
      float back;
      const uint16_t bits = to_bits<FP16>((float)rem, &back);
      *reinterpret_cast<uint16_t*>(Bt + t * 512 + tile_offset(n, k)) = bits;
      rem -= (double)back;
    }
  }

  // ---- load q, params (phase 1) ----
  const double* qe = q + e * (int64_t)(9 * N3);
  double* ae = out_avg + e * (int64_t)(9 * N3);
  for (int f = tid; f < 9 * N3; f += THREADS) {
    const int n = f / 9, s = f - n * 9;
    p64[s * S + n] = __ldg(qe + f);
  }
  const double* pe = params + e * (int64_t)(3 * N3);
  for (int n = tid; n < N3; n += THREADS)
    elastic_coefficients(__ldg(pe + 3 * n), __ldg(pe + 3 * n + 1), __ldg(pe + 3 * n + 2), &coef[n],
                         &coef[S + n], &coef[2 * S + n], &coef[3 * S + n]);
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *taddr_s;

  // ---- FP64 first term r_1 (the correction pass) ----
  float r[NPT][9];   // current term r_k of the owned nodes (0 for slots without a node)
  float cf[NPT][4];
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
#pragma unroll
    for (int s = 0; s < 9; ++s) r[j][s] = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) cf[j][c] = 0.f;
    const int n = tid + j * THREADS;
    if (n >= N3) continue;
    const int x = n % N, y = (n / N) % N, z = n / (N * N);
    double r1[9];
    ck_node_fp64<N, S, LDD>(p64, D0, x, y, z, coef[n], coef[S + n], coef[2 * S + n],
                            coef[3 * S + n], r1);
#pragma unroll
    for (int s = 0; s < 9; ++s) {
      ae[n * 9 + s] = p64[s * S + n] + r1[s];
      r[j][s] = (float)r1[s];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) cf[j][c] = (float)coef[c * S + n];
  }
  __syncthreads();  // phase 1 buffers are dead from here on

  // zero the operand tiles (K and row padding must read as 0) and gacc
  for (int i = tid; i < (int)((Sh::PH2 + 15) / 16); i += THREADS)  // <= B_OFF / 16
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  float tail[NPT][9];
#pragma unroll
  for (int j = 0; j < NPT; ++j)
#pragma unroll
    for (int s = 0; s < 9; ++s) tail[j][s] = 0.f;

  constexpr uint32_t idesc = umma_idesc_m128_n16(FP16 ? 0u : 1u);
  uint32_t phase = 0;
  bool ok = true;

  for (int k = 1; k < N; ++k) {
    // per-quantity maxima of r_k (power-of-two scaling of the slices)
    unsigned int* mx = smax + 9 * (k & 1);
    {
      float m[9];
#pragma unroll
      for (int s = 0; s < 9; ++s) m[s] = 0.f;
#pragma unroll
      for (int j = 0; j < NPT; ++j)
#pragma unroll
        for (int s = 0; s < 9; ++s) m[s] = fmaxf(m[s], fabsf(r[j][s]));
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        float v = m[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) atomicMax(mx + s, __float_as_uint(v));
      }
    }
    __syncthreads();
    if (tid < 9) smax[9 * ((k + 1) & 1) + tid] = 0u;  // buffer of step k+1 (last read in step k-1)
    float sc[9];  // 2^(14 - e_s): scale of quantity s
    const float step = dt_over_dx / (float)(k + 2);  // dt / ((k+2) dx)
#pragma unroll
    for (int s = 0; s < 9; ++s) {
      int es;
      frexpf(__uint_as_float(mx[s]), &es);
      es = es < -100 ? -100 : es;  // keeps 2^(14 - e_s) finite in FP32
      sc[s] = ldexpf(1.f, kScaleExp - es);
      // factor turning a tensor-core result of quantity s back into the step's
      // scaled derivative (read by the TMEM readers after the pass barrier)
      if (tid == 0) {
#pragma unroll
        for (int ps = 0; ps < 3; ++ps)
#pragma unroll
          for (int q6 = 0; q6 < 6; ++q6)
            if (pass_qty(ps, q6) == s) sfac[ps * 6 + q6] = ldexpf(step, es + eD - 2 * kScaleExp);
      }
    }

#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
      float scp[6];  // scales of the pass's six quantities (selects, no indexed arrays)
#pragma unroll
      for (int q6 = 0; q6 < 6; ++q6) scp[q6] = pick_pass(sc, pass, q6);
      // 1. slices of this pass's six quantities into the operand tiles
#pragma unroll
      for (int j = 0; j < NPT; ++j) {
        const int n = tid + j * THREADS;
        if (n >= N3) continue;
        const int x = n % N, y = (n / N) % N, z = n / (N * N);
        int a, b, kk;
        if (pass == 0) { a = z; b = y; kk = x; }
        else if (pass == 1) { a = z; b = x; kk = y; }
        else { a = y; b = x; kk = z; }
#pragma unroll
        for (int q6 = 0; q6 < 6; q6 += 2) {  // two quantities per conversion instruction
          const int row0 = (q6 * N + a) * N + b, row1 = row0 + N * N;
          const int off0 = (row0 >> 7) * 4096 + tile_offset(row0 & 127, kk);
          const int off1 = (row1 >> 7) * 4096 + tile_offset(row1 & 127, kk);
          float rem0 = pick_pass(r[j], pass, q6) * scp[q6];
          float rem1 = pick_pass(r[j], pass, q6 + 1) * scp[q6 + 1];
#pragma unroll
          for (int t = 0; t < T; ++t) {
            uint16_t b0, b1;
            float f0, f1;
            to_bits2<FP16>(rem0, rem1, &b0, &b1, &f0, &f1);
            *reinterpret_cast<uint16_t*>(A + t * TILES * 4096 + off0) = b0;
            *reinterpret_cast<uint16_t*>(A + t * TILES * 4096 + off1) = b1;
            rem0 -= f0;
            rem1 -= f1;
          }
        }
      }
      fence_async_smem();
      __syncthreads();
      // 2. one thread issues the GEMMs: per tile, slice pairs smallest first
      if (tid == 0) {
        tc_fence_after();
#pragma unroll
        for (int m = 0; m < TILES; ++m) {
          int issued = 0;
#pragma unroll
          for (int lvl = T - 1; lvl >= 0; --lvl)
#pragma unroll
            for (int sa = 0; sa <= lvl; ++sa) {
              const int sb = lvl - sa;
              const uint64_t ad = umma_desc(smem_u32(A + (sa * TILES + m) * 4096), 128, 256);
              const uint64_t bd = umma_desc(smem_u32(Bt + sb * 512), 128, 256);
              umma_f16(tmem + m * 16, ad, bd, idesc, issued > 0 ? 1u : 0u);
              ++issued;
            }
        }
        umma_commit(bar);
      }
      // 3. results: warp w reads TMEM lanes 32*(w%4).. of tiles w/4, w/4 + W/4, ...
      const bool arrived = mbar_wait(bar, phase);
      phase ^= 1u;
      if (!__syncthreads_and(arrived ? 1 : 0)) { ok = false; break; }  // uniform decision
      tc_fence_after();
      {
        const int quarter = warp & 3;
        for (int m = warp >> 2; m < TILES; m += THREADS / 128) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(m * 16), v);
          const int row = m * 128 + quarter * 32 + lane;
          if (row < ROWS) {
            const int q6 = row / (N * N);
            const int a = (row / N) % N, b = row % N;
            const int acc = pass_acc(pass, q6);
            const float f = sfac[pass * 6 + q6];
#pragma unroll
            for (int c = 0; c < N; ++c) {
              int node;
              if (pass == 0) node = (a * N + b) * N + c;
              else if (pass == 1) node = (a * N + c) * N + b;
              else node = (c * N + a) * N + b;
              gacc[acc * S + node] = fmaf(f, v[c], gacc[acc * S + node]);
            }
          }
        }
      }
      tc_fence_before();
      __syncthreads();
    }
    if (!ok) break;
    // 4. pointwise elastic update in FP32 for the owned nodes
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
      const int n = tid + j * THREADS;
      if (n >= N3) continue;
      float g[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        g[c] = gacc[c * S + n];
        gacc[c * S + n] = 0.f;
      }
      const float invrho = cf[j][0], lam = cf[j][1], mu = cf[j][2], mu2 = cf[j][3];
      const float ltr = lam * ((g[6] + g[7]) + g[8]);
      float nr[9];
      nr[kV1] = invrho * g[0];
      nr[kV2] = invrho * g[1];
      nr[kV3] = invrho * g[2];
      nr[kS11] = fmaf(mu2, g[6], ltr);
      nr[kS22] = fmaf(mu2, g[7], ltr);
      nr[kS33] = fmaf(mu2, g[8], ltr);
      nr[kS12] = mu * g[3];
      nr[kS13] = mu * g[4];
      nr[kS23] = mu * g[5];
#pragma unroll
      for (int s = 0; s < 9; ++s) {
        r[j][s] = nr[s];
        tail[j][s] += nr[s];
      }
    }
  }

  // ---- FP64 average and faces ----
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int n = tid + j * THREADS;
    if (n >= N3) continue;
#pragma unroll
    for (int s = 0; s < 9; ++s) ae[n * 9 + s] += (double)tail[j][s];
  }
  if (!ok && tid == 0) {
    // the tensor-core work of the last pass did not signal completion in time:
    // report it, give it one more bounded wait, flag the context (bit 2) if
    // the tensor cores are still not drained, then release TMEM and finish
    const bool drained = mbar_wait(bar, phase ^ 1u);
    atomicOr(status, drained ? 1u : 5u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, Sh::TMEM_COLS);

  double* fe = out_faces + e * (int64_t)(6 * N * N * 9);
  for (int o = tid; o < 6 * N * N * 9; o += THREADS) {
    const int s = o % 9;
    int rest = o / 9;
    const int bb = rest % N;
    rest /= N;
    const int aa = rest % N;
    const int f = rest / N;
    const int d = f >> 1;
    const double* ph = phi + (f & 1) * N;
    int base, stride;
    if (d == 0) { base = (aa * N + bb) * N; stride = 1; }
    else if (d == 1) { base = aa * N * N + bb; stride = N; }
    else { base = aa * N + bb; stride = N * N; }
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) acc = fma(ph[i], ae[(base + i * stride) * 9 + s], acc);
    fe[o] = acc;
  }
}

template <int N, int T, bool FP16>
cudaError_t launch_mixed_shape(int64_t E, const double* q, const double* params, double* out_avg,
                               double* out_faces, const double* tables, const double* Dref,
                               double dt_over_dx, int eD, unsigned int* status, cudaStream_t stream) {
  using Sh = MixedShape<N, T, FP16>;
  static_assert(Sh::SMEM <= 232448, "shared memory budget of one CTA exceeded");
  auto kern = mixed_stp_kernel<N, T, FP16>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
  if (err != cudaSuccess) return err;
  if (E > 0x7fffffffLL) return cudaErrorInvalidValue;
  kern<<<(unsigned)E, Sh::THREADS, Sh::SMEM, stream>>>(q, params, out_avg, out_faces, tables, Dref,
                                                       (float)dt_over_dx, eD, E, status);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_mixed_n(int variant, int64_t E, const double* q, const double* params,
                           double* out_avg, double* out_faces, const double* tables,
                           const double* Dref, double dt_over_dx, int eD, unsigned int* status,
                           cudaStream_t stream) {
  switch (variant) {
    case 1: return launch_mixed_shape<N, 2, false>(E, q, params, out_avg, out_faces, tables, Dref, dt_over_dx, eD, status, stream);
    case 2: return launch_mixed_shape<N, 3, false>(E, q, params, out_avg, out_faces, tables, Dref, dt_over_dx, eD, status, stream);
    case 3: return launch_mixed_shape<N, 2, true>(E, q, params, out_avg, out_faces, tables, Dref, dt_over_dx, eD, status, stream);
    case 4: return launch_mixed_shape<N, 3, true>(E, q, params, out_avg, out_faces, tables, Dref, dt_over_dx, eD, status, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mixed

}  // namespace stp
