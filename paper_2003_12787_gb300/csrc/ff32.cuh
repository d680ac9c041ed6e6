// Float-float ("double-float") arithmetic on the FP32 pipes.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)
// (about 48 significant bits). The building blocks are the error-free
// transformations:
//   TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2): s = fl(a + b) and the exact
//     rounding error of that sum, for any a, b;
//   FastTwoSum (Dekker 1971): the same for |a| >= |b|, in three operations;
//   TwoProduct with FMA: p = fl(a b) and the exact error fma(a, b, -p);
// and the compensated dot product Dot2 of Ogita, Rump and Oishi ("Accurate
// sum and dot product", SIAM J. Sci. Comput. 26, 2005), which accumulates the
// high-part products with TwoSum and every error term in a plain FP32 sum.
// The *_rn intrinsics keep the compiler from fusing a product into a later
// addition, which would break the error-free transformations.
//
// Conversions between double and float-float use integer operations on the
// IEEE-754 encodings, not the FP64 pipe: on this GPU a float<->double
// conversion costs as much as a DFMA. They take a power-of-two scale 2^sc
// (exact): split(x, sc) represents x * 2^-sc, widen(f, sc) returns f * 2^sc.
// Scaled values below the FP32 normal range (2^-126) are treated as zero;
// values above it become infinite.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace stp {
namespace ff {

__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}

__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ float2 add(float2 x, float2 y) {
  const float2 s = two_sum(x.x, y.x);
  return fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(x.y, y.y)));
}

__device__ __forceinline__ float2 neg(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 sub(float2 x, float2 y) { return add(x, neg(y)); }

// The same sum without the closing renormalisation: (fl(x.hi + y.hi), rest).
// Such pairs are exact-valued inputs to every operation here (TwoSum and
// TwoProduct take any operands), but after a cancellation the rest can exceed
// ulp(first part), and a Dot2 cross term made from it is then rounded at a
// larger scale: use it for sums that do not feed a product (the lines' mirrored
// sums and differences stay renormalised).
__device__ __forceinline__ float2 add_lazy(float2 x, float2 y) {
  const float2 s = two_sum(x.x, y.x);
  return make_float2(s.x, __fadd_rn(s.y, __fadd_rn(x.y, y.y)));
}
__device__ __forceinline__ float2 sub_lazy(float2 x, float2 y) { return add_lazy(x, neg(y)); }

__device__ __forceinline__ float2 mul(float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  return fast_two_sum(p, e);
}

// Dot2 accumulator: running FP32 sum s of the high products and c of all
// error terms; value() renormalises.
struct Dot {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void fma(float2 x, float2 y) {
    const float p = __fmul_rn(x.x, y.x);
    const float pe = __fmaf_rn(x.x, y.x, -p);
    const float2 t = two_sum(s, p);
    s = t.x;
    float cc = __fmaf_rn(x.x, y.y, c);
    cc = __fmaf_rn(x.y, y.x, cc);
    c = __fadd_rn(cc, __fadd_rn(t.y, pe));
  }
  __device__ __forceinline__ float2 value() const { return fast_two_sum(s, c); }
  __device__ __forceinline__ float2 value_lazy() const { return make_float2(s, c); }
};

// Float whose bits are sign | exponent | mantissa (no checks).
__device__ __forceinline__ float make_f(uint32_t sign, int bexp, uint32_t mant) {
  return __uint_as_float(sign | ((uint32_t)bexp << 23) | (mant & 0x7fffffu));
}

// Biased exponent field of a double (0 for zero and subnormals, 2047 for
// infinities and NaN).
__device__ __forceinline__ int exponent_field(double x) {
  return (int)(((uint64_t)__double_as_longlong(x) >> 52) & 0x7ff);
}

// double -> float-float of x * 2^-sc: hi = x * 2^-sc rounded to the nearest
// float (ties to even), lo = the rest rounded to the nearest float, so
// |hi + lo - x 2^-sc| <= 2^-49 |x 2^-sc| (normalised). Integer operations on
// the encoding only: the 53-bit significand is cut after 24 bits, the cut is
// rounded by the 29 bits below it, and those bits (or their complement when
// hi rounded up) become lo.
__device__ __forceinline__ float2 split(double x, int sc = 0) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7ff);
  const uint64_t m = b & 0xfffffffffffffull;
  if (ex == 0x7ff) {  // infinity or NaN
    return make_float2(__uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u)), 0.f);
  }
  const int fe0 = ex - 1023 - sc + 127;  // biased float exponent of hi before rounding
  if (ex == 0 || fe0 <= 0) return make_float2(__uint_as_float(sign), 0.f);
  if (fe0 >= 255) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
  const uint64_t sig = (1ull << 52) | m;        // 53-bit significand
  uint32_t hm = (uint32_t)(sig >> 29);           // its top 24 bits
  uint32_t r = (uint32_t)(sig & 0x1fffffffu);    // the 29 bits below, value r * 2^(e-52)
  uint32_t lo_sign = sign;
  int fe = fe0;
  if (r > (1u << 28) || (r == (1u << 28) && (hm & 1u))) {  // hi rounds up
    hm += 1u;
    r = (1u << 29) - r;  // lo = -r * 2^(e-52)
    lo_sign ^= 0x80000000u;
    if (hm == (1u << 24)) {
      hm = 1u << 23;
      if (++fe >= 255) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
    }
  }
  const float hi = make_f(sign, fe, hm);
  float lo = 0.f;
  if (r) {
    const int pb = 31 - __clz((int)r);  // leading bit of r (r < 2^29)
    int le = fe0 - 52 + pb;             // biased exponent of lo
    uint32_t mant;
    if (pb > 23) {                      // round r to 24 significant bits
      const int sh = pb - 23;
      mant = r >> sh;
      const uint32_t rem = r & ((1u << sh) - 1u), half = 1u << (sh - 1);
      if (rem > half || (rem == half && (mant & 1u))) ++mant;
      if (mant == (1u << 24)) {
        mant = 1u << 23;
        ++le;
      }
    } else {
      mant = r << (23 - pb);
    }
    if (le > 0) lo = make_f(lo_sign, le, mant);
  }
  return make_float2(hi, lo);
}

// float * 2^sc -> double, exact for normal floats (subnormals give zero).
__device__ __forceinline__ double widen(float f, int sc = 0) {
  const uint32_t u = __float_as_uint(f);
  const int e = (int)((u >> 23) & 0xffu);
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const uint64_t mant = (uint64_t)(u & 0x7fffffu) << 29;
  if (e == 0xff) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | mant));
  const int de = e - 127 + 1023 + sc;
  if (e == 0 || de <= 0) return __longlong_as_double((long long)sign);
  if (de >= 0x7ff) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull));
  return __longlong_as_double((long long)(sign | ((uint64_t)de << 52) | mant));
}

// float-float * 2^sc -> double: one FP64 addition of the exactly widened parts.
__device__ __forceinline__ double to_double(float2 x, int sc = 0) { return widen(x.x, sc) + widen(x.y, sc); }

// Scale exponent for a block of values: the largest finite exponent field
// (folded in by every thread, then reduced), minus the bias, so that the
// largest magnitude scales into [1, 2); 0 for an all-zero block.
__device__ __forceinline__ int scale_from_field(int max_field) {
  return max_field == 0 ? 0 : max_field - 1023;
}

}  // namespace ff
}  // namespace stp
