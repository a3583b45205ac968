// Double-word ("double-float") arithmetic on the FP32 pipe for FP64-class
// reductions and products on GB300, whose FP64 rate is a small fraction of
// its FP32 rate.  A value is represented by an unevaluated sum hi + lo of two
// floats.  Building blocks (published error-free transformations):
//   TwoSum      Knuth, The Art of Computer Programming vol. 2 (1969)
//   FastTwoSum  Dekker, "A floating-point technique for extending the
//               available precision", Numer. Math. 18 (1971)
//   TwoProd     the exact product error via one fused multiply-add
//   Dot2        Ogita, Rump, Oishi, "Accurate sum and dot product",
//               SIAM J. Sci. Comput. 26 (2005): products summed with TwoSum,
//               all error terms gathered in a compensation accumulator.
// With float working precision u = 2^-24 the dot-product result has error
// about u^2 * sum |a_i b_i| (plus the conditioning term of Dot2), i.e. the
// accuracy of an FP64 evaluation.
//
// FP64 <-> double-word conversions use integer operations only (no FP64 or
// conversion pipe): split_f64 truncates the significand to 24 bits for hi and
// builds lo from the remaining 29 bits; dw_to_f64 rebuilds both floats as
// doubles from their bit fields and adds them with one FP64 addition.  (Native
// float<->double conversions execute on the FP64 pipe of this GPU, which is
// why none is used.)  Inputs with |x| < 2^-74 lose their lo part (relative
// error then 2^-23); |x| < 2^-126 becomes a signed zero and |x| >= 2^128 a
// signed infinity.
#ifndef BPJD_DWORD_CUH_
#define BPJD_DWORD_CUH_

#include <cstdint>

namespace bpjd {

struct dw {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ dw split_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);
  dw r;
  if (e < 897) {  // |x| < 2^-126 (including zero): flushed to a signed zero
    r.hi = __uint_as_float(sign);
    r.lo = 0.f;
    return r;
  }
  if (e > 1150) {  // beyond the float range: signed infinity
    r.hi = __uint_as_float(sign | 0x7f800000u);
    r.lo = 0.f;
    return r;
  }
  const unsigned long long mant = b & 0xfffffffffffffULL;
  r.hi = __uint_as_float(sign | ((unsigned int)(e - 896) << 23) | (unsigned int)(mant >> 29));
  // lo = rem * 2^(e - 1075), rem < 2^29, built from its bit pattern (normalised
  // by a leading-zero count, significand truncated to 24 bits): no conversion
  // instruction, which would run on the FP64 pipe
  const unsigned int rem = (unsigned int)(mant & 0x1fffffffULL);
  float lo = 0.f;
  if (rem) {
    const int lz = __clz(rem);
    const int fe = (31 - lz) + e - 948;  // biased float exponent of lo
    if (fe >= 1) {
      const unsigned int m23 = (unsigned int)((((unsigned long long)rem) << (lz + 1)) >> 9) & 0x7fffffu;
      lo = __uint_as_float(((unsigned int)fe << 23) | m23);
    }
  }
  r.lo = sign ? -lo : lo;
  return r;
}

// The float nearest below |x| in magnitude (significand truncated to 24 bits):
// the hi part of split_f64, integer operations only.
__device__ __forceinline__ float f64_hi(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);
  if (e < 897) return __uint_as_float(sign);
  if (e > 1150) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned int)(e - 896) << 23) | (unsigned int)((b & 0xfffffffffffffULL) >> 29));
}

__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xff;
  const unsigned long long s = (unsigned long long)(u >> 31) << 63;
  const unsigned long long m = (unsigned long long)(u & 0x7fffff) << 29;
  unsigned long long ex = (unsigned long long)(e + 896) << 52;
  if (e == 0) return __longlong_as_double((long long)s);  // zero and subnormals: signed zero
  if (e == 0xff) ex = 0x7ffULL << 52;                       // inf / nan
  return __longlong_as_double((long long)(s | ex | m));
}

__device__ __forceinline__ double dw_to_f64(float hi, float lo) {
  return f32_to_f64_bits(hi) + f32_to_f64_bits(lo);
}

// Dot2 accumulator: running sum s and compensation c.
struct dot2 {
  float s, c;
  __device__ __forceinline__ void zero() {
    s = 0.f;
    c = 0.f;
  }
  // += (ah + al) * (bh + bl)
  __device__ __forceinline__ void mac(float ah, float al, float bh, float bl) {
    float p, e;
    two_prod(ah, bh, p, e);
    e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
    float t, u;
    two_sum(s, p, t, u);
    s = t;
    c = __fadd_rn(c, __fadd_rn(u, e));
  }
  // += (ah + al)
  __device__ __forceinline__ void add(float ah, float al) {
    float t, u;
    two_sum(s, ah, t, u);
    s = t;
    c = __fadd_rn(c, __fadd_rn(u, al));
  }
  __device__ __forceinline__ double value() const { return dw_to_f64(s, c); }
};

}  // namespace bpjd

#endif  // BPJD_DWORD_CUH_
