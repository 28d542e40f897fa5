// FP32-pair arithmetic: a value is the unevaluated sum hi + lo of two floats
// (about 48 significant bits, FP32 exponent range). Error-free transforms:
//   TwoProduct (FMA form):  p = a*b, e = fma(a, b, -p)            a*b = p + e exactly
//   TwoSum (Knuth):         s = a+b, t = s-a, e = (a-(s-t)) + (b-t)   a+b = s + e exactly
// Intrinsics with explicit rounding (__fadd_rn, __fmul_rn, __fmaf_rn) keep the
// compiler from contracting or reassociating the transforms.
#pragma once

#include <cuda_runtime.h>

namespace sem {

struct ff {
  float h, l;
};

// double -> pair with integer operations only (GB300's FP64 pipe is slow, and
// conversions run on it): hi keeps the top 24 significand bits of x
// (truncation), lo = x - hi is the remaining 29-bit integer times 2^(e-1075),
// rounded once to float. |x - hi - lo| <= 2^-48 |x|. Values below 2^-74 in
// magnitude lose their lo part; |x| must stay below the FP32 range (~3e38).
__device__ __forceinline__ ff ff_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 897) return {__int_as_float((int)sign), 0.f};          // |x| < 2^-126: flush
  const unsigned hb = sign | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7FFFFF);
  const unsigned mlo = (unsigned)(b & 0x1FFFFFFFu);
  float lo = 0.f;
  if (mlo != 0u && e >= 949) {
    const float scale = __int_as_float((e - 1075 + 127) << 23);  // 2^(e - 1075)
    lo = __fmul_rn(__uint2float_rn(mlo), scale);
    if (sign) lo = -lo;
  }
  return {__int_as_float((int)hb), lo};
}

// float -> double by bit manipulation (exact for normal floats and zero)
__device__ __forceinline__ double ff_f2d(float f) {
  const unsigned fb = (unsigned)__float_as_int(f);
  const unsigned e = (fb >> 23) & 0xFF;
  if (e == 0) return __longlong_as_double((long long)((unsigned long long)(fb >> 31) << 63));  // +-0 (denormals flushed)
  const unsigned long long db = ((unsigned long long)(fb >> 31) << 63) |
                                ((unsigned long long)(e + 896) << 52) |
                                ((unsigned long long)(fb & 0x7FFFFF) << 29);
  return __longlong_as_double((long long)db);
}

// pair -> double: one FP64 addition of the exactly converted parts
__device__ __forceinline__ double ff_join(ff a) { return __dadd_rn(ff_f2d(a.h), ff_f2d(a.l)); }

// renormalise so that |l| <= ulp(h)/2 (TwoSum, valid for any magnitudes)
__device__ __forceinline__ ff ff_norm(const ff a) {
  const float s = __fadd_rn(a.h, a.l);
  const float t = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, t)), __fsub_rn(a.l, t));
  return {s, e};
}

// a + b and a - b, renormalised
__device__ __forceinline__ ff ff_add(const ff a, const ff b) {
  const float s = __fadd_rn(a.h, b.h);
  const float t = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, t)), __fsub_rn(b.h, t));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ ff ff_sub(const ff a, const ff b) { return ff_add(a, ff{-b.h, -b.l}); }

// x * y, unnormalised
__device__ __forceinline__ ff ff_mul(const ff x, const ff y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return {p, e};
}

// acc + x * y, unnormalised (TwoProduct on the high parts, TwoSum into acc.h,
// every lower-order term gathered in acc.l)
__device__ __forceinline__ ff ff_mac(const ff acc, const ff x, const ff y) {
  const float p = __fmul_rn(x.h, y.h);
  const float e = __fmaf_rn(x.h, y.h, -p);
  const float s = __fadd_rn(acc.h, p);
  const float t = __fsub_rn(s, acc.h);
  const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, t)), __fsub_rn(p, t));
  float l = __fadd_rn(acc.l, err);
  l = __fadd_rn(l, e);
  l = __fmaf_rn(x.h, y.l, l);
  l = __fmaf_rn(x.l, y.h, l);
  return {s, l};
}

inline ff ff_host_split(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

}  // namespace sem
