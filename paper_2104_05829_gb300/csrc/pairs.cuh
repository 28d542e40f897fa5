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

// double -> pair: hi = fl32(x), lo = fl32(x - hi). The conversions run on the
// FP64 pipe, which is otherwise idle in this kernel, so they overlap with the
// FP32 work (an integer-only split was measured slower: it adds instructions
// to the FP32/ALU issue path, which is the kernel's limit).
__device__ __forceinline__ ff ff_split(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return {h, l};
}

__device__ __forceinline__ double ff_join(ff a) { return (double)a.h + (double)a.l; }

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

// a + b without the final renormalisation: hi is fl(a.h + b.h) and lo gathers its exact
// rounding error and a.l + b.l. The pair's value is the same to the same order (about
// 2^-48 of |a| + |b|); lo may exceed ulp(hi)/2 after cancellation, which the error-free
// transforms of ff_add and ff_mac accept as inputs (TwoSum and the TwoProduct of the
// high parts stay exact; the low cross terms are rounded relative to |lo|).
__device__ __forceinline__ ff ff_add_u(const ff a, const ff b) {
  const float s = __fadd_rn(a.h, b.h);
  const float t = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, t)), __fsub_rn(b.h, t));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return {s, e};
}
__device__ __forceinline__ ff ff_sub_u(const ff a, const ff b) { return ff_add_u(a, ff{-b.h, -b.l}); }

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
