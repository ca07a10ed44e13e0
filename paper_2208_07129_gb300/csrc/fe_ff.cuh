// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers (|lo| <= ulp(hi) / 2), about 48 significant bits.  GB300 runs
// FP32 at 64 times its FP64 rate, so FP64-accurate contractions built from
// FP32 operations can outrun the FP64 pipe.
//
// Built from the classical error-free transformations:
//   two_sum (Knuth):   s + e = a + b exactly, s = fl(a + b);
//   two_prod (with FMA): p + e = a * b exactly, p = fl(a * b);
// and, for dot products, the compensated scheme of Ogita, Rump and Oishi
// ("Dot2", 2005): the rounded partial sums are carried in s and every
// rounding error (of the sums and of the products) is collected in c, so the
// result is as accurate as if computed in twice the working precision.
// Every operation uses the _rn intrinsics, which the compiler never merges
// into an FMA or reassociates: the transformations are exact only when each
// operation is rounded on its own.
#pragma once

#include <cuda_runtime.h>

namespace fe {

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // nearest double-float to x: hi = fl32(x), lo = fl32(x - hi)
  __host__ __device__ explicit ff(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// s + e with |e| small against s, renormalised (fast two-sum)
__device__ __forceinline__ ff renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return ff(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return renorm(s, e);
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff(-b.hi, -b.lo)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return renorm(p, e);
}

// Compensated dot-product accumulator: value s + c.
struct ffacc {
  float s, c;
};

// acc = a * b (first term)
__device__ __forceinline__ ffacc acc_first(ff a, ff b) {
  ffacc A;
  A.s = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -A.s);
  e = __fmaf_rn(a.hi, b.lo, e);
  A.c = __fmaf_rn(a.lo, b.hi, e);
  return A;
}

// acc += a * b
__device__ __forceinline__ void acc_fma(ffacc& A, ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  float t, q;
  two_sum(A.s, p, t, q);
  A.s = t;
  A.c = __fadd_rn(A.c, __fadd_rn(q, e));
  A.c = __fmaf_rn(a.hi, b.lo, A.c);
  A.c = __fmaf_rn(a.lo, b.hi, A.c);
}

__device__ __forceinline__ ff acc_value(const ffacc& A) { return renorm(A.s, A.c); }

}  // namespace fe
