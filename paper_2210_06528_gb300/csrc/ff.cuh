// Float-float ("double-single") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// giving about 48 significant bits at FP32 throughput.  The building blocks
// are the error-free transformations of Knuth (TwoSum: a + b = s + e exactly)
// and of the fused multiply-add product (TwoProd: a * b = p + e exactly, with
// e = fma(a, b, -p)), combined as in Dekker's 1971 double-length arithmetic.
// Every operation uses the explicitly rounded intrinsics (__fadd_rn,
// __fmul_rn, __fmaf_rn) so that the compiler never contracts or reorders the
// error terms.
#pragma once

#include <cuda_runtime.h>

namespace mfa {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ ff(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ ff(float v) : hi(v), lo(0.f) {}
  __host__ __device__ ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

#ifdef __CUDACC__

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff(s, e);
}

// |a| >= |b| (or a == 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return ff(s, e);
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }

// acc += a * b with one rounding of the error terms (product accumulate)
__device__ __forceinline__ void ff_fma_acc(ff& acc, ff a, ff b) { acc = acc + a * b; }

#endif

}  // namespace mfa
