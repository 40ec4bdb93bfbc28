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

// a += (nh + nl) * (x.hi + x.lo): the product's high part with its exact FMA
// error and the cross terms, TwoSum of the high words, the low word kept
// unnormalised (ff_norm renormalises once at the end of a sum)
__device__ __forceinline__ void ff_acc_prod(ff& a, float nh, float nl, ff x) {
  const float p = __fmul_rn(nh, x.hi);
  float e = __fmaf_rn(nh, x.hi, -p);
  e = __fmaf_rn(nh, x.lo, e);
  e = __fmaf_rn(nl, x.hi, e);
  const float s = __fadd_rn(a.hi, p);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, __fadd_rn(e, err));
}

__device__ __forceinline__ ff ff_norm(ff a) { return fast_two_sum(a.hi, a.lo); }


// ---------------------------------------------------------------------------
// Paired accumulation on the packed FP32 instructions of sm_100 and later
// (one instruction issues the same operation on two lanes).  An ff2 holds two
// independent float-float values, lane x and lane y.  Each lane runs the
// operation sequence of the scalar compensated accumulation (product with its
// FMA error, TwoSum of the high words, unnormalised low word) step for step,
// so the paired sums equal the scalar ones bit for bit.  Subtractions are
// written as fma(a, -1, b), which rounds exactly like b - a, and the product
// enters negated (nn = -nh, a table value), so no negation is issued.
// ---------------------------------------------------------------------------
struct ff2 {
  float2 hi, lo;
};

__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }
__device__ __forceinline__ ff2 ff2_zero() { return ff2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

// a += p lane-wise, given pn = -p and e = the product's exact error terms
__device__ __forceinline__ void ff2_acc(ff2& a, float2 pn, float2 e) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 s = __ffma2_rn(pn, m1, a.hi);   // hi + p
  const float2 bb = __ffma2_rn(a.hi, m1, s);   // s - hi
  const float2 t = __ffma2_rn(bb, m1, s);      // s - bb
  const float2 u = __ffma2_rn(t, m1, a.hi);    // hi - (s - bb)
  const float2 vn = __fadd2_rn(pn, bb);        // -(p - bb)
  const float2 err = __ffma2_rn(vn, m1, u);    // (hi - (s - bb)) + (p - bb)
  a.hi = s;
  a.lo = __fadd2_rn(a.lo, __fadd2_rn(e, err));
}

// a += (nh + nl) * x lane-wise (x a float per lane), nn = -nh
__device__ __forceinline__ void ff2_add_f(ff2& a, float2 nh, float2 nn, float2 nl, float2 x) {
  const float2 pn = __fmul2_rn(nn, x);
  float2 e = __ffma2_rn(nh, x, pn);
  e = __ffma2_rn(nl, x, e);
  ff2_acc(a, pn, e);
}

// a += (nh + nl) * (xh + xl) lane-wise, nn = -nh
__device__ __forceinline__ void ff2_add_v(ff2& a, float2 nh, float2 nn, float2 nl, float2 xh, float2 xl) {
  const float2 pn = __fmul2_rn(nn, xh);
  float2 e = __ffma2_rn(nh, xh, pn);
  e = __ffma2_rn(nh, xl, e);
  e = __ffma2_rn(nl, xh, e);
  ff2_acc(a, pn, e);
}

#endif

}  // namespace mfa
