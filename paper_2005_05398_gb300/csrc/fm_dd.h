// Double-float ("dd") numbers: an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48
// significand bits, computed on the FP32 pipe.  On this GPU float64 runs at 1/64 of the float32 rate, so
// the inner Krylov iterations of the mixed-precision mode (FM_PREC_MIXED, mixed_scheme 2) run their
// operator and Gram-Schmidt in this arithmetic: close to float64 accuracy (relative ~1e-14 per operation),
// far from float64 cost.
//
// Arithmetic (error-free transformations, from the published definitions):
//  * TwoSum (Knuth): s = fl(a + b), e = (a - (s - v)) + (b - v) with v = s - a; then a + b = s + e exactly.
//  * TwoProd with a fused multiply-add: p = fl(a b), e = fma(a, b, -p); then a b = p + e exactly.
//  * addition, multiplication and multiply-add of dd values combine these with one renormalisation
//    (hi = fl(s + e), lo = e - (hi - s)), the "sloppy" double-double forms of Bailey's library.
// Every step uses the round-to-nearest intrinsics, which the compiler never contracts into fused
// multiply-adds (a contraction would change fl(a + b) and break the exactness the forms rely on).
#pragma once

#ifdef __CUDACC__
#define FM_HD __host__ __device__
#else
#define FM_HD
#endif

namespace fmi {

struct alignas(8) dd {
  float hi, lo;
  dd() = default;
  FM_HD constexpr dd(float h, float l) : hi(h), lo(l) {}
  FM_HD constexpr dd(int v) : hi((float)v), lo(0.f) {}  // exact for the small integers the kernels use
  FM_HD dd(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  FM_HD double to_double() const { return (double)hi + (double)lo; }
};

#ifdef __CUDACC__
__device__ __forceinline__ dd dd_renorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return dd(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ dd operator+(dd a, dd b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return dd_renorm(s, e);
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dd_renorm(p, e);
}
// a b + c
__device__ __forceinline__ dd fma(dd a, dd b, dd c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(p, c.hi);
  const float v = __fsub_rn(s, p);
  float t = __fadd_rn(__fsub_rn(p, __fsub_rn(s, v)), __fsub_rn(c.hi, v));
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  return dd_renorm(s, t);
}
__device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = a + b; }
__device__ __forceinline__ dd& operator-=(dd& a, dd b) { return a = a - b; }
#endif

}  // namespace fmi
