// df32: a value represented as the unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2),
// about 48 significant bits, computed entirely on the FP32 pipe.
//
// Error-free transformations used (published methods):
//   two_sum      Knuth, TAOCP vol. 2, 4.2.2: s = fl(a + b) and the exact rounding error e.
//   fast_two_sum Dekker 1971 ("A floating-point technique for extending the available
//                precision"), valid for |a| >= |b|.
//   two_prod     exact product error with one fused multiply-add: e = fma(a, b, -fl(a b)).
// Double-word addition, multiplication, division and square root follow the "sloppy" variants
// of Hida, Li & Bailey (2001, "Algorithms for quad-double precision floating point
// arithmetic"): relative error of a few 2^-44 with respect to the operands' magnitudes, which is
// the scale every tolerance of this library is stated against.
// Plain products use __fmul_rn/__fadd_rn so the compiler cannot contract them into FMAs, which
// would break the error-free transformations.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace frx {

using ::sqrt;   // keep the double overload visible next to sqrt(df32)

struct df32 {
  float hi, lo;
};

__host__ __device__ __forceinline__ df32 df(float hi, float lo) {
  df32 r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// Host-side split of a double into hi + lo (for uploading operators and geometry).
inline df32 df_split_host(double d) {
  const float hi = (float)d;
  return df(hi, (float)(d - (double)hi));
}

__device__ __forceinline__ df32 df_from(double d) {
  const float hi = __double2float_rn(d);
  return df(hi, __double2float_rn(d - (double)hi));
}

__device__ __forceinline__ df32 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fadd_rn(b, __fsub_rn(a, s)));
}

__device__ __forceinline__ df32 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}

__device__ __forceinline__ double to_double(df32 x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ double to_double(double x) { return x; }

__device__ __forceinline__ df32 operator+(df32 x, df32 y) {
  df32 s = two_sum(x.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df32 operator-(df32 x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df32 operator-(df32 x, df32 y) { return x + (-y); }

__device__ __forceinline__ df32 operator*(df32 x, df32 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ df32 operator/(df32 x, df32 y) {
  const float q1 = __fdiv_rn(x.hi, y.hi);
  const df32 r = x - y * df(q1, 0.f);
  const float q2 = __fdiv_rn(r.hi, y.hi);
  return fast_two_sum(q1, q2);
}

__device__ __forceinline__ df32 &operator+=(df32 &x, df32 y) { return x = x + y; }
__device__ __forceinline__ df32 &operator-=(df32 &x, df32 y) { return x = x - y; }
__device__ __forceinline__ df32 &operator*=(df32 &x, df32 y) { return x = x * y; }

__device__ __forceinline__ df32 sqrt(df32 x) {
  if (x.hi <= 0.f) return df(0.f, 0.f);
  const float s = __fsqrt_rn(x.hi);
  const float p = __fmul_rn(s, s);
  const float e = __fmaf_rn(s, s, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), e), x.lo);
  return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}

// Sum of products sum_i c_i x_i.  For double: FMAs.  For df32: the leading parts are summed with
// two_sum and every rounding error (of the products via two_prod and the cross terms, and of the
// sums) is collected in one FP32 error term, normalised once by get() -- the usual compensated
// dot product (Ogita, Rump & Oishi 2005, "Accurate sum and dot product"), 12 FP32 instructions
// per term instead of 18 for a double-float multiply followed by an add.
template <typename T> struct Dot;

template <> struct Dot<double> {
  double s;
  __device__ __forceinline__ Dot() : s(0.0) {}
  __device__ __forceinline__ void add(double c, double x) { s = fma(c, x, s); }
  __device__ __forceinline__ double get() const { return s; }
  __device__ __forceinline__ double raw() const { return s; }
};

template <> struct Dot<float> {
  float s;
  __device__ __forceinline__ Dot() : s(0.f) {}
  __device__ __forceinline__ void add(float c, float x) { s = fmaf(c, x, s); }
  __device__ __forceinline__ float get() const { return s; }
  __device__ __forceinline__ float raw() const { return s; }
};

template <> struct Dot<df32> {
  float s, e;
  __device__ __forceinline__ Dot() : s(0.f), e(0.f) {}
  __device__ __forceinline__ void add(df32 c, df32 x) {
    const float p = __fmul_rn(c.hi, x.hi);
    float err = __fmaf_rn(c.hi, x.hi, -p);
    err = __fmaf_rn(c.hi, x.lo, err);
    err = __fmaf_rn(c.lo, x.hi, err);
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float r = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s = t;
    e = __fadd_rn(e, __fadd_rn(r, err));
  }
  __device__ __forceinline__ df32 get() const {
    const df32 r = two_sum(s, e);
    return fast_two_sum(r.hi, r.lo);
  }
  // The same value s + e with one fast_two_sum: normalised when |s| >= |e|; under cancellation
  // (|e| > |s|) an unevaluated pair whose sum is the dot product to the same absolute error.
  __device__ __forceinline__ df32 raw() const { return fast_two_sum(s, e); }
};

__device__ __forceinline__ df32 fabs(df32 x) { return x.hi < 0.f ? -x : x; }
__device__ __forceinline__ bool operator<(df32 x, df32 y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
__device__ __forceinline__ df32 fmax(df32 x, df32 y) { return x < y ? y : x; }
using ::fabs;
using ::fmax;

// Scalar-type helpers so templated kernels read the same for double and df32.
template <typename T> __device__ __forceinline__ T from_double(double d);
template <> __device__ __forceinline__ double from_double<double>(double d) { return d; }
template <> __device__ __forceinline__ df32 from_double<df32>(double d) { return df_from(d); }
template <> __device__ __forceinline__ float from_double<float>(double d) { return __double2float_rn(d); }

// Arithmetic of the viscous branch (gradients, gradient traces, stress and heat flux): the element
// arithmetic T, or, with FP32_VISCOUS on the double-float path (FR_PREC_MIXED_VF32), plain FP32.
// These terms are scaled by the viscosity, so their FP32 rounding enters the residual in
// proportion to 1/Re (the gradients are taken of the perturbation from the element's first point,
// so large state values do not cancel in FP32).
template <typename T, bool FP32_VISCOUS> struct GradOf { using type = T; };
template <> struct GradOf<df32, true> { using type = float; };
template <typename TG> __device__ __forceinline__ TG to_g(double x);
template <> __device__ __forceinline__ double to_g<double>(double x) { return x; }
template <typename TG> __device__ __forceinline__ TG to_g(df32 x);
template <> __device__ __forceinline__ float to_g<float>(df32 x) { return __fadd_rn(x.hi, x.lo); }
template <> __device__ __forceinline__ df32 to_g<df32>(df32 x) { return x; }
template <typename T> __device__ __forceinline__ T from_g(double x);
template <> __device__ __forceinline__ double from_g<double>(double x) { return x; }
template <typename T> __device__ __forceinline__ T from_g(float x);
template <> __device__ __forceinline__ df32 from_g<df32>(float x) { return df(x, 0.f); }
template <typename T> __device__ __forceinline__ T from_g(df32 x);
template <> __device__ __forceinline__ df32 from_g<df32>(df32 x) { return x; }

}  // namespace frx
