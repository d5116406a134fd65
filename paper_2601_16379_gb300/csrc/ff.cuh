// Float-float ("double-float") arithmetic for the FP64-class tensor-core path.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  On this GPU the FP64 pipe runs at a small fraction
// of the FP32 rate, so the bulk transforms of the FP64-class path (the k-mesh
// DFTs of the pair tensor, Algorithm 2) run in float-float: each operation is a
// handful of FP32 instructions built on the error-free transformations
//   TwoSum  (Knuth):  s = fl(a + b),  e = (a - (s - b')) + (b - b'),  b' = s - a
//   TwoProd (FMA):    p = fl(a b),    e = fma(a, b, -p)
// (Dekker 1971; the "sloppy" addition of Bailey's double-double library, whose
// error is bounded relative to the operands rather than to the result).  The
// relative error of a multiply or add is ~2^-44, far below what the ERIs need.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace isdf {

struct ffloat {
  float hi, lo;
  ffloat() = default;
  __host__ __device__ __forceinline__ constexpr ffloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ ffloat(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ __forceinline__ ffloat(float v) : hi(v), lo(0.f) {}
  // from double: the float nearest to v and the float nearest to the rest
  __host__ __device__ __forceinline__ ffloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ __forceinline__ double to_double() const { return (double)hi + (double)lo; }
};

// complex float-float (16 bytes, the size of a complex128)
struct ffcomplex {
  ffloat x, y;
};

__host__ __device__ __forceinline__ ffloat ff_fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = a + b;
  return ffloat(s, b - (s - a));
}
__host__ __device__ __forceinline__ ffloat ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return ffloat(s, (a - (s - bb)) + (b - bb));
}

__host__ __device__ __forceinline__ ffloat operator+(ffloat a, ffloat b) {
  ffloat s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__host__ __device__ __forceinline__ ffloat operator-(ffloat a) { return ffloat(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ ffloat operator-(ffloat a, ffloat b) { return a + (-b); }
__host__ __device__ __forceinline__ ffloat operator*(ffloat a, ffloat b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return ff_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ ffloat& operator+=(ffloat& a, ffloat b) { return a = a + b; }
__host__ __device__ __forceinline__ ffloat& operator-=(ffloat& a, ffloat b) { return a = a - b; }
__host__ __device__ __forceinline__ ffloat& operator*=(ffloat& a, ffloat b) { return a = a * b; }
// scaling by a power of two is exact
__host__ __device__ __forceinline__ ffloat ff_ldexp(ffloat a, int e) {
  return ffloat(ldexpf(a.hi, e), ldexpf(a.lo, e));
}

__host__ __device__ __forceinline__ ffcomplex cmul(ffcomplex a, ffcomplex b) {
  return ffcomplex{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

}  // namespace isdf
