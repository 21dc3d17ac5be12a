// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, giving a 48-bit significand with the FP32
// exponent range.  Addition uses Knuth's error-free two-sum of the leading
// parts plus the trailing parts, multiplication Dekker's product with the
// exact FP32 fma residual (the classic double-double algorithms, applied to
// float pairs).  All operations run on the FP32 pipes, which on this GPU are
// about 64x faster than FP64; the column kernel instantiated with this type
// computes the operator to about 1e-13 relative, enough for the residuals of
// mixed-precision refinement.
//
// Every operation is spelled with the round-to-nearest intrinsics so that the
// compiler can neither contract nor reorder the error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace bemfft {

struct f32x2 {
  float hi, lo;
  __host__ __device__ constexpr f32x2() : hi(0.0f), lo(0.0f) {}
  __host__ __device__ constexpr f32x2(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr f32x2(float f) : hi(f), lo(0.0f) {}
  __host__ __device__ constexpr f32x2(int i) : hi((float)i), lo(0.0f) {}
  __host__ __device__ constexpr f32x2(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

#if defined(__CUDA_ARCH__)
#define FF_ADD(a, b) __fadd_rn(a, b)
#define FF_SUB(a, b) __fsub_rn(a, b)
#define FF_MUL(a, b) __fmul_rn(a, b)
#define FF_FMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define FF_ADD(a, b) ((a) + (b))
#define FF_SUB(a, b) ((a) - (b))
#define FF_MUL(a, b) ((a) * (b))
#define FF_FMA(a, b, c) fmaf(a, b, c)
#endif

// s + e = a + b exactly (no magnitude condition)
__host__ __device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
  s = FF_ADD(a, b);
  const float bb = FF_SUB(s, a);
  e = FF_ADD(FF_SUB(a, FF_SUB(s, bb)), FF_SUB(b, bb));
}
// s + e = a + b exactly when |a| >= |b|
__host__ __device__ __forceinline__ void ff_quick_two_sum(float a, float b, float& s, float& e) {
  s = FF_ADD(a, b);
  e = FF_SUB(b, FF_SUB(s, a));
}

__host__ __device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b) {
  float s, e;
  ff_two_sum(a.hi, b.hi, s, e);
  e = FF_ADD(e, FF_ADD(a.lo, b.lo));
  f32x2 r;
  ff_quick_two_sum(s, e, r.hi, r.lo);
  return r;
}
__host__ __device__ __forceinline__ f32x2 operator-(f32x2 a) { return f32x2(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b) { return a + (-b); }
__host__ __device__ __forceinline__ f32x2 operator*(f32x2 a, f32x2 b) {
  const float p = FF_MUL(a.hi, b.hi);
  float e = FF_FMA(a.hi, b.hi, -p);
  e = FF_FMA(a.hi, b.lo, e);
  e = FF_FMA(a.lo, b.hi, e);
  f32x2 r;
  ff_quick_two_sum(p, e, r.hi, r.lo);
  return r;
}
__host__ __device__ __forceinline__ f32x2& operator+=(f32x2& a, f32x2 b) { return a = a + b; }
__host__ __device__ __forceinline__ f32x2& operator-=(f32x2& a, f32x2 b) { return a = a - b; }
__host__ __device__ __forceinline__ f32x2& operator*=(f32x2& a, f32x2 b) { return a = a * b; }
__host__ __device__ __forceinline__ bool operator>(f32x2 a, int b) { return a.hi > (float)b || (a.hi == (float)b && a.lo > 0.0f); }

#undef FF_ADD
#undef FF_SUB
#undef FF_MUL
#undef FF_FMA

}  // namespace bemfft
