// Double-float ("float-float") arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, giving about 48 significant bits with FP32 instructions only.
// Built from the error-free transformations TwoSum (Knuth) and TwoProd (with a fused
// multiply-add); used where FP64 would otherwise be needed in an inner loop, since FP64 runs
// at 1/64 of the FP32 rate on this GPU.  No operation here may be re-associated or contracted:
// the file is compiled without fast-math, and every product whose rounding matters is an
// explicitly rounded multiply (__fmul_rn), which the compiler never fuses into an addition.
#pragma once
#include <cuda_runtime.h>

namespace dmpc {

struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_make(float h) { return {h, 0.f}; }
__device__ __forceinline__ dfl df_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (any magnitudes)
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ dfl quick_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return {s, e};
}
// p + e = a * b exactly
__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  return {p, e};
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  dfl s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
// a * f with f a float
__device__ __forceinline__ dfl df_mulf(dfl a, float f) {
  dfl p = two_prod(a.hi, f);
  p.lo = fmaf(a.lo, f, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  dfl p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, p.lo);
}
// acc + f * a, f a float (one rounding of the low part)
__device__ __forceinline__ dfl df_fmaf(dfl acc, float f, dfl a) { return df_add(acc, df_mulf(a, f)); }

// a / b: float quotient plus one correction from the double-float remainder (Dekker's method)
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  const float q1 = a.hi / b.hi;
  const dfl r = df_sub(a, df_mulf(b, q1));
  const float q2 = r.hi / b.hi;
  return quick_two_sum(q1, q2);
}

// Compensated accumulation, the Dot2 scheme of Ogita, Rump and Oishi (2005): s is the running
// FP32 sum and c collects the exact rounding error of every addition (TwoSum) and product
// (TwoProd) together with the low-order cross products, so s + c is as accurate as a sum carried
// in twice the precision and then rounded.  The dependent chain per term is one addition on s,
// with the error terms hanging off it, instead of the renormalising double-float addition.
struct dacc {
  float s, c;
};
__device__ __forceinline__ dacc dacc_zero() { return {0.f, 0.f}; }
__device__ __forceinline__ void dacc_add(dacc& a, float x) {
  const float t = a.s + x;
  const float z = t - a.s;
  a.c += (a.s - (t - z)) + (x - z);
  a.s = t;
}
__device__ __forceinline__ void dacc_add(dacc& a, dfl x) {
  dacc_add(a, x.hi);
  a.c += x.lo;
}
// a += m * v, m a float
__device__ __forceinline__ void dacc_fma(dacc& a, float m, dfl v) {
  const float p = __fmul_rn(m, v.hi);
  const float e = fmaf(m, v.hi, -p);
  dacc_add(a, p);
  a.c += fmaf(m, v.lo, e);
}
// a += u * v, both double-float (u.lo * v.lo is below the precision kept)
__device__ __forceinline__ void dacc_fma(dacc& a, dfl u, dfl v) {
  const float p = __fmul_rn(u.hi, v.hi);
  const float e = fmaf(u.hi, v.hi, -p);
  dacc_add(a, p);
  a.c += fmaf(u.hi, v.lo, fmaf(u.lo, v.hi, e));
}
__device__ __forceinline__ dfl dacc_get(const dacc& a) { return two_sum(a.s, a.c); }

// Sum over a warp (butterfly; every lane gets the same value).
__device__ __forceinline__ dfl df_warp_sum(dfl v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    dfl o;
    o.hi = __shfl_xor_sync(0xffffffffu, v.hi, off);
    o.lo = __shfl_xor_sync(0xffffffffu, v.lo, off);
    v = df_add(v, o);
  }
  return v;
}

}  // namespace dmpc
