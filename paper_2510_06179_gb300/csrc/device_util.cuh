// Device utilities for the DiffMPC hot path on sm_103a: forward-mode dual numbers,
// hyper-dual numbers for mixed second derivatives, and "team" primitives (a team is the
// group of threads that owns one OCP: one or more whole warps).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dmpc {

// ------------------------------------------------------------------------------------
// Scalar math overloads used by the model templates (float / double / Dual / HDual).
__device__ __forceinline__ float m_sin(float x) { return sinf(x); }
__device__ __forceinline__ float m_cos(float x) { return cosf(x); }
__device__ __forceinline__ float m_tan(float x) { return tanf(x); }
__device__ __forceinline__ float m_atan(float x) { return atanf(x); }
__device__ __forceinline__ float m_abs(float x) { return fabsf(x); }
__device__ __forceinline__ float m_val(float x) { return x; }
__device__ __forceinline__ double m_sin(double x) { return sin(x); }
__device__ __forceinline__ double m_cos(double x) { return cos(x); }
__device__ __forceinline__ double m_tan(double x) { return tan(x); }
__device__ __forceinline__ double m_atan(double x) { return atan(x); }
__device__ __forceinline__ double m_abs(double x) { return fabs(x); }
__device__ __forceinline__ double m_val(double x) { return x; }

// ------------------------------------------------------------------------------------
// Dual<N>: value and N tangents (first derivatives along N seed directions).
template <int N>
struct Dual {
  float v;
  float d[N];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(float c) : v(c) {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = 0.f;
  }
  __device__ __forceinline__ static Dual seed(float c, int k) {
    Dual r(c);
    if (k >= 0 && k < N) r.d[k] = 1.f;
    return r;
  }
};

template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = fmaf(a.v, b.d[i], b.v * a.d[i]);
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(float s, const Dual<N>& a) {
  Dual<N> r; r.v = s * a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = s * a.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> operator*(const Dual<N>& a, float s) { return s * a; }
template <int N>
__device__ __forceinline__ Dual<N> operator+(const Dual<N>& a, float s) { Dual<N> r = a; r.v += s; return r; }
template <int N>
__device__ __forceinline__ Dual<N> operator+(float s, const Dual<N>& a) { return a + s; }
template <int N>
__device__ __forceinline__ Dual<N> operator-(const Dual<N>& a, float s) { Dual<N> r = a; r.v -= s; return r; }
template <int N>
__device__ __forceinline__ Dual<N> operator-(float s, const Dual<N>& a) { Dual<N> r = -a; r.v += s; return r; }
template <int N>
__device__ __forceinline__ Dual<N> chain(const Dual<N>& a, float f, float df) {
  Dual<N> r; r.v = f;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = df * a.d[i];
  return r;
}
template <int N>
__device__ __forceinline__ Dual<N> recip(const Dual<N>& a) { float iv = 1.f / a.v; return chain(a, iv, -iv * iv); }
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) { return a * recip(b); }
template <int N>
__device__ __forceinline__ Dual<N> operator/(const Dual<N>& a, float s) { return a * (1.f / s); }
template <int N>
__device__ __forceinline__ Dual<N> operator/(float s, const Dual<N>& a) { return s * recip(a); }
template <int N>
__device__ __forceinline__ Dual<N> m_sin(const Dual<N>& a) { float s, c; sincosf(a.v, &s, &c); return chain(a, s, c); }
template <int N>
__device__ __forceinline__ Dual<N> m_cos(const Dual<N>& a) { float s, c; sincosf(a.v, &s, &c); return chain(a, c, -s); }
template <int N>
__device__ __forceinline__ Dual<N> m_tan(const Dual<N>& a) { float t = tanf(a.v); return chain(a, t, 1.f + t * t); }
template <int N>
__device__ __forceinline__ Dual<N> m_atan(const Dual<N>& a) { return chain(a, atanf(a.v), 1.f / (1.f + a.v * a.v)); }
template <int N>
__device__ __forceinline__ Dual<N> m_abs(const Dual<N>& a) { return a.v < 0.f ? -a : a; }
template <int N>
__device__ __forceinline__ float m_val(const Dual<N>& a) { return a.v; }

// ------------------------------------------------------------------------------------
// HDual<P>: value v, first derivative e along one direction (the adjoint-solution
// direction z~), first derivatives t[P] along P parameter directions, and the mixed
// second derivatives et[P] = d2/(d e d theta_j).  Used by the theta-contraction of the
// backward pass: d/dtheta [ lambda^T (dPhi/dz) z~ ] needs exactly these mixed terms.
template <int P>
struct HDual {
  float v, e;
  float t[P], et[P];
  __device__ __forceinline__ HDual() {}
  __device__ __forceinline__ HDual(float c) : v(c), e(0.f) {
#pragma unroll
    for (int i = 0; i < P; ++i) { t[i] = 0.f; et[i] = 0.f; }
  }
};

template <int P>
__device__ __forceinline__ HDual<P> operator+(const HDual<P>& a, const HDual<P>& b) {
  HDual<P> r; r.v = a.v + b.v; r.e = a.e + b.e;
#pragma unroll
  for (int i = 0; i < P; ++i) { r.t[i] = a.t[i] + b.t[i]; r.et[i] = a.et[i] + b.et[i]; }
  return r;
}
template <int P>
__device__ __forceinline__ HDual<P> operator-(const HDual<P>& a) {
  HDual<P> r; r.v = -a.v; r.e = -a.e;
#pragma unroll
  for (int i = 0; i < P; ++i) { r.t[i] = -a.t[i]; r.et[i] = -a.et[i]; }
  return r;
}
template <int P>
__device__ __forceinline__ HDual<P> operator-(const HDual<P>& a, const HDual<P>& b) { return a + (-b); }
template <int P>
__device__ __forceinline__ HDual<P> operator*(const HDual<P>& a, const HDual<P>& b) {
  HDual<P> r; r.v = a.v * b.v; r.e = fmaf(a.e, b.v, a.v * b.e);
#pragma unroll
  for (int i = 0; i < P; ++i) {
    r.t[i] = fmaf(a.t[i], b.v, a.v * b.t[i]);
    r.et[i] = fmaf(a.et[i], b.v, fmaf(a.e, b.t[i], fmaf(a.t[i], b.e, a.v * b.et[i])));
  }
  return r;
}
template <int P>
__device__ __forceinline__ HDual<P> operator*(float s, const HDual<P>& a) {
  HDual<P> r; r.v = s * a.v; r.e = s * a.e;
#pragma unroll
  for (int i = 0; i < P; ++i) { r.t[i] = s * a.t[i]; r.et[i] = s * a.et[i]; }
  return r;
}
template <int P>
__device__ __forceinline__ HDual<P> operator*(const HDual<P>& a, float s) { return s * a; }
template <int P>
__device__ __forceinline__ HDual<P> operator+(const HDual<P>& a, float s) { HDual<P> r = a; r.v += s; return r; }
template <int P>
__device__ __forceinline__ HDual<P> operator+(float s, const HDual<P>& a) { return a + s; }
template <int P>
__device__ __forceinline__ HDual<P> operator-(const HDual<P>& a, float s) { HDual<P> r = a; r.v -= s; return r; }
template <int P>
__device__ __forceinline__ HDual<P> operator-(float s, const HDual<P>& a) { HDual<P> r = -a; r.v += s; return r; }
// unary phi with phi'(v) = d1 and phi''(v) = d2
template <int P>
__device__ __forceinline__ HDual<P> chain2(const HDual<P>& a, float f, float d1, float d2) {
  HDual<P> r; r.v = f; r.e = d1 * a.e;
#pragma unroll
  for (int i = 0; i < P; ++i) { r.t[i] = d1 * a.t[i]; r.et[i] = fmaf(d1, a.et[i], d2 * a.e * a.t[i]); }
  return r;
}
template <int P>
__device__ __forceinline__ HDual<P> recip(const HDual<P>& a) {
  float iv = 1.f / a.v;
  return chain2(a, iv, -iv * iv, 2.f * iv * iv * iv);
}
template <int P>
__device__ __forceinline__ HDual<P> operator/(const HDual<P>& a, const HDual<P>& b) { return a * recip(b); }
template <int P>
__device__ __forceinline__ HDual<P> operator/(const HDual<P>& a, float s) { return a * (1.f / s); }
template <int P>
__device__ __forceinline__ HDual<P> operator/(float s, const HDual<P>& a) { return s * recip(a); }
template <int P>
__device__ __forceinline__ HDual<P> m_sin(const HDual<P>& a) { float s, c; sincosf(a.v, &s, &c); return chain2(a, s, c, -s); }
template <int P>
__device__ __forceinline__ HDual<P> m_cos(const HDual<P>& a) { float s, c; sincosf(a.v, &s, &c); return chain2(a, c, -s, -c); }
template <int P>
__device__ __forceinline__ HDual<P> m_tan(const HDual<P>& a) {
  float t = tanf(a.v); float s2 = 1.f + t * t; return chain2(a, t, s2, 2.f * t * s2);
}
template <int P>
__device__ __forceinline__ HDual<P> m_atan(const HDual<P>& a) {
  float d = 1.f / (1.f + a.v * a.v); return chain2(a, atanf(a.v), d, -2.f * a.v * d * d);
}
template <int P>
__device__ __forceinline__ HDual<P> m_abs(const HDual<P>& a) { return a.v < 0.f ? -a : a; }
template <int P>
__device__ __forceinline__ float m_val(const HDual<P>& a) { return a.v; }

// ------------------------------------------------------------------------------------
// Team: TEAM threads (a multiple of 32) cooperating on one OCP.  Teams of one warp
// synchronise with __syncwarp; larger teams use a named barrier (id = team index + 1).
template <int TEAM>
struct Team {
  static constexpr int NW = TEAM / 32;
  int lane;          // 0 .. TEAM-1
  int bar_id;        // named barrier id (TEAM > 32)
  float* red;        // per-team reduction scratch: 2 buffers x NW x RED_MAX floats
  int buf;
  static constexpr int RED_MAX = 48;

  __device__ __forceinline__ void sync() const {
    if (TEAM <= 32) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(TEAM) : "memory");
    }
  }

  // Sum each of NV values over the team; every thread receives the totals, bitwise
  // identical across threads (butterfly pairs add commutatively; cross-warp partials are
  // summed in the same order by all threads).  Acts as a full team barrier.
  template <int NV>
  __device__ __forceinline__ void sum(float (&v)[NV]) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int j = 0; j < NV; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
    }
    if (TEAM <= 32) {
      __syncwarp();
      return;
    }
    float* rb = red + buf * (NW * RED_MAX);
    int w = lane >> 5;
    if ((lane & 31) == 0) {
#pragma unroll
      for (int j = 0; j < NV; ++j) rb[w * RED_MAX + j] = v[j];
    }
    sync();
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      float s = 0.f;
      for (int q = 0; q < NW; ++q) s += rb[q * RED_MAX + j];
      v[j] = s;
    }
    buf ^= 1;
  }

  // Bitwise OR of an int over the team (status flags); every thread receives the result.
  __device__ __forceinline__ int bor(int v) {
    v = __reduce_or_sync(0xffffffffu, (unsigned)v);
    if (TEAM <= 32) return v;
    float* rb = red + buf * (NW * RED_MAX);
    int w = lane >> 5;
    if ((lane & 31) == 0) reinterpret_cast<int*>(rb)[w] = v;
    sync();
    int o = 0;
    for (int q = 0; q < NW; ++q) o |= reinterpret_cast<int*>(rb)[q];
    buf ^= 1;
    return o;
  }

  // double-precision variant (each double takes two float slots of the scratch).
  template <int NV>
  __device__ __forceinline__ void sum(double (&v)[NV]) {
    static_assert(2 * NV <= RED_MAX, "reduction too wide");
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int j = 0; j < NV; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
    }
    if (TEAM <= 32) {
      __syncwarp();
      return;
    }
    double* rb = reinterpret_cast<double*>(red + buf * (NW * RED_MAX));
    int w = lane >> 5;
    if ((lane & 31) == 0) {
#pragma unroll
      for (int j = 0; j < NV; ++j) rb[w * (RED_MAX / 2) + j] = v[j];
    }
    sync();
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = 0.0;
      for (int q = 0; q < NW; ++q) s += rb[q * (RED_MAX / 2) + j];
      v[j] = s;
    }
    buf ^= 1;
  }
};

}  // namespace dmpc
