// Shared device helpers for the IE kernels: complex arithmetic in float2/double2, launch checks.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace ie {

constexpr int TWN = 1024;  // length of the twiddle table exp(-2 pi i k / TWN); longest pencil

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using C = typename cplx_t<T>::type;

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T re, T im) { C<T> c; c.x = re; c.y = im; return c; }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// conj(a) * b
template <typename V> __host__ __device__ __forceinline__ V cmulc(V a, V b) {
  V r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.x * b.y - a.y * b.x;
  return r;
}
// a * conj(b)
template <typename V> __host__ __device__ __forceinline__ V cmul_conjb(V a, V b) {
  V r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
template <typename V> __host__ __device__ __forceinline__ V czero() { V r; r.x = 0; r.y = 0; return r; }
// y + a, or y - a when neg
__device__ __forceinline__ float2 add_signed(float2 y, bool neg, float2 a) {
  const float s = neg ? -1.f : 1.f;
  return make_float2(fmaf(s, a.x, y.x), fmaf(s, a.y, y.y));
}
__device__ __forceinline__ double2 add_signed(double2 y, bool neg, double2 a) {
  const double s = neg ? -1.0 : 1.0;
  return make_double2(fma(s, a.x, y.x), fma(s, a.y, y.y));
}
// real scalar times complex
template <typename S, typename V> __host__ __device__ __forceinline__ V cscale(S s, V a) {
  V r;
  r.x = s * a.x;
  r.y = s * a.y;
  return r;
}

__device__ __forceinline__ float2 to_c(double2 a, float) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_c(double2 a, double) { return a; }
__device__ __forceinline__ float2 to_c(float2 a, float) { return a; }
__device__ __forceinline__ double2 to_c64(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 to_c64(double2 a) { return a; }

// ------------------------------------------------------------------ double-float arithmetic
// A real number held as an unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2), giving about
// 46 significant bits from the FP32 pipes. Built from the error-free transformations TwoSum (Knuth),
// FastTwoSum (Dekker) and the FMA form of TwoProd; additions use the short ("sloppy") form whose
// error is bounded relative to |a| + |b|, which is what the normwise error analysis of the FFT needs.
struct df {
  float hi, lo;
  __host__ __device__ constexpr df() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};
__host__ __device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = a + b;
  return df(s, b - (s - a));
}
__host__ __device__ __forceinline__ df operator+(df a, df b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return fast_two_sum(s, e + (a.lo + b.lo));
}
__host__ __device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__host__ __device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ double to_double(df a) { return (double)a.hi + (double)a.lo; }

struct dfc {  // complex double-float, 16 bytes like double2
  df x, y;
};
template <> struct cplx_t<df> { using type = dfc; };
__host__ __device__ __forceinline__ dfc operator+(dfc a, dfc b) { return dfc{a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ dfc operator-(dfc a, dfc b) { return dfc{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ dfc add_signed(dfc y, bool neg, dfc a) { return neg ? y - a : y + a; }
__device__ __forceinline__ dfc to_c(double2 a, df) { return dfc{df(a.x), df(a.y)}; }
__device__ __forceinline__ double2 to_c64(dfc a) { return make_double2(to_double(a.x), to_double(a.y)); }

// Global field and contrast types of a convolution carried out in arithmetic T: the double-float
// kernels read and write complex128 fields and an FP64 contrast.
template <typename T> struct Field {
  using type = C<T>;
  using real = T;
};
template <> struct Field<df> {
  using type = double2;
  using real = double;
};
template <typename T> using FieldC = typename Field<T>::type;
template <typename T> using FieldR = typename Field<T>::real;

// value as stored in the global field of a convolution in arithmetic T
__device__ __forceinline__ float2 to_field(float2 v) { return v; }
__device__ __forceinline__ double2 to_field(double2 v) { return v; }
__device__ __forceinline__ double2 to_field(dfc v) { return to_c64(v); }

// read-only cached load of one complex value
__device__ __forceinline__ float2 ldgv(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldgv(const double2* p) { return __ldg(p); }
__device__ __forceinline__ dfc ldgv(const dfc* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return dfc{df(v.x, v.y), df(v.z, v.w)};
}

}  // namespace ie
