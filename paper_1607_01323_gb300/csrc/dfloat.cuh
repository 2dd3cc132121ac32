// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi)), about 48 significant bits.  Products use the exact
// FMA-based product error, sums Knuth's TwoSum, so every operation is accurate
// to about 2^-46 relative (Dekker, "A floating-point technique for extending
// the available precision", Numer. Math. 18 (1971); Knuth, TAOCP vol. 2,
// 4.2.2).  It exists because this GPU issues 64 FP32 FMAs per FP64 FMA: an FP64
// operator evaluated in double-float on the FP32 pipes keeps the FP64 result
// to the parity tolerance (1e-12 of ||A|| ||x||) at a fraction of the cost.
//
// Conversions to and from double use only integer and FP32 instructions (no
// FP64 pipe): the top 24 mantissa bits of the double become hi (truncated),
// the next 23 become lo.
#pragma once

#include <cstdint>

namespace sipg {

#ifdef __CUDACC__
using ::fma;  // keep the float / double overloads visible next to the double-float one
#endif

struct __align__(8) dfl {  // 8-byte aligned: one 64-bit load or store per value
  float hi, lo;
  __host__ __device__ constexpr dfl() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  // only used for small integer constants (0, 1, 2, 0.5) in the kernels
  __host__ __device__ constexpr explicit dfl(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ constexpr explicit dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

#ifdef __CUDACC__
// exact sum s + err = a + b (TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = a + b;
  const float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ dfl df_norm(float s, float t) {
  const float hi = s + t;
  return dfl(hi, t - (hi - s));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df_norm(s, e + (a.lo + b.lo));
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_norm(p, e);
}

__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { return a = a * b; }

// c + a b with the exact product error and TwoSum
__device__ __forceinline__ dfl fma(dfl a, dfl b, dfl c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, err;
  two_sum(c.hi, p, s, err);
  return df_norm(s, err + (c.lo + e));
}

// sum_b a[b] * v[b] over n terms: exact product errors and TwoSum on the high
// parts, all error terms in one FP32 accumulator, one renormalisation at the
// end (12 instead of 15 FP32 operations per term; the accumulated error terms
// are ~2^-24 of the sum, so their FP32 rounding stays ~n 2^-48 relative)
template <int N>
__device__ __forceinline__ dfl df_dot(const dfl* __restrict__ a, const dfl (&v)[N]) {
  float s = 0.f, err = 0.f;
#pragma unroll
  for (int b = 0; b < N; ++b) {
    const float p = a[b].hi * v[b].hi;
    float e = fmaf(a[b].hi, v[b].hi, -p);
    e = fmaf(a[b].hi, v[b].lo, e);
    e = fmaf(a[b].lo, v[b].hi, e);
    float t, te;
    two_sum(s, p, t, te);
    s = t;
    err += te + e;
  }
  return df_norm(s, err);
}

__device__ __forceinline__ bool operator!=(dfl a, dfl b) { return a.hi != b.hi || a.lo != b.lo; }
__device__ __forceinline__ bool operator>(dfl a, dfl b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// double -> double-float without FP64 instructions.  Values below 2^-100 in
// magnitude become zero; the tolerance of the operator is relative to the
// largest entry, so this is far below it.
__device__ __forceinline__ dfl df_from_double(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const int ex = (int)((u >> 52) & 0x7ff);
  const int fe = ex - 1023 + 127;
  if (fe < 24 || fe > 254) return dfl(0.f, 0.f);  // tiny, zero, or out of FP32 range
  const unsigned man_hi = (unsigned)(u >> 29) & 0x7fffffu;
  const float hi = __int_as_float((int)(sign | ((unsigned)fe << 23) | man_hi));
  // remaining 29 mantissa bits; keep the top 23 (exact in FP32 via the 2^23 trick)
  const unsigned r = (unsigned)(u >> 6) & 0x7fffffu;
  const float rf = __int_as_float(0x4B000000 | (int)r) - 8388608.0f;  // = r exactly
  // value of r: r * 2^(ex - 1023 - 52 + 6); scale by an FP32 power of two
  const int se = ex - 1023 - 46 + 127;
  const float scale = se > 0 ? __int_as_float(se << 23) : 0.f;
  const float lo = __int_as_float(__float_as_int(rf * scale) | (int)sign);
  return dfl(hi, lo);
}

// FP32 -> FP64 widening by bit manipulation (exact; FP32 denormals become 0)
__device__ __forceinline__ double f32_widen(float f) {
  const unsigned b = (unsigned)__float_as_int(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned long long s = (unsigned long long)(b & 0x80000000u) << 32;
  if (e == 0) return __longlong_as_double((long long)s);
  const unsigned long long bits = s | ((unsigned long long)(e - 127 + 1023) << 52) |
                                  ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}

// double-float -> double: both parts widen exactly, one FP64 add
__device__ __forceinline__ double df_to_double(dfl a) { return f32_widen(a.hi) + f32_widen(a.lo); }
#endif  // __CUDACC__

}  // namespace sipg
