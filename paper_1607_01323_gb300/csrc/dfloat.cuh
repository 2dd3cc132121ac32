// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32
// numbers (|lo| <= ulp(hi)), about 48 significant bits.  Products use the exact
// FMA-based product error, sums Knuth's TwoSum, so every operation is accurate
// to about 2^-46 relative (Dekker, "A floating-point technique for extending
// the available precision", Numer. Math. 18 (1971); Knuth, TAOCP vol. 2,
// 4.2.2).  It exists because this GPU issues 64 FP32 FMAs per FP64 FMA: an FP64
// operator evaluated in double-float on the FP32 pipes keeps the FP64 result
// to the parity tolerance (1e-12 of ||A|| ||x||) at a fraction of the cost.
//
// Conversions to and from double use integer and FP32 instructions (the FP64
// pipe only on the rare out-of-range path of the unscaled conversion) and
// carry a per-call power-of-two scale (below).  Kernels issue the loads of a
// group of values before converting them: the out-of-line call of a rare
// path would otherwise keep each load waiting for the previous conversion.
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

// ------------------------------------------------------------ conversions
// Each call that evaluates FP64 data in double-float first finds a scale
// exponent s with max |v| 2^-s in [1/2, 1) over the finite entries of its input
// (df_scale_key below, reduced by the launcher's scale pass), converts every
// input value to v 2^-s and every result back with 2^s (both exact powers of
// two).  Values then keep their 48 bits wherever they lie in the FP64 range;
// entries below 2^-103 of the largest become 0, which is far under the
// operator's tolerance (relative to the largest entry).  NaN and +-inf pass
// through as NaN / +-inf, so a non-finite input gives a non-finite output.

// key of a double: E + kScaleBias for a finite nonzero value in [2^E, 2^(E+1))
// (E in [-1074, 1023], subnormals included), 0 for zero, NaN and +-inf
constexpr int kScaleBias = 1100;
__host__ __device__ inline int df_scale_from_key(int key) { return key > 0 ? key - kScaleBias + 1 : 0; }

__device__ __forceinline__ int df_scale_key(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int ex = (int)((u >> 52) & 0x7ff);
  if (ex == 0x7ff) return 0;
  if (ex != 0) return ex - 1023 + kScaleBias;
  const unsigned long long man = u & 0xfffffffffffffull;
  if (!man) return 0;
  return (63 - __clzll((long long)man)) - 1074 + kScaleBias;
}

// Block-wide maximum of the keys of one pass over the input, one atomicMax per
// block into dsc[0]; the last block to count itself in dsc[1] turns the
// maximum into the scale exponent dsc[2] and clears dsc[0] and dsc[1] for the
// next call (no waiting: each block counts once).  Called by every thread of
// every block of the grid.
__device__ __forceinline__ void df_scale_reduce(int key, int* dsc) {
  __shared__ int wmax[32];
  key = __reduce_max_sync(0xffffffffu, key);
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = key;
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) k = max(k, wmax[w]);
    if (k) atomicMax(dsc, k);
    __threadfence();  // this block's maximum is visible before its count
    if (atomicAdd(reinterpret_cast<unsigned*>(dsc + 1), 1u) == gridDim.x * gridDim.y - 1) {
      __threadfence();
      dsc[2] = df_scale_from_key(atomicExch(dsc, 0));
      atomicExch(dsc + 1, 0);
    }
  }
}

// double -> double-float of d 2^-s, the cases outside the common range:
// +-inf stays +-inf, NaN becomes a quiet NaN, subnormal doubles are
// normalised first, values beyond 2^127 of the scale become +-inf (not met
// when s is the call's scale) and values below 2^-103 of it become 0
static __device__ __noinline__ dfl df_from_double_rare(unsigned long long u, int s) {
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  int ex = (int)((u >> 52) & 0x7ff);
  unsigned long long man = u & 0xfffffffffffffull;
  if (ex == 0x7ff) return dfl(__int_as_float((int)(sign | (man ? 0x7fc00000u : 0x7f800000u))), 0.f);
  if (ex == 0) {
    if (!man) return dfl(__int_as_float((int)sign), 0.f);
    const int b = 63 - __clzll((long long)man);
    man = (man << (52 - b)) & 0xfffffffffffffull;
    ex = b - 51;
  }
  const int fe = ex - 1023 - s + 127;
  if (fe > 254) return dfl(__int_as_float((int)(sign | 0x7f800000u)), 0.f);
  if (fe < 24) return dfl(__int_as_float((int)sign), 0.f);
  const float hi = __int_as_float((int)(sign | ((unsigned)fe << 23) | (unsigned)(man >> 29)));
  const unsigned r = (unsigned)(man >> 6) & 0x7fffffu;
  const float rf = __int_as_float(0x4B000000 | (int)r) - 8388608.0f;
  const int se = fe - 46;
  const float scale = se > 0 ? __int_as_float(se << 23) : 0.f;
  return dfl(hi, __int_as_float(__float_as_int(rf * scale) | (int)sign));
}

// double -> double-float of d 2^-s without FP64 instructions: the top 24
// significant bits become hi (truncated), the next 23 lo.  The common case
// (a normal double whose scaled exponent leaves room for lo) takes one
// range test; everything else goes through df_from_double_rare.
__device__ __forceinline__ dfl df_from_double(double d, int s) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int ex = (int)((u >> 52) & 0x7ff);
  const int fe = ex - 1023 - s + 127;  // biased FP32 exponent of hi
  if (__builtin_expect((unsigned)(ex - 1) > 2045u || (unsigned)(fe - 47) > 207u, 0)) return df_from_double_rare(u, s);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const float hi = __int_as_float((int)(sign | ((unsigned)fe << 23) | ((unsigned)(u >> 29) & 0x7fffffu)));
  // the next 23 significand bits, r exactly in FP32 (2^23 trick), weight 2^(fe - 127 - 46)
  const unsigned r = (unsigned)(u >> 6) & 0x7fffffu;
  const float rf = __int_as_float(0x4B000000 | (int)r) - 8388608.0f;
  return dfl(hi, __int_as_float(__float_as_int(rf * __int_as_float((fe - 46) << 23)) | (int)sign));
}

// unscaled conversion of coefficients and geometry (their range is the
// mesh's), all inline: the fast path of df_from_double(d, 0); a value whose
// FP32 exponent leaves no room for a normal lo (|d| < 2^-80 or >= 2^128),
// zero, inf or NaN becomes its FP32 rounding with lo = 0
__device__ __forceinline__ dfl df_from_double(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int fe = (int)((u >> 52) & 0x7ff) - 1023 + 127;
  if (__builtin_expect((unsigned)(fe - 47) > 207u, 0)) return dfl(__double2float_rn(d), 0.f);
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const float hi = __int_as_float((int)(sign | ((unsigned)fe << 23) | ((unsigned)(u >> 29) & 0x7fffffu)));
  const unsigned r = (unsigned)(u >> 6) & 0x7fffffu;
  const float rf = __int_as_float(0x4B000000 | (int)r) - 8388608.0f;
  return dfl(hi, __int_as_float(__float_as_int(rf * __int_as_float((fe - 46) << 23)) | (int)sign));
}

// f 2^s as a double, the cases outside the common range: FP32 zeros and
// subnormals (below the scaled range's resolution) give 0, inf / NaN stay
// inf / NaN, results beyond the FP64 range +-inf, results below the normal
// FP64 range the correctly rounded (to nearest even) subnormal
static __device__ __noinline__ double f32_widen_rare(float f, int s) {
  const unsigned b = (unsigned)__float_as_int(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned long long sg = (unsigned long long)(b & 0x80000000u) << 32;
  const unsigned long long mant = (unsigned long long)(b & 0x7fffffu);
  if (e == 0) return __longlong_as_double((long long)sg);
  if (e == 0xff) return __longlong_as_double((long long)(sg | (0x7ffull << 52) | (mant << 29)));
  const int E = (int)e - 127 + s;  // unbiased exponent of the result
  if (E > 1023) return __longlong_as_double((long long)(sg | (0x7ffull << 52)));
  if (E >= -1022) return __longlong_as_double((long long)(sg | ((unsigned long long)(E + 1023) << 52) | (mant << 29)));
  // value = m 2^(E - 23) with m = 2^23 + mant; as a multiple of 2^-1074:
  // m 2^-sh, exact for sh <= 0, rounded to nearest even for sh > 0
  const int sh = -1074 - (E - 23);
  const unsigned long long m = (1ull << 23) | mant;
  if (sh <= 0) return __longlong_as_double((long long)(sg | (m << -sh)));
  if (sh > 25) return __longlong_as_double((long long)sg);  // below half the smallest subnormal
  unsigned long long q = m >> sh;
  const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  if (rem > half || (rem == half && (q & 1))) ++q;  // a carry into bit 52 gives the smallest normal
  return __longlong_as_double((long long)(sg | q));
}

// f 2^s as a double, exact in the common case: one range test
__device__ __forceinline__ double f32_widen(float f, int s) {
  const unsigned b = (unsigned)__float_as_int(f);
  const int e = (int)((b >> 23) & 0xffu);
  const int E = e - 127 + 1023 + s;  // biased FP64 exponent
  if (__builtin_expect((unsigned)(e - 1) > 253u || (unsigned)(E - 1) > 2045u, 0)) return f32_widen_rare(f, s);
  return __longlong_as_double((long long)(((unsigned long long)(b & 0x80000000u) << 32) |
                                          ((unsigned long long)E << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}
__device__ __forceinline__ double f32_widen(float f) { return f32_widen(f, 0); }

// double-float -> double of a 2^s: both parts widen exactly, one FP64 add
__device__ __forceinline__ double df_to_double(dfl a, int s) { return f32_widen(a.hi, s) + f32_widen(a.lo, s); }
__device__ __forceinline__ double df_to_double(dfl a) { return df_to_double(a, 0); }
#endif  // __CUDACC__

}  // namespace sipg
