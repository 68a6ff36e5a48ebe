// Double-float arithmetic: a value is the unevaluated sum hi + lo of two fp32
// words (about 48 significant bits), computed on the FP32 pipes with the
// error-free transformations of Dekker (1971, "A floating-point technique for
// extending the available precision") and Knuth (TwoSum), in the accumulate
// form of Ogita, Rump and Oishi (2005, "Accurate sum and dot product", Dot2):
// products are split exactly with one fused multiply-add, sums with TwoSum,
// and the low words are accumulated without renormalising after every term.
//
// Used for the outer CG's operator apply when the hierarchy asks for it: on
// GB300 the FP32 pipes issue about 60 times the FP64 rate, so ~12 fp32
// operations per emulated multiply-add still outrun the FP64 pipe.  The
// exponent range is fp32's: magnitudes must stay within about 1e-30 .. 1e30.
#pragma once

#include <cuda_runtime.h>

namespace pmg {

struct dfloat;
#ifdef __CUDACC__
__device__ __forceinline__ dfloat split_double(double x);
__device__ __forceinline__ double join_double(float hi, float lo);
#endif

struct dfloat {
  float hi, lo;
  __host__ __device__ constexpr dfloat() : hi(0.0f), lo(0.0f) {}
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  // split of a double into hi + lo (host: hi = fl32(x), lo = fl32(x - hi); device:
  // the bit-level split of split_double, which needs no FP64 instruction)
  __host__ __device__ explicit dfloat(double x);
  __host__ __device__ explicit dfloat(int x) : hi((float)x), lo(0.0f) {}
  __host__ __device__ explicit operator double() const;
};

#ifdef __CUDACC__

// Conversions without the FP64 pipe (on GB300 a double <-> float conversion
// costs as much as an FP64 multiply-add).  split_double: hi takes the top 24
// significand bits of x (truncated, so exact as fp32), lo the next 29 bits
// (rounded to 24): |x - (hi + lo)| <= 2^-48 |x|.  Magnitudes outside fp32's
// normal range become 0 or +-inf.
__device__ __forceinline__ dfloat split_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffu);
  const int eh = e - 1023 + 127;                       // fp32 biased exponent of hi
  if (eh <= 0) return dfloat(__int_as_float((int)sign), 0.0f);
  if (eh >= 255) return dfloat(__int_as_float((int)(sign | 0x7f800000u | (e == 0x7ff && (b << 12) ? 0x400000u : 0u))), 0.0f);
  const unsigned long long m = b & 0xfffffffffffffull;  // 52 fraction bits
  const float hi = __int_as_float((int)(sign | ((unsigned)eh << 23) | (unsigned)(m >> 29)));
  const unsigned rem = (unsigned)(m & 0x1fffffffu);   // remainder, units of 2^(e - 1075)
  float lo = __uint2float_rn(rem);
  const int es = e - 1075 + 127;                       // fp32 biased exponent of 2^(e - 1075)
  lo = es > 0 ? __fmul_rn(lo, __int_as_float(es << 23)) : ldexpf(lo, e - 1075);
  return dfloat(hi, sign ? -lo : lo);
}

// fp32 -> fp64 by re-biasing the exponent (normal numbers, zero, inf, nan;
// fp32 subnormals become 0)
__device__ __forceinline__ double widen(float f) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned ef = (u >> 23) & 0xffu;
  const unsigned long long frac = (unsigned long long)(u & 0x7fffffu) << 29;
  if (ef == 0) return __longlong_as_double((long long)sign);
  const unsigned long long ed = (ef == 255) ? 0x7ffull : (unsigned long long)(ef - 127 + 1023);
  return __longlong_as_double((long long)(sign | (ed << 52) | frac));
}

__device__ __forceinline__ double join_double(float hi, float lo) { return widen(hi) + widen(lo); }

// TwoSum: s + t == a + b exactly, s = fl(a + b)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// Fast2Sum (|a| >= |b|): renormalise a pair
__device__ __forceinline__ dfloat renorm(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// a * b: exact product of the high words by one FMA, cross terms into the low word
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dfloat(p, e);
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float s, t;
  two_sum(a.hi, b.hi, s, t);
  return renorm(s, __fadd_rn(t, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }

// c + a * b in the accumulate form (no renormalisation of the result).  Named
// madd, not fma: an fma overload in this namespace would hide ::fma for doubles.
__device__ __forceinline__ dfloat madd(dfloat a, dfloat b, dfloat c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  two_sum(c.hi, p, s, t);
  return dfloat(s, __fadd_rn(__fadd_rn(c.lo, e), t));
}

__device__ __forceinline__ bool operator!=(dfloat a, dfloat b) { return a.hi != b.hi || a.lo != b.lo; }

__device__ __forceinline__ dfloat ldg(const dfloat* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return dfloat(v.x, v.y);
}

#endif  // __CUDACC__

__host__ __device__ inline dfloat::dfloat(double x) {
#ifdef __CUDA_ARCH__
  *this = split_double(x);
#else
  hi = (float)x;
  lo = (float)(x - (double)hi);
#endif
}

__host__ __device__ inline dfloat::operator double() const {
#ifdef __CUDA_ARCH__
  return join_double(hi, lo);
#else
  return (double)hi + (double)lo;
#endif
}

}  // namespace pmg
