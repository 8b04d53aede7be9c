// Double-FP32 ("float-float") arithmetic for the FP64 outer solve on a part whose FP64 pipe is
// ~57x slower than its FP32 pipe. A value is hi + lo with two floats; products use Dekker's
// error-free product via FMA (p = a*b, e = fma(a, b, -p)), sums use Knuth's TwoSum. Vectors stay
// IEEE FP64 in memory: a double is split EXACTLY into hi + lo with integer operations only
// (hi = the double truncated to 24 significant bits, lo = the remaining mantissa bits, rounded to
// 24 bits), so the representation error is below 2^-47 relative. Values whose magnitude lies
// outside the normal float range (about 1e-38 .. 3e38) lose the lo part or overflow; the outer
// solve keeps its vectors near unit norm, far inside that range.
#pragma once
#include <cmath>
#include <cstring>

#include "emg_types.cuh"

namespace df {

struct f2 {
  float hi, lo;
};

// Bit access (device intrinsics, memcpy on the host).
HD unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}
HD double bdouble(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}
HD unsigned fbits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}
HD float bfloat(unsigned b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}

// Split of a double into hi + lo with integer and FP32 operations only (none on the FP64 pipe,
// which on this part is ~57x slower): hi = the double truncated to 24 significant bits (the sign,
// the rebiased exponent and the top 23 mantissa bits), lo = the next 23 mantissa bits, built as
// ((1 + m 2^-23) - 1) 2^(e-1046), exact. The bits below (6 of 52) are dropped: hi + lo differs
// from x by less than 2^-46 |x|. Magnitudes outside the normal float range (about 1e-38 .. 3e38)
// give hi = 0 (tiny) or an infinity (huge; NaN stays NaN); lo is dropped below about 1e-31.
HD f2 split(double x) {
  const unsigned long long b = dbits(x);
  const unsigned hib = (unsigned)(b >> 32), lob = (unsigned)b;
  const unsigned sgn = hib & 0x80000000u;
  const int e = (int)((hib >> 20) & 0x7ffu);  // biased exponent of x
  f2 r;
  if (e >= 897 && e <= 1150) {
    r.hi = bfloat(sgn | ((unsigned)(e - 896) << 23) | ((hib & 0xfffffu) << 3) | (lob >> 29));
    float lo = 0.0f;
    if (e >= 920) {
      const float f = bfloat(0x3f800000u | ((lob & 0x1fffffffu) >> 6)) - 1.0f;  // (top 23 of the 29 low bits) 2^-23
      lo = f * bfloat((unsigned)(e - 919) << 23);                               // times 2^(e-1046)
    }
    r.lo = sgn ? -lo : lo;
  } else if (e < 897) {
    r.hi = bfloat(sgn);
    r.lo = 0.0f;
  } else {
    const bool nan = e == 2047 && ((hib & 0xfffffu) | lob) != 0;
    r.hi = bfloat(nan ? 0x7fc00000u : (sgn | 0x7f800000u));
    r.lo = 0.0f;
  }
  return r;
}

// A float widened to a double by assembling its bits (no FP64 instruction); subnormal floats
// take the plain conversion.
HD double widen(float f) {
  const unsigned u = fbits(f);
  const unsigned ex = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  if (ex == 0) return m == 0 ? bdouble(sgn) : (double)f;
  const unsigned long long dex = ex == 255 ? 0x7ffull : (unsigned long long)(ex + 896);
  return bdouble(sgn | (dex << 52) | ((unsigned long long)m << 29));
}

// hi + lo as a double: two assembled widenings and one FP64 addition (instead of two conversions
// and an addition on the FP64 pipe).
HD double join(float hi, float lo) { return widen(hi) + widen(lo); }

// Knuth TwoSum: s + e == a + b exactly.
HD void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Accumulator: hi + lo (lo unnormalised).
struct acc {
  float hi = 0.f, lo = 0.f;
  // += a * b (a, b float-float)
  HD void fma_ff(f2 a, f2 b) {
    float p = a.hi * b.hi;
    float e = std::fma(a.hi, b.hi, -p);
    e = std::fma(a.hi, b.lo, e);
    e = std::fma(a.lo, b.hi, e);
    float s, t;
    two_sum(hi, p, s, t);
    hi = s;
    lo += t + e;
  }
  // -= a * b
  HD void fms_ff(f2 a, f2 b) {
    f2 na = {-a.hi, -a.lo};
    fma_ff(na, b);
  }
  HD void add(f2 a) {
    float s, t;
    two_sum(hi, a.hi, s, t);
    hi = s;
    lo += t + a.lo;
  }
  HD double to_double() const { return join(hi, lo); }
  HD f2 norm() const {
    f2 r;
    two_sum(hi, lo, r.hi, r.lo);
    return r;
  }
};

}  // namespace df
