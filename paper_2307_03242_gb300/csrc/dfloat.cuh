// Double-FP32 ("float-float") arithmetic for the FP64 outer solve on a part whose FP64 pipe is
// ~57x slower than its FP32 pipe. A value is hi + lo with two floats; products use Dekker's
// error-free product via FMA (p = a*b, e = fma(a, b, -p)), sums use Knuth's TwoSum. IEEE doubles
// (the caller's vectors) are split into hi + lo with integer and FP32 operations only (hi = the
// double truncated to 24 significant bits, lo = the next 23 mantissa bits), so the representation
// error is below 2^-46 relative, and assembled back the same way (join); the outer solve's
// internal vectors are stored as float-float pairs (cff). Values whose magnitude lies outside the
// normal float range (about 1e-38 .. 3e38) lose the lo part or overflow; the outer solve keeps
// its vectors near unit norm, far inside that range.
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

// Leading-zero count of a nonzero 32-bit word.
HD int clz32(unsigned v) {
#ifdef __CUDA_ARCH__
  return __clz((int)v);
#else
  return __builtin_clz(v);
#endif
}

// Bits of a float widened to a double, assembled with integer operations only (no FP64
// instruction, no conversion): normal floats move their exponent and mantissa, subnormal ones are
// normalised with a leading-zero count, infinities and NaNs keep their class and payload.
HD unsigned long long widen_bits(float f) {
  const unsigned u = fbits(f);
  const unsigned ex = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  if (ex == 0) {
    if (m == 0) return sgn;
    const int p = 31 - clz32(m);  // leading bit of the subnormal mantissa: the value is 1.f 2^(p-149)
    return sgn | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
  }
  const unsigned long long dex = ex == 255 ? 0x7ffull : (unsigned long long)(ex + 896);
  return sgn | (dex << 52) | ((unsigned long long)m << 29);
}
HD double widen(float f) { return bdouble(widen_bits(f)); }

// Knuth TwoSum: s + e == a + b exactly.
HD void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// hi + lo as a double with FP32 and integer operations only. The pair is first normalised with
// TwoSum (exact: s + e = hi + lo, |e| <= ulp(s)/2). e is then added to the bits of s widened:
// in units of the double ulp of s, 2^(E_s - 52), e is its 24-bit integer mantissa shifted by
// E_e - E_s + 29 <= 5 (one more when s is a power of two and e has the opposite sign, whose sum
// lies in the binade below, where the unit is half as large). Adding or subtracting that integer
// to the bit pattern is exact for the bits that fit in 53; the bits of e below the double's
// last place are truncated (an error below one ulp of the result).
HD double join(float hi, float lo) {
  float s, e;
  two_sum(hi, lo, s, e);
  const unsigned long long d = widen_bits(s);
  const unsigned us = fbits(s), ue = fbits(e);
  const int es = (int)((us >> 23) & 0xffu), ee = (int)((ue >> 23) & 0xffu);
  const unsigned me = (ue & 0x7fffffu) | (ee != 0 ? 0x800000u : 0u);
  if (es == 0 || es == 255 || me == 0) return bdouble(d);  // zero, subnormal (e is 0), non-finite
  const bool opp = ((us ^ ue) >> 31) != 0;
  int sh = (ee != 0 ? ee : 1) - es + 29;
  if (opp && (us & 0x7fffffu) == 0) sh += 1;
  const unsigned long long off =
      sh >= 0 ? ((unsigned long long)me << sh) : (sh > -32 ? (unsigned long long)(me >> -sh) : 0ull);
  return bdouble(opp ? d - off : d + off);
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
  // += a (a float)
  HD void add(float a) {
    float s, t;
    two_sum(hi, a, s, t);
    hi = s;
    lo += t;
  }
  HD double to_double() const { return join(hi, lo); }
  HD f2 norm() const {
    f2 r;
    two_sum(hi, lo, r.hi, r.lo);
    return r;
  }
};


// x as a float when it is a power of two inside the normal float range, else 0 (integer
// operations on the bits of x).
HD float pow2_float(double x) {
  const unsigned long long b = dbits(x);
  if (b & 0xfffffffffffffull) return 0.0f;
  const int e = (int)((b >> 52) & 0x7ffu) - 1023;
  if (e < -126 || e > 127) return 0.0f;
  return bfloat((unsigned)(b >> 32 & 0x80000000u) | ((unsigned)(e + 127) << 23));
}

// bscale * b - r. With bs = pow2_float(bscale) != 0 it is evaluated in float-float (the scaling
// of the split b by a power of two is exact); otherwise in FP64.
HD acc scaled_sub_acc(double b, float bs, double bscale, const acc& r) {
  acc t;
  if (bs == 0.0f) {
    t.add(split(bscale * b - r.to_double()));
    return t;
  }
  const f2 bb = split(b);
  t.hi = bb.hi * bs;
  t.lo = bb.lo * bs;
  const f2 rn = r.norm();
  t.add({-rn.hi, -rn.lo});
  return t;
}
HD double scaled_sub(double b, float bs, double bscale, const acc& r) {
  return scaled_sub_acc(b, bs, bscale, r).to_double();
}

// A complex float-float value in memory: the normalised hi and lo floats of the real part, then
// of the imaginary part (16 bytes, the size of a complex double). The outer solve keeps its
// internal Krylov vectors in this form, so that its vector kernels neither split nor assemble
// doubles; the caller's vectors (b, x, an applied y) stay IEEE FP64.
struct __align__(16) cff {
  float rh, rl, ih, il;
};
HD cff to_cff(const acc& re, const acc& im) {
  const f2 a = re.norm(), b = im.norm();
  return {a.hi, a.lo, b.hi, b.lo};
}
HD cff to_cff(double re, double im) {
  const f2 a = split(re), b = split(im);
  return {a.hi, a.lo, b.hi, b.lo};
}

}  // namespace df
