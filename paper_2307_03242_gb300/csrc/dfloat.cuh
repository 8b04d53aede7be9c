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

// Exact split of a double into hi (24 significant bits, truncated) + lo (low 29 mantissa bits,
// rounded to 24). Integer operations and one int->float conversion; no FP64 arithmetic.
HD f2 split(double x) {
  f2 r;
#ifdef __CUDA_ARCH__
  r.hi = __double2float_rz(x);
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
#else
  r.hi = (float)x;
  if (std::fabs((double)r.hi) > std::fabs(x)) r.hi = std::nextafter(r.hi, 0.0f);
  unsigned long long b;
  std::memcpy(&b, &x, sizeof b);
#endif
  const unsigned int hib = (unsigned int)(b >> 32);
  const unsigned int lob = (unsigned int)b & 0x1fffffffu;
  const int e = (int)((hib >> 20) & 0x7ffu);  // biased exponent of x
  // lo = lob * 2^(e-1075) = (lob * 2^-52) * 2^(e-1023); the second factor is a normal float for
  // e >= 897, i.e. whenever hi is a normal float; below that lo is dropped.
#ifdef __CUDA_ARCH__
  float sc = (e >= 897 && e <= 1150) ? __int_as_float((e - 896) << 23) : 0.0f;
  float lo = __uint2float_rn(lob) * 0x1p-52f * sc;
#else
  float sc = 0.0f;
  if (e >= 897 && e <= 1150) {
    const int bits = (e - 896) << 23;
    std::memcpy(&sc, &bits, sizeof sc);
  }
  float lo = (float)lob * 0x1p-52f * sc;
#endif
  r.lo = (hib & 0x80000000u) ? -lo : lo;
  return r;
}

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
  HD double to_double() const { return (double)hi + (double)lo; }
  HD f2 norm() const {
    f2 r;
    two_sum(hi, lo, r.hi, r.lo);
    return r;
  }
};

}  // namespace df
