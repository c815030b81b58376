// pbat_num.cuh -- number formats used by the PBAT engine.
//
// * u128: unsigned 128-bit fixed point.  Every per-state probability sum on
//   the device is an exact integer sum of table entries scaled by 2^127, so
//   the enumeration order never changes a result and the T1 - T0 gradient
//   terms cancel exactly where they should.
// * dd: double-double (unevaluated sum hi + lo, ~106-bit significand) built
//   from the error-free transformations TwoSum (Knuth, TAOCP vol. 2) and
//   TwoProduct via fused multiply-add (Dekker 1971 / Ogita-Rump-Oishi 2005).
//   It carries per-work-item masses and the final reductions.
#pragma once
#include <stdint.h>
#include <math.h>

#ifdef __CUDACC__
#define PBAT_HD __host__ __device__ __forceinline__
#else
#define PBAT_HD inline
#endif

struct dd {
  double hi, lo;
};

PBAT_HD dd dd_make(double h) { return dd{h, 0.0}; }

PBAT_HD dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return dd{s, e};
}

PBAT_HD dd fast_two_sum(double a, double b) {  // requires |a| >= |b| or a == 0
  double s = a + b;
  double e = b - (s - a);
  return dd{s, e};
}

PBAT_HD dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  return dd{p, e};
}

PBAT_HD dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}

PBAT_HD dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }

PBAT_HD dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

PBAT_HD dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return fast_two_sum(p.hi, p.lo);
}

PBAT_HD dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return fast_two_sum(p.hi, p.lo);
}

// exact power-of-two scaling
PBAT_HD dd dd_ldexp(dd a, int e) { return dd{ldexp(a.hi, e), ldexp(a.lo, e)}; }

// 1 - p exactly (p in [0, 1] is a double, so 1 - p fits a double-double)
PBAT_HD dd dd_one_minus(double p) { return two_sum(1.0, -p); }

struct u128 {
  uint64_t lo, hi;
};

PBAT_HD u128 u128_zero() { return u128{0, 0}; }

#ifdef __CUDA_ARCH__
__device__ __forceinline__ void u128_add_to(u128& a, const u128 b) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;"
      : "+l"(a.lo), "+l"(a.hi)
      : "l"(b.lo), "l"(b.hi));
}
__device__ __forceinline__ u128 u128_sub(const u128 a, const u128 b) {
  u128 r;
  asm("sub.cc.u64 %0, %2, %4;\n\tsubc.u64 %1, %3, %5;"
      : "=l"(r.lo), "=l"(r.hi)
      : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
  return r;
}
#else
inline void u128_add_to(u128& a, const u128 b) {
  uint64_t lo = a.lo + b.lo;
  a.hi += b.hi + (lo < a.lo ? 1u : 0u);
  a.lo = lo;
}
inline u128 u128_sub(const u128 a, const u128 b) {
  u128 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1u : 0u);
  return r;
}
#endif

// Value of a u128 as a double-double (relative error below 2^-100).
PBAT_HD dd u128_to_dd(const u128 v) {
  // v = hi * 2^64 + lo.  Split hi into a rounded-down double and an exact
  // remainder < 2^11, so that every piece converts with a known error.
#ifdef __CUDA_ARCH__
  double h = __ull2double_rd(v.hi);
#else
  double h = (double)v.hi;
  if (h >= 18446744073709551616.0) h = nextafter(h, 0.0);
  while ((uint64_t)h > v.hi) h = nextafter(h, 0.0);
#endif
  uint64_t hr = v.hi - (uint64_t)h;  // < 2^11
  double top = ldexp(h, 64);
  double mid = ldexp((double)hr, 64);  // exact: hr < 2^11
  // lo needs 64 bits: split into two 32-bit halves, each exact in a double
  double l1 = ldexp((double)(v.lo >> 32), 32);
  double l0 = (double)(v.lo & 0xffffffffu);
  dd r = two_sum(top, mid);
  r = dd_add(r, two_sum(l1, l0));
  return r;
}
