// pbat_engine.h -- host-side types of the PBAT engine.
#pragma once
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include <math.h>

#include "pbat.h"
#include "pbat_num.cuh"

namespace pbat {

struct GraphIn {
  int n, m;
  const int32_t* tail;
  const int32_t* head;
  int directed, source, sink;
};

struct DeviceInfo {
  int device = -1;
  int sms = 0;
  int smem_optin = 0;
  int cc_major = 0, cc_minor = 0;
};

// How one network's 2^m states are split (equal division, Sec. 4.3):
//   ell lane arcs (one pattern per warp lane), L walk arcs (Gray walk per
//   thread), d prefix arcs (one work item per prefix value).
struct Plan {
  bool grad = false;
  bool wide = false;      // n > 32: 64-bit node masks
  int ell = 0, L = 0, d = 0;
  int range_bits = 0;
  int prune = 1;
  int nthr = 128;
  size_t smem = 0;
  unsigned long long task_lo = 0, n_tasks = 0;
  std::vector<int> perm;  // internal arc position -> input arc index
};

// Device + pinned host scratch, pooled across calls (one user at a time).
struct Scratch {
  int device = -1;
  bool busy = false;
  void* dmem = nullptr;
  size_t dbytes = 0;
  void* hmem = nullptr;
  size_t hbytes = 0;
};
int scratch_acquire(int device, size_t dbytes, size_t hbytes, Scratch** out);
void scratch_release(Scratch* s);

int run_single(const GraphIn& g, const double* p, bool grad, pbat_options* opt, void* stream,
               double* R_out, uint64_t* Nk_out, double* dRdp_out);

int fail(int code, const char* fmt, ...);
void clear_error();
bool fault_at(const char* site);   // PBAT_FAULT host-side fault injection
const char* last_error();
int validate_graph(const GraphIn& g);
int validate_p(const double* p, int m);
int validate_options(const pbat_options* o, int m);
int device_info(DeviceInfo& out);

// ---- host numeric helpers (fixed point, double-double) ----
typedef unsigned __int128 uint128_host;

// x = M * 2^ex2 with an integer M < 2^53, read from the bits of a finite x > 0
inline void double_parts(double x, uint64_t& M, int& ex2) {
  uint64_t bits;
  memcpy(&bits, &x, sizeof bits);
  const int bexp = (int)((bits >> 52) & 0x7ff);
  M = bits & ((1ull << 52) - 1);
  if (bexp) {
    M |= 1ull << 52;
    ex2 = bexp - 1075;
  } else {
    ex2 = -1074;
  }
}

// round(x * 2^e) for a finite double x >= 0 whose result is below 2^128
inline uint128_host scaled_round_u(double x, int e) {
  if (!(x > 0.0)) return 0;
  uint64_t M;
  int ex2;
  double_parts(x, M, ex2);
  const int sh = ex2 + e;
  if (sh >= 0) return (uint128_host)M << sh;
  if (-sh >= 64) return 0;   // below one half (M < 2^53)
  const uint64_t half = (uint64_t)1 << (-sh - 1);
  return (uint128_host)((M + half) >> (-sh));
}

// round((v.hi + v.lo) * 2^127) for v in [0, 1]
inline u128 to_fixed127(dd v) {
  uint128_host r = scaled_round_u(v.hi, 127);
  if (v.lo > 0)
    r += scaled_round_u(v.lo, 127);
  else if (v.lo < 0)
    r -= scaled_round_u(-v.lo, 127);
  return u128{(uint64_t)r, (uint64_t)(r >> 64)};
}

// Products of arc reliabilities in the kernels' integer floating point:
// value m * 2^(-63 - e) with m in [2^63, 2^64) (or m = 0) and e >= 0, m
// rounded from the double-double.
struct MxHost {
  uint64_t m;
  int32_t e, pad;
};
inline MxHost to_mx(dd v) {
  MxHost out{0, 0, 0};
  if (!(v.hi > 0.0)) return out;
  uint64_t M;
  int ex2;
  double_parts(v.hi, M, ex2);
  const int k = ex2 + 64 - __builtin_clzll(M);   // v.hi in [2^(k-1), 2^k)
  int e = 1 - k;
  uint128_host r = scaled_round_u(v.hi, 64 - k);
  if (v.lo > 0)
    r += scaled_round_u(v.lo, 64 - k);
  else if (v.lo < 0)
    r -= scaled_round_u(-v.lo, 64 - k);
  if (r >> 64) {
    r >>= 1;
    --e;
  } else if (!(r >> 63)) {
    r <<= 1;
    ++e;
  }
  if (e < 0) {  // a rounded product of reliabilities never exceeds 1
    r = (uint128_host)1 << 63;
    e = 0;
  }
  out.m = (uint64_t)r;
  out.e = e;
  return out;
}

// A non-negative 256-bit fixed-point number at scale 2^250, held as 32-bit
// chunks in eight 64-bit limbs whose upper halves carry, as a double-double.
inline dd limbs256_to_dd(const unsigned long long* limbs) {
  uint32_t chunk[10];
  uint128_host carry = 0;
  for (int i = 0; i < 8; ++i) {
    const uint128_host v = (uint128_host)limbs[i] + carry;
    chunk[i] = (uint32_t)(v & 0xffffffffu);
    carry = v >> 32;
  }
  chunk[8] = (uint32_t)(carry & 0xffffffffu);
  chunk[9] = (uint32_t)(carry >> 32);
  dd s = dd{0.0, 0.0};
  for (int i = 9; i >= 0; --i) s = dd_add(s, dd_make(ldexp((double)chunk[i], 32 * i - 250)));
  return s;
}

inline dd dd_recip(double x) {
  // Newton step on 1/x in double-double: y1 = y0 + y0 * (1 - x y0)
  const double y0 = 1.0 / x;
  const dd xy = two_prod(x, y0);
  const dd e = dd_sub(dd_make(1.0), xy);
  return dd_add(dd_make(y0), dd_mul_d(e, y0));
}

inline dd dd_recip_dd(dd x) {
  const double y0 = 1.0 / x.hi;
  const dd e = dd_sub(dd_make(1.0), dd_mul_d(x, y0));
  return dd_add(dd_make(y0), dd_mul_d(e, y0));
}

inline uint64_t binom_u64(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint128_host r = 1;
  for (int i = 1; i <= k; ++i) r = r * (uint128_host)(n - k + i) / (uint128_host)i;
  return (uint64_t)r;
}


inline dd arc_w(const double* p, int arc, int bit) {
  return bit ? dd_make(p[arc]) : dd_one_minus(p[arc]);
}

// out[v], v < 2^n: the double-double product over the n arcs arcs[x] of
// p (bit x of v set) or 1 - p (clear) -- every pattern's mass (Eq. 1
// restricted to those arcs).
inline void product_table(const double* p, const int* arcs, int n, dd* out) {
  out[0] = dd_make(1.0);
  for (int x = 0; x < n; ++x) {
    const dd w0 = arc_w(p, arcs[x], 0), w1 = arc_w(p, arcs[x], 1);
    for (int v = (1 << x) - 1; v >= 0; --v) {
      out[v + (1 << x)] = dd_mul(out[v], w1);
      out[v] = dd_mul(out[v], w0);
    }
  }
}

// Byte tables of subset sums: for each byte b of a 32-entry weight vector
// w (entries past n_valid are zero), out[(b * 256 + v) * stride] is the sum
// of w[8 b + i] over the set bits i of v, at scale 2^62.  The weights are
// rounded once to 2^-126, summed exactly in 128 bits, and the sum rounded
// once to 2^-62.
inline void byte_table_sums(const dd* w, int n_valid, unsigned long long* out, int stride) {
  uint128_host fw[32];
  for (int j = 0; j < 32; ++j) {
    if (j >= n_valid) {
      fw[j] = 0;
      continue;
    }
    fw[j] = scaled_round_u(w[j].hi, 126);
    if (w[j].lo > 0)
      fw[j] += scaled_round_u(w[j].lo, 126);
    else if (w[j].lo < 0)
      fw[j] -= scaled_round_u(-w[j].lo, 126);
  }
  const uint128_host half = (uint128_host)1 << 63;
  for (int b = 0; b < 4; ++b) {
    uint128_host sb[256];
    sb[0] = 0;
    out[(size_t)(b * 256) * stride] = 0;
    for (int v = 1; v < 256; ++v) {
      sb[v] = sb[v & (v - 1)] + fw[8 * b + __builtin_ctz((unsigned)v)];
      out[(size_t)(b * 256 + v) * stride] = (unsigned long long)((sb[v] + half) >> 64);
    }
  }
}

inline unsigned long long fixed_u64(dd v, int scale) {
  // round((hi + lo) * 2^scale) for 0 <= v, result < 2^64
  uint128_host r = scaled_round_u(v.hi, scale);
  if (v.lo > 0)
    r += scaled_round_u(v.lo, scale);
  else if (v.lo < 0)
    r -= scaled_round_u(-v.lo, scale);
  return (unsigned long long)r;
}

}  // namespace pbat
