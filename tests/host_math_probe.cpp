// Test probe for the engine's host arithmetic (pbat_engine.h): reads one
// request per line on stdin, writes one answer per line on stdout.  Doubles
// and integers travel as hexadecimal bit patterns, so the test compares
// exact values.  Built by tests/test_host_math.py with the host C++ compiler.
//
//   S <x bits> <e>          scaled_round_u(x, e)         -> <hi64> <lo64>
//   F <hi bits> <lo bits>   to_fixed127({hi, lo})        -> <hi64> <lo64>
//   M <hi bits> <lo bits>   to_mx({hi, lo})              -> <m> <e>
//   L <l0> ... <l7>         limbs256_to_dd(limbs)        -> <hi bits> <lo bits>
//   B <n> <k>               binom_u64(n, k)              -> <value>
//   R <x bits>              dd_recip(x)                  -> <hi bits> <lo bits>
//   P <n> <p bits> x n      product_table over arcs 0..n-1 -> 2^n lines <hi bits> <lo bits>
//   T <n> <hi lo bits> x n  byte_table_sums(w, n, out, 1)  -> 1024 lines <value>
//   X <hi bits> <lo bits> <scale>  fixed_u64({hi, lo}, scale) -> <value>
#include <cstdio>
#include <cstring>

#include "pbat_engine.h"

using namespace pbat;

static double dbl(unsigned long long b) {
  double x;
  memcpy(&x, &b, sizeof x);
  return x;
}

static unsigned long long bits(double x) {
  unsigned long long b;
  memcpy(&b, &x, sizeof b);
  return b;
}

int main() {
  char op;
  while (scanf(" %c", &op) == 1) {
    if (op == 'S') {
      unsigned long long x;
      int e;
      if (scanf("%llx %d", &x, &e) != 2) return 1;
      const uint128_host r = scaled_round_u(dbl(x), e);
      printf("%llx %llx\n", (unsigned long long)(r >> 64), (unsigned long long)r);
    } else if (op == 'F') {
      unsigned long long h, l;
      if (scanf("%llx %llx", &h, &l) != 2) return 1;
      const u128 r = to_fixed127(dd{dbl(h), dbl(l)});
      printf("%llx %llx\n", (unsigned long long)r.hi, (unsigned long long)r.lo);
    } else if (op == 'M') {
      unsigned long long h, l;
      if (scanf("%llx %llx", &h, &l) != 2) return 1;
      const MxHost r = to_mx(dd{dbl(h), dbl(l)});
      printf("%llx %d\n", (unsigned long long)r.m, (int)r.e);
    } else if (op == 'L') {
      unsigned long long limbs[8];
      for (int i = 0; i < 8; ++i)
        if (scanf("%llx", &limbs[i]) != 1) return 1;
      const dd r = limbs256_to_dd(limbs);
      printf("%llx %llx\n", bits(r.hi), bits(r.lo));
    } else if (op == 'B') {
      int n, k;
      if (scanf("%d %d", &n, &k) != 2) return 1;
      printf("%llx\n", (unsigned long long)binom_u64(n, k));
    } else if (op == 'R') {
      unsigned long long x;
      if (scanf("%llx", &x) != 1) return 1;
      const dd r = dd_recip(dbl(x));
      printf("%llx %llx\n", bits(r.hi), bits(r.lo));
    } else if (op == 'P') {
      int n;
      if (scanf("%d", &n) != 1 || n < 0 || n > 10) return 1;
      double p[10];
      int arcs[10];
      for (int i = 0; i < n; ++i) {
        unsigned long long b;
        if (scanf("%llx", &b) != 1) return 1;
        p[i] = dbl(b);
        arcs[i] = i;
      }
      dd out[1 << 10];
      product_table(p, arcs, n, out);
      for (int v = 0; v < (1 << n); ++v) printf("%llx %llx\n", bits(out[v].hi), bits(out[v].lo));
    } else if (op == 'T') {
      int n;
      if (scanf("%d", &n) != 1 || n < 0 || n > 32) return 1;
      dd w[32];
      for (int i = 0; i < n; ++i) {
        unsigned long long h, l;
        if (scanf("%llx %llx", &h, &l) != 2) return 1;
        w[i] = dd{dbl(h), dbl(l)};
      }
      unsigned long long out[1024];
      byte_table_sums(w, n, out, 1);
      for (int i = 0; i < 1024; ++i) printf("%llx\n", out[i]);
    } else if (op == 'X') {
      unsigned long long h, l;
      int sc;
      if (scanf("%llx %llx %d", &h, &l, &sc) != 3) return 1;
      printf("%llx\n", fixed_u64(dd{dbl(h), dbl(l)}, sc));
    } else {
      return 2;
    }
  }
  return 0;
}
