/*
 * pbat_oracle.c -- plain CPU oracle for exact two-terminal reliability by
 * full enumeration of arc states (arXiv 2209.09711, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test-suite, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header or table with
 * the CUDA engine.
 *
 * What it computes, written out as plainly as possible:
 *
 *   * State order (Sec. 3.1 Rules 1-2, Table 2; Sec. 4.2 Eq. 2-3): the state
 *     with index x in [0, 2^m) has arc a_k (1-based) working iff bit (m-k) of
 *     x is set, i.e. x_1 is the most significant coordinate and the backward
 *     BAT visits x = 0, 1, ..., 2^m - 1 in order.
 *   * Pr(X) = prod_k (x_k ? p_k : 1 - p_k)  (Eq. 1; Table 4's printed values
 *     fix the product reading of the garbled Sec. 2.2 notation).
 *   * Connectivity: PLSA (Sec. 3.2, STEP P0-P4).  Layer L_1 = {source};
 *     L_l = nodes not seen before with a working arc from a node of L_{l-1};
 *     an empty layer means "disconnected", a layer holding the sink means
 *     "connected".  (The paper's layer rule does not exclude visited nodes;
 *     excluding them is needed for STEP P2 to ever fire and does not change
 *     which nodes are reachable.)  Undirected arcs work both ways.
 *   * R = sum over connected X of Pr(X)  (Eq. 1), N_k = number of connected X
 *     with k working arcs (the reliability-polynomial coefficients).
 *   * Gradient, two independent ways:
 *       T1_i - T0_i where T1_i (T0_i) sums prod_{j != i} over connected X with
 *       x_i = 1 (x_i = 0): the derivative of Eq. 1 term by term;
 *       the critical-state sum: over X with x_i = 1, X connected and
 *       X - e_i disconnected, add prod_{j != i}.  R is affine in each p_i, so
 *       dR/dp_i = R(p_i = 1) - R(p_i = 0) equals both.
 *
 * Sums are long double with Neumaier (compensated) summation, so the
 * oracle's own rounding stays far below the 1e-12 parity tolerance even for
 * 2^27 terms.  Values cross the ABI as (hi, lo) double pairs.
 *
 * Parity pins: see tests/test_oracle_pins.py (closed forms, the paper's
 * worked example, invariants of N_k, brute force with an independent
 * union-find connectivity).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 64
#define ORC_MAXM 63

typedef struct {
  long double s, c; /* Neumaier running sum and compensation */
} orc_sum;

static void orc_add(orc_sum* a, long double x) {
  long double t = a->s + x;
  if ((a->s >= 0 ? a->s : -a->s) >= (x >= 0 ? x : -x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}

static long double orc_val(const orc_sum* a) { return a->s + a->c; }

static void orc_split(long double v, double* hi, double* lo) {
  double h = (double)v;
  *hi = h;
  *lo = (double)(v - (long double)h);
}

/* Is arc k (0-based) working in state index x of an m-arc network? */
static int orc_arc_on(uint64_t x, int m, int k) { return (int)((x >> (m - 1 - k)) & 1u); }

/*
 * PLSA (Sec. 3.2).  Returns 1 if sink is reached from source in G(X).
 * If layer_of is non-null, layer_of[v] receives the 1-based layer of every
 * node placed in a layer (0 for nodes never placed).
 */
static int orc_plsa(int n, int m, const int* tail, const int* head, int directed, int source,
                    int sink, uint64_t x, int* layer_of) {
  int seen[ORC_MAXN];
  int cur[ORC_MAXN], nxt[ORC_MAXN];
  int ncur = 0, nnxt, l, k, i;
  for (i = 0; i < n; ++i) seen[i] = 0;
  if (layer_of)
    for (i = 0; i < n; ++i) layer_of[i] = 0;
  /* STEP P0: l = 2, L_1 = {source} */
  cur[ncur++] = source;
  seen[source] = 1;
  if (layer_of) layer_of[source] = 1;
  for (l = 2;; ++l) {
    /* STEP P1: L_l = unseen v with a working arc u -> v, u in L_{l-1} */
    int inprev[ORC_MAXN];
    for (i = 0; i < n; ++i) inprev[i] = 0;
    for (i = 0; i < ncur; ++i) inprev[cur[i]] = 1;
    nnxt = 0;
    for (k = 0; k < m; ++k) {
      int u = tail[k], v = head[k];
      if (!orc_arc_on(x, m, k)) continue;
      if (inprev[u] && !seen[v]) {
        seen[v] = 1;
        nxt[nnxt++] = v;
      }
      if (!directed && inprev[v] && !seen[u]) {
        seen[u] = 1;
        nxt[nnxt++] = u;
      }
    }
    if (layer_of)
      for (i = 0; i < nnxt; ++i) layer_of[nxt[i]] = l;
    /* STEP P2: empty layer -> disconnected */
    if (nnxt == 0) return 0;
    /* STEP P3: sink in L_l -> connected */
    if (seen[sink]) return 1;
    /* STEP P4 */
    for (i = 0; i < nnxt; ++i) cur[i] = nxt[i];
    ncur = nnxt;
  }
}

static long double orc_pr(int m, const double* p, uint64_t x, int skip) {
  long double w = 1.0L;
  int k;
  for (k = 0; k < m; ++k) {
    if (k == skip) continue;
    w *= orc_arc_on(x, m, k) ? (long double)p[k] : 1.0L - (long double)p[k];
  }
  return w;
}

static int orc_check(int n, int m, const int* tail, const int* head, int source, int sink) {
  int k;
  if (n < 2 || n > ORC_MAXN || m < 0 || m > ORC_MAXM) return -1;
  if (source < 0 || source >= n || sink < 0 || sink >= n || source == sink) return -1;
  for (k = 0; k < m; ++k)
    if (tail[k] < 0 || tail[k] >= n || head[k] < 0 || head[k] >= n || tail[k] == head[k]) return -1;
  return 0;
}

/* Connectivity of one state; -1 on bad input. */
int orc_connected(int n, int m, const int* tail, const int* head, int directed, int source,
                  int sink, uint64_t x) {
  if (orc_check(n, m, tail, head, source, sink)) return -1;
  return orc_plsa(n, m, tail, head, directed, source, sink, x, NULL);
}

/* PLSA layers of one state (Table 3); returns connectivity, -1 on bad input. */
int orc_plsa_layers(int n, int m, const int* tail, const int* head, int directed, int source,
                    int sink, uint64_t x, int* layer_of) {
  if (orc_check(n, m, tail, head, source, sink)) return -1;
  return orc_plsa(n, m, tail, head, directed, source, sink, x, layer_of);
}

/* Pr(X) of one state as (hi, lo). */
void orc_state_probability(int m, const double* p, uint64_t x, double* hi, double* lo) {
  orc_split(orc_pr(m, p, x, -1), hi, lo);
}

/*
 * Enumerate the states whose top `prefix_bits` coordinates, read as an
 * integer, lie in [prefix_lo, prefix_hi) -- the equal divisions of Sec. 4.3
 * (Eq. 6) with chi = 2^prefix_bits; prefix_bits = 0 with [0, 1) is the whole
 * space.  Outputs (any may be NULL):
 *   R_hi/R_lo         sum of Pr(X) over connected X
 *   Nk[m+1]           counts of connected X by number of working arcs
 *   T1_hi/lo[m], T0_hi/lo[m]  sums of prod_{j != i} over connected X with
 *                     x_i = 1 / x_i = 0
 * Returns 0, or -1 on bad input.
 */
int orc_enumerate(int n, int m, const int* tail, const int* head, int directed, const double* p,
                  int source, int sink, int prefix_bits, uint64_t prefix_lo, uint64_t prefix_hi,
                  double* R_hi, double* R_lo, uint64_t* Nk, double* T1_hi, double* T1_lo,
                  double* T0_hi, double* T0_lo) {
  orc_sum R = {0, 0};
  orc_sum T1[ORC_MAXM], T0[ORC_MAXM];
  int want_grad = (T1_hi || T0_hi);
  uint64_t x, x0, x1;
  int k, i;
  if (orc_check(n, m, tail, head, source, sink)) return -1;
  if (prefix_bits < 0 || prefix_bits > m) return -1;
  if (prefix_hi > ((uint64_t)1 << prefix_bits) || prefix_lo > prefix_hi) return -1;
  for (k = 0; k < m; ++k) {
    if (!(p[k] >= 0.0 && p[k] <= 1.0)) return -1;
    T1[k].s = T1[k].c = T0[k].s = T0[k].c = 0;
  }
  if (Nk)
    for (k = 0; k <= m; ++k) Nk[k] = 0;
  x0 = prefix_lo << (m - prefix_bits);
  x1 = prefix_hi << (m - prefix_bits);
  for (x = x0; x < x1; ++x) {
    if (!orc_plsa(n, m, tail, head, directed, source, sink, x, NULL)) continue;
    orc_add(&R, orc_pr(m, p, x, -1));
    if (Nk) {
      int c = 0;
      for (k = 0; k < m; ++k) c += orc_arc_on(x, m, k);
      Nk[c] += 1;
    }
    if (want_grad) {
      for (i = 0; i < m; ++i) {
        long double w = orc_pr(m, p, x, i);
        if (orc_arc_on(x, m, i))
          orc_add(&T1[i], w);
        else
          orc_add(&T0[i], w);
      }
    }
  }
  if (R_hi) orc_split(orc_val(&R), R_hi, R_lo);
  for (i = 0; i < m; ++i) {
    if (T1_hi) orc_split(orc_val(&T1[i]), &T1_hi[i], &T1_lo[i]);
    if (T0_hi) orc_split(orc_val(&T0[i]), &T0_hi[i], &T0_lo[i]);
  }
  return 0;
}

/*
 * dR/dp_i by the critical-state sum over the whole space: for every
 * connected X and every working arc i, if X - e_i is disconnected, add
 * prod_{j != i} of X's factors.  Every term is non-negative, so there is no
 * cancellation.  Returns 0, or -1 on bad input.
 */
int orc_grad_critical(int n, int m, const int* tail, const int* head, int directed,
                      const double* p, int source, int sink, double* G_hi, double* G_lo) {
  orc_sum G[ORC_MAXM];
  uint64_t x, nstates;
  int i;
  if (orc_check(n, m, tail, head, source, sink)) return -1;
  for (i = 0; i < m; ++i) {
    if (!(p[i] >= 0.0 && p[i] <= 1.0)) return -1;
    G[i].s = G[i].c = 0;
  }
  nstates = (uint64_t)1 << m;
  for (x = 0; x < nstates; ++x) {
    if (!orc_plsa(n, m, tail, head, directed, source, sink, x, NULL)) continue;
    for (i = 0; i < m; ++i) {
      uint64_t bit;
      if (!orc_arc_on(x, m, i)) continue;
      bit = (uint64_t)1 << (m - 1 - i);
      if (orc_plsa(n, m, tail, head, directed, source, sink, x & ~bit, NULL)) continue;
      orc_add(&G[i], orc_pr(m, p, x, i));
    }
  }
  for (i = 0; i < m; ++i) orc_split(orc_val(&G[i]), &G_hi[i], &G_lo[i]);
  return 0;
}

/* Size of long double in bits of mantissa, for reporting. */
int orc_long_double_mant_bits(void) {
  long double e = 1.0L;
  int b = 0;
  while ((long double)1.0L + e != 1.0L) {
    e /= 2;
    ++b;
  }
  return b;
}
