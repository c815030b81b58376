/*
 * pbat_cpu.c -- the paper's parallel BAT (PBAT) on the host cores, in plain
 * C with POSIX threads.  This is the timed CPU baseline of the benchmark: the
 * method of arXiv 2209.09711 as the paper runs it, on a CPU, in FP64.  It is
 * not the oracle (that one is a single-threaded long-double brute force kept
 * for parity); it shares no code with the oracle or with the CUDA engine.
 *
 * What it runs (Sec. 5.1, PBAT STEP 0-3):
 *   STEP 0-1  chi threads; the state space is cut into equal divisions by its
 *             first d coordinates (Sec. 4.3, Eq. 6-7): division iota is every
 *             state X whose first d coordinates, read as a binary number,
 *             equal iota.  The caller passes the list of divisions to run
 *             (all 2^d of them for the whole space, or an evenly spread
 *             sample for timing); they are dealt to the threads in equal
 *             contiguous blocks, one block per thread.
 *   STEP 2    each thread walks its divisions in binary-addition order (the
 *             BAT of Sec. 3.1: the last zero coordinate becomes one and every
 *             coordinate after it zero -- binary counting on the free
 *             coordinates) and, for each state, runs the PLSA of Sec. 3.2:
 *             layer L_1 = {source}; layer L_l = the nodes not yet placed that
 *             a working arc joins to a node of L_{l-1}; an empty layer means
 *             disconnected, a layer holding the sink means connected.  Node
 *             sets are 64-bit masks.  A connected state adds Pr(X) (Eq. 1) to
 *             the thread's sum, kept in double with Kahan compensation, and
 *             counts toward N_k with k its number of working arcs.
 *   STEP 3    R = R_1 + ... + R_chi, the thread sums added in thread order
 *             (again with compensation).
 *
 * Pr(X) is the product over arcs of p_k (arc working) or 1 - p_k (failed),
 * formed as the product of per-byte tables of those factors (at most eight
 * table entries per state).  With want_grad the thread also sums, for every
 * arc i, prod_{j != i} of the state's factors into T1_i (x_i = 1) or T0_i
 * (x_i = 0), from prefix and suffix products; dR/dp_i = T1_i - T0_i is Eq. 1
 * differentiated term by term (the paper computes R only).
 *
 * Coordinates: arc a_k (k = 1..m) is bit m - k of the state index, so x_1 is
 * the most significant coordinate (Sec. 4.2, Table 2).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PCPU_MAXN 64
#define PCPU_MAXM 63

typedef struct {
  double s, c; /* Kahan running sum and compensation */
} pcpu_kahan;

static void pcpu_add(pcpu_kahan* a, double x) {
  double y = x - a->c;
  double t = a->s + y;
  a->c = (t - a->s) - y;
  a->s = t;
}

typedef struct {
  /* network */
  int n, m, directed, source, sink;
  int arc_u[PCPU_MAXM], arc_v[PCPU_MAXM]; /* arc by BIT position (bit b = arc a_{m-b}) */
  const double* p;                        /* input order */
  double pb[PCPU_MAXM], qb[PCPU_MAXM];    /* p and 1 - p by bit position */
  double bytetab[8][256];                 /* per byte of the state index: product of factors */
  int nbytes;
  /* work */
  int prefix_bits;
  const uint64_t* divs;
  int d0, d1; /* this thread's slice of divs */
  int want_grad;
  /* results of this thread */
  pcpu_kahan R;
  uint64_t Nk[PCPU_MAXM + 1];
  pcpu_kahan T1[PCPU_MAXM], T0[PCPU_MAXM];
} pcpu_job;

/* PLSA on the working arcs of state x (Sec. 3.2, STEP P0-P4). */
static int pcpu_plsa(const pcpu_job* J, uint64_t x) {
  uint64_t adj[PCPU_MAXN];
  int b;
  for (b = 0; b < J->n; ++b) adj[b] = 0;
  for (b = 0; b < J->m; ++b) {
    if (!((x >> b) & 1u)) continue;
    adj[J->arc_u[b]] |= (uint64_t)1 << J->arc_v[b];
    if (!J->directed) adj[J->arc_v[b]] |= (uint64_t)1 << J->arc_u[b];
  }
  {
    const uint64_t tbit = (uint64_t)1 << J->sink;
    uint64_t layer = (uint64_t)1 << J->source, seen = layer; /* STEP P0 */
    for (;;) {
      uint64_t next = 0, l = layer;
      while (l) { /* STEP P1 */
        const int u = __builtin_ctzll(l);
        l &= l - 1;
        next |= adj[u];
      }
      next &= ~seen;
      if (!next) return 0;         /* STEP P2 */
      if (next & tbit) return 1;   /* STEP P3 */
      seen |= next;                /* STEP P4 */
      layer = next;
    }
  }
}

static void* pcpu_thread(void* arg) {
  pcpu_job* J = (pcpu_job*)arg;
  const int m = J->m, free_bits = m - J->prefix_bits;
  const uint64_t per_div = (uint64_t)1 << free_bits;
  int i, di;
  for (di = J->d0; di < J->d1; ++di) {
    const uint64_t base = J->divs[di] << free_bits; /* STEP 2.2: the division's first state */
    uint64_t s;
    for (s = 0; s < per_div; ++s) { /* STEP 2.3-2.6: binary addition on the free coordinates */
      const uint64_t x = base | s;
      double w;
      if (!pcpu_plsa(J, x)) continue; /* STEP 2.5 */
      w = J->bytetab[0][x & 0xffu];
      for (i = 1; i < J->nbytes; ++i) w *= J->bytetab[i][(x >> (8 * i)) & 0xffu];
      pcpu_add(&J->R, w);
      J->Nk[__builtin_popcountll(x)] += 1;
      if (J->want_grad) {
        /* prod_{j != b} by prefix and suffix products over bit positions */
        double pre[PCPU_MAXM + 1], suf = 1.0;
        pre[0] = 1.0;
        for (i = 0; i < m; ++i) pre[i + 1] = pre[i] * (((x >> i) & 1u) ? J->pb[i] : J->qb[i]);
        for (i = m - 1; i >= 0; --i) {
          const double ex = pre[i] * suf;
          if ((x >> i) & 1u)
            pcpu_add(&J->T1[i], ex);
          else
            pcpu_add(&J->T0[i], ex);
          suf *= ((x >> i) & 1u) ? J->pb[i] : J->qb[i];
        }
      }
    }
  }
  return NULL;
}

/*
 * Run PBAT over the divisions divs[0 .. n_divs-1] (each an integer in
 * [0, 2^prefix_bits): the states whose first prefix_bits coordinates equal
 * it) on `threads` POSIX threads.  Outputs (Nk_out, dRdp_out nullable):
 *   R_out      sum of Pr(X) over the connected states of those divisions
 *   Nk_out     [m + 1] counts of connected states by working arcs
 *   dRdp_out   [m] (input arc order) T1_i - T0_i over those divisions
 * Returns 0, or -1 on bad input, -2 if a thread cannot be started.
 */
int pcpu_enumerate(int n, int m, const int* tail, const int* head, int directed, const double* p,
                   int source, int sink, int prefix_bits, const uint64_t* divs, int n_divs,
                   int threads, int want_grad, double* R_out, uint64_t* Nk_out, double* dRdp_out) {
  pcpu_job* jobs;
  pthread_t* tid;
  int t, k, b, rc = 0, started = 0;
  pcpu_kahan R = {0, 0}, G1[PCPU_MAXM], G0[PCPU_MAXM];
  if (n < 2 || n > PCPU_MAXN || m < 1 || m > PCPU_MAXM || !tail || !head || !p || !R_out) return -1;
  if (source < 0 || source >= n || sink < 0 || sink >= n || source == sink) return -1;
  if (prefix_bits < 0 || prefix_bits > m || n_divs < 0 || (n_divs > 0 && !divs)) return -1;
  if (want_grad && !dRdp_out) return -1;
  for (k = 0; k < m; ++k) {
    if (tail[k] < 0 || tail[k] >= n || head[k] < 0 || head[k] >= n || tail[k] == head[k]) return -1;
    if (!(p[k] >= 0.0 && p[k] <= 1.0)) return -1;
  }
  for (k = 0; k < n_divs; ++k)
    if (prefix_bits < 64 && divs[k] >= ((uint64_t)1 << prefix_bits)) return -1;
  if (threads < 1) threads = 1;
  if (threads > n_divs && n_divs > 0) threads = n_divs;
  jobs = (pcpu_job*)calloc((size_t)threads, sizeof(pcpu_job));
  tid = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
  if (!jobs || !tid) {
    free(jobs);
    free(tid);
    return -2;
  }
  for (t = 0; t < threads; ++t) {
    pcpu_job* J = &jobs[t];
    int by, v;
    J->n = n;
    J->m = m;
    J->directed = directed != 0;
    J->source = source;
    J->sink = sink;
    J->p = p;
    for (b = 0; b < m; ++b) {
      const int a = m - 1 - b; /* bit b holds input arc a (0-based) */
      J->arc_u[b] = tail[a];
      J->arc_v[b] = head[a];
      J->pb[b] = p[a];
      J->qb[b] = 1.0 - p[a];
    }
    J->nbytes = (m + 7) / 8;
    for (by = 0; by < J->nbytes; ++by)
      for (v = 0; v < 256; ++v) {
        double w = 1.0;
        for (b = 0; b < 8 && 8 * by + b < m; ++b)
          w *= ((v >> b) & 1) ? J->pb[8 * by + b] : J->qb[8 * by + b];
        J->bytetab[by][v] = w;
      }
    J->prefix_bits = prefix_bits;
    J->divs = divs;
    J->d0 = (int)((long long)n_divs * t / threads);
    J->d1 = (int)((long long)n_divs * (t + 1) / threads);
    J->want_grad = want_grad;
  }
  for (t = 0; t < threads; ++t) {
    if (pthread_create(&tid[t], NULL, pcpu_thread, &jobs[t]) != 0) {
      rc = -2;
      break;
    }
    ++started;
  }
  for (t = 0; t < started; ++t) pthread_join(tid[t], NULL);
  if (rc == 0) {
    /* STEP 3: the final sum over the threads, in thread order */
    for (k = 0; k < m; ++k) G1[k].s = G1[k].c = G0[k].s = G0[k].c = 0;
    if (Nk_out)
      for (k = 0; k <= m; ++k) Nk_out[k] = 0;
    for (t = 0; t < threads; ++t) {
      pcpu_add(&R, jobs[t].R.s);
      pcpu_add(&R, -jobs[t].R.c);
      if (Nk_out)
        for (k = 0; k <= m; ++k) Nk_out[k] += jobs[t].Nk[k];
      if (want_grad)
        for (b = 0; b < m; ++b) {
          pcpu_add(&G1[b], jobs[t].T1[b].s);
          pcpu_add(&G1[b], -jobs[t].T1[b].c);
          pcpu_add(&G0[b], jobs[t].T0[b].s);
          pcpu_add(&G0[b], -jobs[t].T0[b].c);
        }
    }
    *R_out = R.s - R.c;
    if (want_grad)
      for (b = 0; b < m; ++b) dRdp_out[m - 1 - b] = (G1[b].s - G1[b].c) - (G0[b].s - G0[b].c);
  }
  free(jobs);
  free(tid);
  return rc;
}
