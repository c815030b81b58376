/*
 * pbat_factoring.c -- a second exact method for two-terminal reliability of
 * UNDIRECTED networks, independent of the brute force in pbat_oracle.c.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the product path never
 * calls, links or loads it, and it shares nothing with the CUDA engine.  It
 * gives exact values of R (Eq. 1), of the counts N_k and of the T1/T0 sums
 * at sizes the brute force cannot finish (2^40 states and more), so that the
 * GPU results of full-size workloads can be compared value by value.
 *
 * Method: factoring on every arc in turn (pivotal decomposition, the
 * textbook identity R(G) = p_e R(G with e contracted) + (1 - p_e) R(G with e
 * deleted)), organised as a dynamic program over a fixed arc order.  After
 * the first i arcs have been decided, what the rest of the enumeration still
 * needs to know about the decided arcs is only which "frontier" nodes they
 * joined: a partition of the nodes that have decided and undecided arcs,
 * plus the source and the sink (kept in the frontier throughout).  The
 * program keeps one record per partition reached:
 *   w     the summed probability of the decided-arc states leading to it,
 *   N[j]  how many of those states have j working arcs.
 * Deciding the next arc e = {u, v}: its failed branch keeps the partition
 * (w times 1 - p_e); its working branch merges the blocks of u and v (w
 * times p_e, counts shifted by one).  A branch that puts source and sink in
 * one block is connected whatever the remaining r arcs do: it adds w to R
 * and N[j] * C(r, i) to N_{j + i} for i = 0..r.  Nodes whose last arc has
 * been decided leave the frontier.  Records left at the end are the
 * disconnected states.  Summing every state of {0,1}^m this way is exactly
 * Eq. 1; nothing is approximated (long double sums, uint64 counts).
 *
 * The arc order is chosen greedily to keep the frontier small (the next arc
 * adds the fewest new frontier nodes net of the nodes it retires; ties by
 * arc index).  Frontiers of up to 16 nodes are supported, partitions being
 * stored as 4-bit block labels in one 64-bit key.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FAC_MAXN 64
#define FAC_MAXM 63
#define FAC_MAXF 16

typedef struct {
  long double s, c; /* Neumaier sum */
} fac_sum;

static void fac_add(fac_sum* a, long double x) {
  long double t = a->s + x;
  if ((a->s >= 0 ? a->s : -a->s) >= (x >= 0 ? x : -x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}

/* A set of records keyed by partition, open addressing. */
typedef struct {
  int m1;          /* m + 1 counts per record */
  size_t n, cap;   /* records, capacity (power of two) */
  uint64_t* key;
  unsigned char* used;
  long double* w;
  uint64_t* N;     /* cap * m1 */
} fac_table;

static int fac_table_init(fac_table* T, int m1, size_t cap) {
  T->m1 = m1;
  T->n = 0;
  T->cap = cap;
  T->key = (uint64_t*)calloc(cap, sizeof(uint64_t));
  T->used = (unsigned char*)calloc(cap, 1);
  T->w = (long double*)calloc(cap, sizeof(long double));
  T->N = (uint64_t*)calloc(cap * (size_t)m1, sizeof(uint64_t));
  return (T->key && T->used && T->w && T->N) ? 0 : -1;
}

static void fac_table_free(fac_table* T) {
  free(T->key);
  free(T->used);
  free(T->w);
  free(T->N);
  memset(T, 0, sizeof *T);
}

static size_t fac_hash(uint64_t k, size_t cap) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  return (size_t)k & (cap - 1);
}

static int fac_table_grow(fac_table* T);

/* Add (w, counts shifted by `shift`) to the record of partition `key`. */
static int fac_table_add(fac_table* T, uint64_t key, long double w, const uint64_t* N, int shift) {
  size_t h;
  int j;
  if (2 * (T->n + 1) > T->cap && fac_table_grow(T)) return -1;
  h = fac_hash(key, T->cap);
  while (T->used[h] && T->key[h] != key) h = (h + 1) & (T->cap - 1);
  if (!T->used[h]) {
    T->used[h] = 1;
    T->key[h] = key;
    T->n++;
  }
  T->w[h] += w;
  for (j = 0; j + shift < T->m1; ++j) T->N[h * (size_t)T->m1 + j + shift] += N[j];
  return 0;
}

static int fac_table_grow(fac_table* T) {
  fac_table U;
  size_t i;
  if (fac_table_init(&U, T->m1, T->cap * 2)) {
    fac_table_free(&U);
    return -1;
  }
  for (i = 0; i < T->cap; ++i)
    if (T->used[i] && fac_table_add(&U, T->key[i], T->w[i], T->N + i * (size_t)T->m1, 0)) {
      fac_table_free(&U);
      return -1;
    }
  fac_table_free(T);
  *T = U;
  return 0;
}

static int fac_label(uint64_t key, int pos) { return (int)((key >> (4 * pos)) & 15u); }

/* Greedy arc order: fewest new frontier nodes net of retired ones. */
static void fac_order(int n, int m, const int* tail, const int* head, int source, int sink,
                      int* order) {
  int rem[FAC_MAXN], infront[FAC_MAXN], done[FAC_MAXM];
  int i, k;
  memset(rem, 0, sizeof rem);
  memset(infront, 0, sizeof infront);
  memset(done, 0, sizeof done);
  for (k = 0; k < m; ++k) {
    rem[tail[k]]++;
    rem[head[k]]++;
  }
  infront[source] = infront[sink] = 1;
  for (i = 0; i < m; ++i) {
    int best = -1, bnet = 0, bnew = 0;
    for (k = 0; k < m; ++k) {
      int u, v, add, ret;
      if (done[k]) continue;
      u = tail[k];
      v = head[k];
      add = !infront[u] + (!infront[v] && v != u);
      ret = (rem[u] == 1 && u != source && u != sink) + (rem[v] == 1 && v != source && v != sink);
      if (best < 0 || add - ret < bnet || (add - ret == bnet && add < bnew)) {
        best = k;
        bnet = add - ret;
        bnew = add;
      }
    }
    order[i] = best;
    done[best] = 1;
    infront[tail[best]] = infront[head[best]] = 1;
    rem[tail[best]]--;
    rem[head[best]]--;
    (void)n;
  }
}

/*
 * R and N_k of an undirected network by factoring.  p[k] in [0, 1].
 * Outputs: R as (hi, lo); Nk[m + 1] (nullable); *max_records (nullable) the
 * largest number of partitions held at once.
 * Returns 0; -1 bad input; -2 a frontier wider than 16 nodes; -3 out of memory.
 */
int orc_factor(int n, int m, const int* tail, const int* head, const double* p, int source,
               int sink, double* R_hi, double* R_lo, uint64_t* Nk, int* max_records) {
  int order[FAC_MAXM], last[FAC_MAXN];
  int front[FAC_MAXF + 2], nf;
  uint64_t binom[FAC_MAXM + 1][FAC_MAXM + 1];
  uint64_t Nout[FAC_MAXM + 1];
  fac_sum R = {0, 0};
  fac_table cur, nxt;
  int i, j, k, rc = 0, maxrec = 1;
  if (n < 2 || n > FAC_MAXN || m < 1 || m > FAC_MAXM || !tail || !head || !p) return -1;
  if (source < 0 || source >= n || sink < 0 || sink >= n || source == sink) return -1;
  for (k = 0; k < m; ++k) {
    if (tail[k] < 0 || tail[k] >= n || head[k] < 0 || head[k] >= n || tail[k] == head[k]) return -1;
    if (!(p[k] >= 0.0 && p[k] <= 1.0)) return -1;
  }
  for (i = 0; i <= m; ++i)
    for (j = 0; j <= m; ++j)
      binom[i][j] = j == 0 ? 1 : (i == 0 ? 0 : binom[i - 1][j - 1] + binom[i - 1][j]);
  memset(Nout, 0, sizeof Nout);
  fac_order(n, m, tail, head, source, sink, order);
  for (i = 0; i < n; ++i) last[i] = -1;
  for (i = 0; i < m; ++i) last[tail[order[i]]] = last[head[order[i]]] = i;
  /* frontier: source (label 0) and sink (label 1), in separate blocks */
  nf = 2;
  front[0] = source;
  front[1] = sink;
  if (fac_table_init(&cur, m + 1, 64)) {
    fac_table_free(&cur);
    return -3;
  }
  {
    uint64_t one[FAC_MAXM + 1];
    memset(one, 0, sizeof one);
    one[0] = 1;
    fac_table_add(&cur, (uint64_t)1 << 4, 1.0L, one, 0); /* labels: source 0, sink 1 */
  }
  for (i = 0; i < m && rc == 0; ++i) {
    const int e = order[i], u = tail[e], v = head[e];
    const int left = m - i - 1; /* arcs still undecided after this one */
    int nf2 = nf, pu = -1, pv = -1, keep[FAC_MAXF + 2], nkeep = 0;
    int front2[FAC_MAXF + 2];
    size_t h;
    memcpy(front2, front, sizeof(int) * nf);
    for (j = 0; j < nf; ++j) {
      if (front[j] == u) pu = j;
      if (front[j] == v) pv = j;
    }
    if (pu < 0) front2[pu = nf2++] = u;
    if (pv < 0) front2[pv = nf2++] = v;
    /* positions that stay after this arc: source, sink, nodes with arcs left */
    for (j = 0; j < nf2; ++j)
      if (front2[j] == source || front2[j] == sink || last[front2[j]] > i) keep[nkeep++] = j;
    if (nkeep > FAC_MAXF) {
      rc = -2;
      break;
    }
    if (fac_table_init(&nxt, m + 1, 64)) {
      rc = -3;
      break;
    }
    for (h = 0; h < cur.cap && rc == 0; ++h) {
      int lab[FAC_MAXF + 2], b;
      if (!cur.used[h]) continue;
      /* current labels; new frontier nodes get fresh blocks */
      {
        int mx = -1;
        for (j = 0; j < nf; ++j) {
          lab[j] = fac_label(cur.key[h], j);
          if (lab[j] > mx) mx = lab[j];
        }
        for (j = nf; j < nf2; ++j) lab[j] = ++mx;
      }
      for (b = 0; b < 2 && rc == 0; ++b) {
        int L[FAC_MAXF + 2], map[FAC_MAXF + 2], nb = 0;
        uint64_t key = 0;
        const long double w =
            cur.w[h] * (b ? (long double)p[e] : 1.0L - (long double)p[e]);
        const uint64_t* N = cur.N + h * (size_t)cur.m1;
        memcpy(L, lab, sizeof(int) * nf2);
        if (b) { /* arc works: merge the blocks of u and v */
          const int from = L[pv], to = L[pu];
          for (j = 0; j < nf2; ++j)
            if (L[j] == from) L[j] = to;
        }
        if (L[0] == L[1]) { /* source and sink joined: every completion connects */
          int q, r;
          fac_add(&R, w);
          for (q = 0; q <= m; ++q) {
            if (!N[q]) continue;
            for (r = 0; r <= left; ++r) Nout[q + b + r] += N[q] * binom[left][r];
          }
          continue;
        }
        /* keep the surviving positions, relabel blocks by first occurrence */
        for (j = 0; j < FAC_MAXF + 2; ++j) map[j] = -1;
        for (j = 0; j < nkeep; ++j) {
          const int l = L[keep[j]];
          if (map[l] < 0) map[l] = nb++;
          key |= (uint64_t)map[l] << (4 * j);
        }
        if (fac_table_add(&nxt, key, w, N, b)) rc = -3;
      }
    }
    fac_table_free(&cur);
    cur = nxt;
    for (j = 0; j < nkeep; ++j) front[j] = front2[keep[j]];
    nf = nkeep;
    if ((int)cur.n > maxrec) maxrec = (int)cur.n;
  }
  fac_table_free(&cur);
  if (rc) return rc;
  {
    const long double v = R.s + R.c;
    const double hi = (double)v;
    *R_hi = hi;
    *R_lo = (double)(v - (long double)hi);
  }
  if (Nk)
    for (k = 0; k <= m; ++k) Nk[k] = Nout[k];
  if (max_records) *max_records = maxrec;
  return 0;
}
