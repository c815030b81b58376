/*
 * pbat.h -- C ABI of the GB300 PBAT engine: exact two-terminal reliability
 * of a binary-state network by enumerating every arc-state vector.
 *
 * Problem (arXiv 2209.09711, Sec. 2 and Sec. 5.1 "Input/Output" of PBAT):
 * a network G(V, E, D_b) with n nodes and m arcs, where arc a_k works with
 * probability p_k independently of the others (Sec. 2.4 assumption 2).
 * The reliability is
 *
 *     R = sum over arc-state vectors X in {0,1}^m with the sink reachable
 *         from the source in G(X) of  prod_k (x_k ? p_k : 1 - p_k)   (Eq. 1)
 *
 * and the engine also returns the reliability-polynomial counts
 * N_k = #{connected X with exactly k working arcs} and the gradient
 * dR/dp_k.  Connectivity is the PLSA reachability test of Sec. 3.2.
 *
 * Conventions shared by every call:
 *   - Node ids are 0-based, in [0, n_nodes).  The paper's source node 1 and
 *     sink node n are simply `source` and `sink` here.
 *   - Arc k joins tail[k] and head[k].  directed != 0: usable tail -> head
 *     only; directed == 0: usable both ways.  Loops (tail == head) are
 *     rejected (Sec. 2.4 assumption 3); parallel arcs are accepted -- the
 *     sum in Eq. 1 is unchanged by them.
 *   - Arc order is the paper's coordinate order: arc 0 is the first
 *     coordinate x_1, the most significant bit of the state index
 *     (Sec. 4.2, Eq. 2-3).  The engine may permute arcs internally; every
 *     output is in input arc order.
 *   - Limits: 2 <= n_nodes <= 64, 1 <= n_arcs <= 63.
 *   - All pointers are HOST pointers unless a name says otherwise.  The
 *     caller owns every array; the library copies what it needs and keeps no
 *     pointer after the call returns.
 *   - Every call returns PBAT_OK (0) or a negative PBAT_E* code.  On error no
 *     output array is written, and pbat_last_error() (thread-local) gives a
 *     one-line reason.  No C++ exception crosses this boundary.
 *   - Environment: PBAT_AUTOTUNE_CACHE names a file that keeps the
 *     autotuner's choices across processes.  PBAT_FAULT, for failure-
 *     detection tests, lists host-side sites to fail ("plan", "compile",
 *     "alloc", "launch", comma-separated): each fails as its real call can,
 *     with the same error code, before any GPU work of that step.
 *   - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).
 *     The calls are synchronous: they return after the results are on the
 *     host.  Calls are re-entrant; concurrent calls from several host
 *     threads are allowed.
 */
#ifndef PBAT_H
#define PBAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PBAT_OK 0
#define PBAT_EINVAL (-1)   /* malformed input: ids out of range, loop, source == sink, p not in [0,1] */
#define PBAT_ERANGE (-2)   /* n_nodes > 64, n_arcs > 63, or a size past a stated maximum */
#define PBAT_ECUDA (-3)    /* a CUDA runtime/driver call or a kernel failed */
#define PBAT_ETIMEOUT (-4) /* opt->time_budget_s ran out on the device; results discarded */
#define PBAT_ENOMEM (-5)   /* device or host allocation failed */
#define PBAT_ENOTSUP (-6)  /* the requested algorithm cannot run this input */

/* Connectivity kernels (the "a5" step of the hot path). */
#define PBAT_ALGO_AUTO 0
#define PBAT_ALGO_FRONTIER 1  /* one state per thread, bitmask frontier expansion (PLSA) */
#define PBAT_ALGO_BITSLICE 2  /* 32 states per thread word, kernel specialised per graph */

typedef struct pbat_options {
  int struct_size;      /* sizeof(pbat_options); set by pbat_options_init */
  int algo;             /* PBAT_ALGO_*; AUTO: the bit-sliced kernel, re-run exactly with the
                           frontier kernel when R is too small for the bit-sliced kernel's
                           fixed-point error bound to give 1e-12 relative accuracy */
  int prefix_bits;      /* d: arcs fixed per work item (equal division, Sec. 4.3); -1 = auto */
  int walk_bits;        /* L: arcs each thread walks in Gray-code order; -1 = auto */
  int block_threads;    /* threads per CTA; -1 = auto */
  int prune;            /* 1 (default): exact monotone prefix prune; 0: walk every state;
                           2: the prune, with the bit-sliced kernels' prefix arcs chosen
                           to maximise the work items it resolves (a deterministic search
                           at planning time, tenths of a second for 30-40 arcs, kept per
                           network).  Every setting gives the same exact results. */
  int autotune;         /* 1 (default): for problems of at least 2^26 states with walk_bits,
                           block_threads and prefix_bits all -1, time candidate launch
                           shapes once per network structure and keep the fastest
                           (in memory, and in the file named by PBAT_AUTOTUNE_CACHE) */
  int occupancy;        /* blocks per SM the bit-sliced single-network kernels are compiled
                           for: k >= 1 gives them __launch_bounds__(threads, k), so the
                           compiler keeps their registers within 65536 / (k * threads);
                           0 = the compiler's own register choice; -1 (default) = 0, or
                           the autotuner's choice when it runs.  The bit-sliced batched
                           module takes it as its launch bounds (128 threads, k blocks;
                           0 and -1 = 4 blocks).  Results do not depend on it. */
  int launches;         /* bit-sliced single-network kernels with the prune on: 1 = one
                           launch; 2 = two launches, the first resolving what the prune can
                           and deferring the work items left to walk, the second walking
                           them (at most 2^24 items, else one launch); 0 (default) = two
                           for the fused kernel with 2^18 to 2^24 items, else one, or the
                           autotuner's choice when it runs.  Results do not depend on it. */
  int range_bits;       /* 0 (default) = whole space.  Otherwise only the states whose
                           first range_bits coordinates, read as an integer, lie in
                           [range_lo, range_hi) -- the divisions range_lo..range_hi-1 of
                           Eq. 6 with chi = 2^range_bits.  Partial results of disjoint
                           ranges add up to the full result (checkpoint / resume). */
  uint64_t range_lo;
  uint64_t range_hi;
  double time_budget_s; /* > 0: the device stops after this many seconds and the call
                           returns PBAT_ETIMEOUT; 0 = no limit */
  uint64_t stats[8];    /* out, filled by the last call that took these options:
                           [0] states enumerated by walking, [1] states resolved by the
                           prune, [2] bytes copied host -> device, [3] bytes copied
                           device -> host, [4] summed device time in ns of the
                           enumeration kernel over the launches since the last read (CUDA
                           events on the launch stream), [5] kernels launched (one per
                           bit-sliced launch; the frontier kernel adds a reduce), [6] work
                           items per launch, [7] launches timed in [4] */
} pbat_options;

/* Fill *opt with the defaults above. */
void pbat_options_init(pbat_options* opt);

/*
 * R and N_k of one network (Eq. 1; PBAT STEP 0-3 of Sec. 5.1).
 *   p        [n_arcs] arc reliabilities, each in [0, 1]
 *   opt      nullable (defaults)
 *   R_out    out, 1 double: R (or the partial R of opt's range)
 *   Nk_out   out, nullable, n_arcs + 1 uint64: N_0 .. N_m
 */
int pbat_reliability(int n_nodes, int n_arcs, const int32_t* tail, const int32_t* head,
                     int directed, const double* p, int source, int sink,
                     pbat_options* opt, void* cuda_stream, double* R_out, uint64_t* Nk_out);

/*
 * As pbat_reliability, plus the gradient dR/dp_k (Birnbaum importance of
 * arc k) from one fused enumeration.  R is affine in every p_k, so
 * dR/dp_k = R(p_k = 1) - R(p_k = 0); the engine differentiates Eq. 1 term
 * by term in exact fixed-point sums.
 *   dRdp_out out, n_arcs doubles (input arc order)
 * With opt->range_bits > 0 the gradient is that of the partial R.
 */
int pbat_reliability_grad(int n_nodes, int n_arcs, const int32_t* tail, const int32_t* head,
                          int directed, const double* p, int source, int sink,
                          pbat_options* opt, void* cuda_stream, double* R_out, uint64_t* Nk_out,
                          double* dRdp_out);

/* One network of a batch. */
typedef struct pbat_graph {
  int n_nodes;
  int n_arcs;
  const int32_t* tail;
  const int32_t* head;
  int directed;
  int source;
  int sink;
} pbat_graph;

/*
 * Many networks, each with n_pvec arc-reliability vectors, in one
 * persistent launch (captured once in a CUDA graph and replayed).  Each
 * state's connectivity is computed once and weighted by every p-vector.
 * With dRdp_out, one launch of the gradient module gives R, N_k and dR/dp
 * for every (network, p-vector); pairs whose R or gradient the bit-sliced
 * fixed-point bounds cannot certify to 1e-12 (small R) are re-run exactly
 * with the frontier kernel, one enumeration each.  opt->stats[4] holds the
 * device time of the batched launch in ns.
 *   p         per graph g: n_pvec x m_g doubles (vector-major), concatenated in
 *             graph order
 *   R_out     out, n_graphs x n_pvec doubles (graph-major)
 *   Nk_out    out, nullable, sum over g of (m_g + 1) uint64, graph order
 *   dRdp_out  out, nullable, same layout as p
 * Limits: 1 <= n_graphs <= 4096, 1 <= n_pvec <= 64.
 */
int pbat_reliability_batched(int n_graphs, const pbat_graph* graphs, int n_pvec,
                             const double* p, pbat_options* opt, void* cuda_stream,
                             double* R_out, uint64_t* Nk_out, double* dRdp_out);

/*
 * Prepared enumerations.  pbat_plan_create validates the input, plans the
 * equal division, builds the tables and uploads them to the device once;
 * pbat_plan_execute then runs the whole enumeration (every kernel, no host
 * work, no copies) on `cuda_stream` and returns without waiting;
 * pbat_plan_read copies the results of the last execute back and waits.
 * A plan owns its device scratch until pbat_plan_destroy; one plan must not
 * be executed on two streams at once.
 *   want_grad  0: R and N_k; 1: R, N_k and dR/dp (fused kernel)
 *   plan_out   out: the new plan
 */
typedef struct pbat_plan_s* pbat_plan;
int pbat_plan_create(int n_nodes, int n_arcs, const int32_t* tail, const int32_t* head,
                     int directed, const double* p, int source, int sink, int want_grad,
                     pbat_options* opt, void* cuda_stream, pbat_plan* plan_out);
int pbat_plan_execute(pbat_plan plan, void* cuda_stream);
int pbat_plan_read(pbat_plan plan, void* cuda_stream, double* R_out, uint64_t* Nk_out,
                   double* dRdp_out);
void pbat_plan_destroy(pbat_plan plan);
/* Describe a plan (no device work): out8 = {algo (PBAT_ALGO_FRONTIER or
 * PBAT_ALGO_BITSLICE), lane arcs, thread arcs (0 for the frontier kernel),
 * walk arcs, prefix arcs, threads per block, blocks, 1 if the gradient is
 * computed}. */
int pbat_plan_describe(pbat_plan plan, int* out8);
/* Copy the plan's statistics (the pbat_options.stats[8] layout, as filled by
 * the last pbat_plan_read) into stats_out[8]. */
int pbat_plan_stats(pbat_plan plan, uint64_t* stats_out);

/*
 * pbat_reliability_noalloc -- R and N_k exactly as pbat_reliability computes
 * them, for callers that cannot allocate device memory: code whose device
 * memory belongs to a framework's caching allocator or is capped per
 * process, and latency-critical paths that must not stall on an
 * allocation.  The paper has no counterpart; this is an engineering entry
 * point of this library.
 *
 * It calls no cudaMalloc, cudaFree, cudaMallocHost or other allocating
 * routine.  Its scratch is one static 512 KiB device array inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  Limits that follow from that size: opt->walk_bits <= 12 (a larger
 * value returns PBAT_ERANGE, where pbat_reliability would quietly use 12),
 * and the persistent grid is capped at the number of per-block partials
 * that fit.  The gradient is not offered here.
 *   arguments, layout and ownership: as pbat_reliability (host arrays in and
 *   out; opt nullable, algo must be AUTO or FRONTIER; opt->stats untouched)
 * Every call looks up the array's device address with the caller's device
 * current (a lookup, no allocation), so a device reset between calls is
 * harmless.  The call copies through host memory and waits for its stream,
 * so it must not be called while that stream is being captured into a CUDA
 * graph: it returns PBAT_ENOTSUP then.  Every call shares the one array;
 * work of two calls that overlapped on the GPU would race on it, so the
 * library runs the calls one at a time (a lock held for the whole call).
 * A call uses a few KiB of the caller's stack.
 */
int pbat_reliability_noalloc(int n_nodes, int n_arcs, const int32_t* tail, const int32_t* head,
                             int directed, const double* p, int source, int sink,
                             const pbat_options* opt, void* cuda_stream, double* R_out,
                             uint64_t* Nk_out);

/*
 * Diagnostic, no GPU needed: the CUDA C++ source the engine generates and
 * compiles (NVRTC) for the bit-sliced kernel of this network and options --
 * the per-graph connectivity program of the PLSA test (Sec. 3.2) as
 * straight-line Boolean elimination on 32-state words, inside the kernel
 * template.  The first line lists the internal arc order.
 *   p          nullable; with want_grad the plan depends on p (walk arcs need
 *              p in [2^-20, 1 - 2^-20]); NULL treats every arc as eligible
 *   want_grad  0: the R + N_k kernel's plan; 1: the fused kernel's plan
 * Writes at most cap bytes (NUL-terminated) to buf (nullable) and returns the
 * full length, or a negative PBAT_E* code.
 */
int pbat_kernel_source(int n_nodes, int n_arcs, const int32_t* tail, const int32_t* head,
                       int directed, const double* p, int source, int sink, int want_grad,
                       const pbat_options* opt, char* buf, size_t cap);

/* Diagnostic, no GPU needed: the CUDA C++ source of the batched bit-sliced
 * module (every network's connectivity program and the persistent kernel)
 * for these networks and n_pvec p-vectors.  Same buffer convention as
 * pbat_kernel_source. */
int pbat_batch_kernel_source(int n_graphs, const pbat_graph* graphs, int n_pvec,
                             const pbat_options* opt, char* buf, size_t cap);

/* Diagnostic, no GPU needed: the CUDA C++ source of the batched gradient
 * module (every network's connectivity program and the persistent kernel
 * that also forms dR/dp for every p-vector).  p: as for
 * pbat_reliability_batched, or NULL; it decides which arcs may be walk
 * arcs (p in [2^-20, 1 - 2^-20] under every p-vector).  Same buffer
 * convention as pbat_kernel_source. */
int pbat_batch_grad_kernel_source(int n_graphs, const pbat_graph* graphs, int n_pvec,
                                  const double* p, const pbat_options* opt, char* buf,
                                  size_t cap);

/* Thread-local description of the last error in this thread ("" if none). */
const char* pbat_last_error(void);

/* ABI version: major * 10000 + minor * 100 + patch. */
int pbat_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PBAT_H */
