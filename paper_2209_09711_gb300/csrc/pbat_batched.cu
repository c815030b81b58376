// pbat_batched.cu -- many networks, many p-vectors, one persistent launch:
// the entry point, and the frontier (one state per thread) variant.  The
// default path is the bit-sliced batched module of pbat_bitslice.cu; this
// variant runs on request (PBAT_ALGO_FRONTIER), past that module's limits,
// and as the independent cross-check of its tests.
//
// The work items of every network (its prefix values, Sec. 4.3 equal
// division) are laid end to end, networks with the most items first, and a
// persistent grid takes them from one atomic ticket.  Each state's
// connectivity (PLSA, Sec. 3.2, as bitmask frontier expansion) is computed
// once and its walk-arc mass is added for every p-vector of the chunk, each
// into its own 128-bit fixed-point register sum.  Per item and p-vector the
// result Pr(prefix) * sum_lanes Pr(lane) * T is added exactly into five
// 64-bit limbs of a 160-bit fixed-point accumulator with integer atomics, so
// the batched R does not depend on the order items finish.  The sequence
// (scratch reset + one kernel per chunk of up to 16 p-vectors) is captured
// once in a CUDA graph per batch structure and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "pbat.h"
#include "pbat_engine.h"
#include "pbat_internal.h"

namespace pbat {

constexpr int kBatchWalkBits = 8;
constexpr int kBatchChunk = 16;
constexpr int kLimbs = 5;           // 160-bit accumulator, 32-bit chunks per 64-bit limb
constexpr int kLimbScale = 158;     // value * 2^158 < 2^160 for value <= 1

struct BatchGraphDev {
  int n, m, directed, source, sink, ell, L, d;
  unsigned long long task_begin, n_tasks, free_mask;
  int wmid_off;  // u128 index of p-vector 0's walk table; vector k at + (k << L)
  int nk_off;    // first N_k slot of this network
  int gidx;      // index of this network in input order
  int pad;
  unsigned char au[64], av[64];
  unsigned long long grp[64];
  unsigned long long binom[64];
};

struct BatchArrays {
  const BatchGraphDev* graphs;
  const double* bp;   // [(g*K + k) * 64 + arc]
  const dd* bq;       // [(g*K + k) * 64 + arc]
  const dd* blane;    // [(g*K + k) * 32 + j]
  const u128* bwmid;  // walk tables
  unsigned long long* limbs;  // [(g*K + k) * kLimbs + i]
  unsigned long long* nk;
  unsigned long long* counter;
  unsigned int* status;
  int G, K;
  unsigned long long total_tasks;
  unsigned long long budget_ns;
  int prune;
  int max_n;
};

__device__ __forceinline__ unsigned long long b_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ dd b_warp_sum(dd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = dd_add(v, w);
  }
  return v;
}

__device__ bool b_state_connected(const BatchGraphDev& Gd, unsigned long long x) {
  unsigned long long reach = 1ull << Gd.source;
  const unsigned long long tb = 1ull << Gd.sink;
  for (int pass = 0; pass < Gd.n; ++pass) {
    const unsigned long long before = reach;
    for (int k = 0; k < Gd.m; ++k) {
      if (!((x >> k) & 1ull)) continue;
      const unsigned long long bu = 1ull << Gd.au[k], bv = 1ull << Gd.av[k];
      if (reach & bu) reach |= bv;
      if (!Gd.directed && (reach & bv)) reach |= bu;
    }
    if (reach & tb) return true;
    if (reach == before) return false;
  }
  return (reach & tb) != 0;
}

__device__ __forceinline__ bool b_sink_reached(const unsigned long long* adj, int stride,
                                               unsigned long long sbit, unsigned long long tbit) {
  unsigned long long vis = sbit, fr = sbit;
  while (fr) {
    const int u = __ffsll((long long)fr) - 1;
    fr &= fr - 1;
    const unsigned long long nb = adj[u * stride] & ~vis;
    if (nb & tbit) return true;
    vis |= nb;
    fr |= nb;
  }
  return false;
}

// Atomically add round(x * 2^kLimbScale) (x may be negative) to the limbs.
__device__ void limb_add(unsigned long long* limbs, double x) {
  if (x == 0.0) return;
  const bool neg = x < 0.0;
  int ex;
  const double mant = frexp(fabs(x), &ex);
  long long M = (long long)ldexp(mant, 53);
  int e = ex - 53 + kLimbScale;
  if (e < 0) {
    if (-e > 62) return;
    M = (M + (1ll << (-e - 1))) >> (-e);
    e = 0;
    if (M == 0) return;
  }
  const int c = e >> 5, sh = e & 31;
  const unsigned __int128 v = (unsigned __int128)(unsigned long long)M << sh;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const unsigned long long chunk = (unsigned long long)(uint32_t)(v >> (32 * i));
    if (chunk && c + i < kLimbs)
      atomicAdd(&limbs[c + i], neg ? (unsigned long long)(-(long long)chunk) : chunk);
  }
}

__device__ __forceinline__ void limb_add_dd(unsigned long long* limbs, dd v) {
  limb_add(limbs, v.hi);
  limb_add(limbs, v.lo);
}

template <int KC>
__global__ void __launch_bounds__(128) batched_kernel(const __grid_constant__ BatchArrays A,
                                                      int k0) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nthr = blockDim.x, tid = threadIdx.x, lane = tid & 31;
  unsigned long long* adj = reinterpret_cast<unsigned long long*>(smem) + tid;
  const int kc = min(KC, A.K - k0);
  const unsigned long long t_start = b_globaltimer();

  for (;;) {
    unsigned long long task = 0;
    if (lane == 0) {
      task = atomicAdd(A.counter, 1ull);
      if (A.budget_ns && b_globaltimer() - t_start > A.budget_ns) {
        atomicOr(A.status, 1u);
        task = ~0ull;
      }
    }
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= A.total_tasks) break;
    int lo = 0, hi = A.G - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (A.graphs[mid].task_begin <= task) lo = mid; else hi = mid - 1;
    }
    const BatchGraphDev& Gd = A.graphs[lo];
    const int ell = Gd.ell, L = Gd.L, m = Gd.m, n = Gd.n, top = ell + L;
    const unsigned long long prefix = task - Gd.task_begin;
    const unsigned long long xpre = prefix << top;
    const int gk0 = Gd.gidx * A.K + k0;
    // prefix mass of p-vector k0 + lane, one lane per vector
    dd wpre_l = dd{0.0, 0.0};
    if (lane < kc) {
      const double* pp = A.bp + (size_t)(gk0 + lane) * 64;
      const dd* qq = A.bq + (size_t)(gk0 + lane) * 64;
      wpre_l = dd{1.0, 0.0};
      for (int j = 0; j < Gd.d; ++j) {
        const int k = top + j;
        wpre_l = ((prefix >> j) & 1ull) ? dd_mul_d(wpre_l, pp[k]) : dd_mul(wpre_l, qq[k]);
      }
    }
    const int pc_pre = __popcll((long long)prefix);
    if (A.prune) {
      if (!b_state_connected(Gd, xpre | Gd.free_mask)) continue;
      if (b_state_connected(Gd, xpre)) {
        if (k0 == 0)
          for (int j = lane; j <= top; j += 32) atomicAdd(&A.nk[Gd.nk_off + pc_pre + j], Gd.binom[j]);
        if (lane < kc) limb_add_dd(A.limbs + (size_t)(gk0 + lane) * kLimbs, wpre_l);
        continue;
      }
    }
    const bool lane_on = lane < (1 << ell);
    unsigned long long x = xpre | (unsigned long long)(lane_on ? lane : 0);
    for (int u = 0; u < n; ++u) adj[u * nthr] = 0ull;
    for (int k = 0; k < m; ++k) {
      if ((x >> k) & 1ull) {
        adj[Gd.au[k] * nthr] |= 1ull << Gd.av[k];
        if (!Gd.directed) adj[Gd.av[k] * nthr] |= 1ull << Gd.au[k];
      }
    }
    const unsigned long long sbit = 1ull << Gd.source, tbit = 1ull << Gd.sink;
    bool conn = b_sink_reached(adj, nthr, sbit, tbit);
    u128 T[KC];
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) T[kk] = u128_zero();
    uint32_t ncnt[kBatchWalkBits + 1];
#pragma unroll
    for (int c = 0; c <= kBatchWalkBits; ++c) ncnt[c] = 0;
    const u128* W0 = A.bwmid + Gd.wmid_off + ((size_t)k0 << L);
    auto add_state = [&](uint32_t g, int pc) {
#pragma unroll
      for (int kk = 0; kk < KC; ++kk)
        if (kk < kc) u128_add_to(T[kk], W0[((size_t)kk << L) + g]);
#pragma unroll
      for (int c = 0; c <= kBatchWalkBits; ++c) ncnt[c] += (c == pc) ? 1u : 0u;
    };
    if (conn) add_state(0, 0);
    uint32_t g = 0;
    int pc = 0;
    const uint32_t nW = 1u << L;
    for (uint32_t s = 1; s < nW; ++s) {
      const int b = __ffs(s) - 1;
      const int k = ell + b;
      const unsigned long long bit = 1ull << k;
      x ^= bit;
      g ^= 1u << b;
      const bool added = (x & bit) != 0ull;
      const int u = Gd.au[k], v = Gd.av[k];
      const bool present = (x & Gd.grp[k]) != 0ull;
      unsigned long long* ru = adj + u * nthr;
      *ru = present ? (*ru | (1ull << v)) : (*ru & ~(1ull << v));
      if (!Gd.directed) {
        unsigned long long* rv = adj + v * nthr;
        *rv = present ? (*rv | (1ull << u)) : (*rv & ~(1ull << u));
      }
      pc += added ? 1 : -1;
      if (added != conn) conn = b_sink_reached(adj, nthr, sbit, tbit);
      if (conn) add_state(g, pc);
    }
    if (k0 == 0 && lane_on) {
      const int base = Gd.nk_off + pc_pre + __popc(lane);
#pragma unroll
      for (int c = 0; c <= kBatchWalkBits; ++c)
        if (ncnt[c]) atomicAdd(&A.nk[base + c], (unsigned long long)ncnt[c]);
    }
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      if (kk >= kc) break;
      const dd t = dd_ldexp(u128_to_dd(T[kk]), -127);
      const dd lw = lane_on ? A.blane[(size_t)(gk0 + kk) * 32 + lane] : dd{0.0, 0.0};
      const dd wsum = b_warp_sum(dd_mul(lw, t));
      dd wp;
      wp.hi = __shfl_sync(0xffffffffu, wpre_l.hi, kk);
      wp.lo = __shfl_sync(0xffffffffu, wpre_l.lo, kk);
      if (lane == kk) limb_add_dd(A.limbs + (size_t)(gk0 + kk) * kLimbs, dd_mul(wp, wsum));
    }
  }
}

template <int KC>
static cudaError_t launch_batched_kc(const BatchArrays& A, int k0, int grid, int nthr, size_t smem,
                                     cudaStream_t st) {
  batched_kernel<KC><<<grid, nthr, smem, st>>>(A, k0);
  return cudaGetLastError();
}

static const void* batched_kernel_ptr(int kc) {
  switch (kc) {
    case 1: return (const void*)batched_kernel<1>;
    case 2: return (const void*)batched_kernel<2>;
    case 4: return (const void*)batched_kernel<4>;
    case 8: return (const void*)batched_kernel<8>;
    default: return (const void*)batched_kernel<16>;
  }
}

static int chunk_template(int kc) { return kc <= 1 ? 1 : kc <= 2 ? 2 : kc <= 4 ? 4 : kc <= 8 ? 8 : 16; }

static cudaError_t launch_batched(int kct, const BatchArrays& A, int k0, int grid, int nthr,
                                  size_t smem, cudaStream_t st) {
  switch (kct) {
    case 1: return launch_batched_kc<1>(A, k0, grid, nthr, smem, st);
    case 2: return launch_batched_kc<2>(A, k0, grid, nthr, smem, st);
    case 4: return launch_batched_kc<4>(A, k0, grid, nthr, smem, st);
    case 8: return launch_batched_kc<8>(A, k0, grid, nthr, smem, st);
    default: return launch_batched_kc<16>(A, k0, grid, nthr, smem, st);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
#define PBAT_BCUDA(call)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(PBAT_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                  __FILE__, __LINE__);                                                    \
  } while (0)

static size_t bup(size_t x) { return (x + 255) & ~(size_t)255; }

// One cached batch: scratch layout plus the instantiated CUDA graph.
struct BatchEntry {
  std::string key;
  bool busy = false;
  int device = -1;
  Scratch* scr = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t captured_on = nullptr;
  // layout (byte offsets into the device / host scratch)
  size_t o_graphs, o_bp, o_bq, o_blane, o_wmid, o_limbs, o_nk, o_counter, o_status;
  size_t upload_bytes;  // [o_graphs, o_limbs) is uploaded from the same host offsets
  size_t d_total, h_total;
  std::vector<int> order;  // launch order -> input graph index
  std::vector<BatchGraphDev> gd;  // in launch order
  std::vector<std::vector<int>> perm;
  int G = 0, K = 0, grid = 0, nthr = 128, max_n = 2;
  size_t smem = 0;
  unsigned long long total_tasks = 0;
  int nk_total = 0;
  BatchArrays A{};
};

static std::mutex g_bmu;
static std::vector<BatchEntry*> g_batches;

static std::string batch_key(int device, int G, const pbat_graph* graphs, int K,
                             const pbat_options& o) {
  std::string k;
  auto put = [&](long long v) { k.append((const char*)&v, sizeof v); };
  put(device); put(G); put(K); put(o.prune); put(o.walk_bits); put(o.block_threads);
  put(o.occupancy); put(o.autotune);
  put((long long)(o.time_budget_s * 1e9));
  for (int i = 0; i < G; ++i) {
    const pbat_graph& g = graphs[i];
    put(g.n_nodes); put(g.n_arcs); put(g.directed); put(g.source); put(g.sink);
    k.append((const char*)g.tail, sizeof(int32_t) * g.n_arcs);
    k.append((const char*)g.head, sizeof(int32_t) * g.n_arcs);
  }
  return k;
}

static int batch_build(BatchEntry& E, int G, const pbat_graph* graphs, int K,
                       const pbat_options& o, const DeviceInfo& dev) {
  E.G = G;
  E.K = K;
  E.device = dev.device;
  const int Lb = o.walk_bits >= 0 ? std::min(o.walk_bits, kBatchWalkBits) : kBatchWalkBits;
  std::vector<BatchGraphDev> gd(G);
  E.perm.assign(G, {});
  int nk_off = 0;
  std::vector<int> nk_offs(G);
  for (int i = 0; i < G; ++i) {
    nk_offs[i] = nk_off;
    nk_off += graphs[i].n_arcs + 1;
  }
  E.nk_total = nk_off;
  std::vector<unsigned long long> items(G);
  for (int i = 0; i < G; ++i) {
    const pbat_graph& g = graphs[i];
    BatchGraphDev& b = gd[i];
    memset(&b, 0, sizeof b);
    const int m = g.n_arcs;
    b.n = g.n_nodes; b.m = m; b.directed = g.directed ? 1 : 0;
    b.source = g.source; b.sink = g.sink;
    b.ell = std::min(kMaxLaneBits, m);
    b.L = std::max(0, std::min(Lb, m - b.ell));
    b.d = m - b.ell - b.L;
    if (b.d >= 48) return fail(PBAT_ERANGE, "network %d: %d prefix bits is too many", i, b.d);
    b.n_tasks = 1ull << b.d;
    b.free_mask = (b.ell + b.L >= 64) ? ~0ull : ((1ull << (b.ell + b.L)) - 1ull);
    b.nk_off = nk_offs[i];
    b.gidx = i;
    E.perm[i].resize(m);
    for (int k = 0; k < m; ++k) E.perm[i][k] = m - 1 - k;  // state word == paper index
    for (int k = 0; k < m; ++k) {
      const int a = E.perm[i][k];
      b.au[k] = (unsigned char)g.tail[a];
      b.av[k] = (unsigned char)g.head[a];
    }
    for (int k = 0; k < m; ++k) {
      unsigned long long gm = 0;
      for (int j = 0; j < m; ++j) {
        const bool same = g.directed ? (b.au[k] == b.au[j] && b.av[k] == b.av[j])
                                     : ((b.au[k] == b.au[j] && b.av[k] == b.av[j]) ||
                                        (b.au[k] == b.av[j] && b.av[k] == b.au[j]));
        if (same) gm |= 1ull << j;
      }
      b.grp[k] = gm;
    }
    for (int j = 0; j < 64; ++j) b.binom[j] = binom_u64(b.ell + b.L, j);
    items[i] = b.n_tasks;
    E.max_n = std::max(E.max_n, b.n);
  }
  // longest first: networks with the most work items start first
  E.order.resize(G);
  std::iota(E.order.begin(), E.order.end(), 0);
  std::stable_sort(E.order.begin(), E.order.end(),
                   [&](int a, int b) { return items[a] > items[b]; });
  unsigned long long begin = 0;
  int wmid_off = 0;
  std::vector<int> wmid_offs(G);
  for (int i = 0; i < G; ++i) {
    wmid_offs[i] = wmid_off;
    wmid_off += K << gd[i].L;
  }
  E.gd.resize(G);
  for (int r = 0; r < G; ++r) {
    const int i = E.order[r];
    gd[i].task_begin = begin;
    gd[i].wmid_off = wmid_offs[i];
    begin += gd[i].n_tasks;
    E.gd[r] = gd[i];
  }
  E.total_tasks = begin;
  // scratch layout: the upload block [graphs .. wmid] mirrors the host staging
  size_t off = 0;
  E.o_graphs = off; off = bup(off + sizeof(BatchGraphDev) * G);
  E.o_bp = off; off = bup(off + sizeof(double) * 64 * (size_t)G * K);
  E.o_bq = off; off = bup(off + sizeof(dd) * 64 * (size_t)G * K);
  E.o_blane = off; off = bup(off + sizeof(dd) * 32 * (size_t)G * K);
  E.o_wmid = off; off = bup(off + sizeof(u128) * (size_t)wmid_off);
  E.upload_bytes = off;
  E.o_limbs = off; off = bup(off + 8 * (size_t)kLimbs * G * K);
  E.o_nk = off; off = bup(off + 8 * (size_t)E.nk_total);
  E.o_counter = off; off = bup(off + 8);
  E.o_status = off; off = bup(off + 4);
  E.d_total = off;
  E.h_total = off;
  int rc = scratch_acquire(dev.device, E.d_total, E.h_total, &E.scr);
  if (rc) return rc;
  char* d = (char*)E.scr->dmem;
  memcpy((char*)E.scr->hmem + E.o_graphs, E.gd.data(), sizeof(BatchGraphDev) * G);
  // launch shape
  E.nthr = o.block_threads > 0 ? std::min(o.block_threads, 128) : 128;
  E.smem = (size_t)E.max_n * E.nthr * 8;
  const int kct = chunk_template(std::min(K, kBatchChunk));
  const void* kfn = batched_kernel_ptr(kct);
  PBAT_BCUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)E.smem));
  int per_sm = 0;
  PBAT_BCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, E.nthr, E.smem));
  if (per_sm < 1) return fail(PBAT_ERANGE, "batched kernel cannot be resident");
  long long grid = (long long)per_sm * dev.sms;
  const long long need = (long long)((E.total_tasks + E.nthr / 32 - 1) / (E.nthr / 32));
  E.grid = (int)std::max(1LL, std::min(grid, need));
  BatchArrays& A = E.A;
  A.graphs = (const BatchGraphDev*)(d + E.o_graphs);
  A.bp = (const double*)(d + E.o_bp);
  A.bq = (const dd*)(d + E.o_bq);
  A.blane = (const dd*)(d + E.o_blane);
  A.bwmid = (const u128*)(d + E.o_wmid);
  A.limbs = (unsigned long long*)(d + E.o_limbs);
  A.nk = (unsigned long long*)(d + E.o_nk);
  A.counter = (unsigned long long*)(d + E.o_counter);
  A.status = (unsigned int*)(d + E.o_status);
  A.G = G;
  A.K = K;
  A.total_tasks = E.total_tasks;
  A.budget_ns = o.time_budget_s > 0 ? (unsigned long long)(o.time_budget_s * 1e9) : 0ull;
  A.prune = o.prune ? 1 : 0;
  A.max_n = E.max_n;
  return PBAT_OK;
}

// Record the launch sequence on `st` (used both for capture and as-is).
static int batch_enqueue(BatchEntry& E, cudaStream_t st) {
  char* d = (char*)E.scr->dmem;
  PBAT_BCUDA(cudaMemsetAsync(d + E.o_limbs, 0, E.d_total - E.o_limbs, st));
  const int kct = chunk_template(std::min(E.K, kBatchChunk));
  for (int k0 = 0; k0 < E.K; k0 += kBatchChunk) {
    if (k0 > 0) PBAT_BCUDA(cudaMemsetAsync(d + E.o_counter, 0, 8, st));
    PBAT_BCUDA(launch_batched(kct, E.A, k0, E.grid, E.nthr, E.smem, st));
  }
  return PBAT_OK;
}

static void batch_fill_tables(BatchEntry& E, const pbat_graph* graphs, const double* p) {
  char* h = (char*)E.scr->hmem;
  double* bp = (double*)(h + E.o_bp);
  dd* bq = (dd*)(h + E.o_bq);
  dd* blane = (dd*)(h + E.o_blane);
  u128* bw = (u128*)(h + E.o_wmid);
  const int K = E.K;
  size_t poff = 0;
  for (int i = 0; i < E.G; ++i) {
    const int m = graphs[i].n_arcs;
    const std::vector<int>& perm = E.perm[i];
    // find this network's descriptor (same ell/L for every p-vector)
    const BatchGraphDev* b = nullptr;
    for (const auto& x : E.gd)
      if (x.gidx == i) { b = &x; break; }
    for (int k = 0; k < K; ++k) {
      const double* pv = p + poff + (size_t)k * m;
      const size_t gk = (size_t)i * K + k;
      for (int j = 0; j < 64; ++j) {
        if (j < m) {
          bp[gk * 64 + j] = pv[perm[j]];
          bq[gk * 64 + j] = dd_one_minus(pv[perm[j]]);
        } else {
          bp[gk * 64 + j] = 0.0;
          bq[gk * 64 + j] = dd{0.0, 0.0};
        }
      }
      for (int j = 0; j < 32; ++j) {
        dd w = dd_make(j < (1 << b->ell) ? 1.0 : 0.0);
        if (j < (1 << b->ell))
          for (int a = 0; a < b->ell; ++a) w = dd_mul(w, arc_w(pv, perm[a], (j >> a) & 1));
        blane[gk * 32 + j] = w;
      }
      u128* tab = bw + b->wmid_off + ((size_t)k << b->L);
      for (int gi = 0; gi < (1 << b->L); ++gi) {
        dd w = dd_make(1.0);
        for (int a = 0; a < b->L; ++a) w = dd_mul(w, arc_w(pv, perm[b->ell + a], (gi >> a) & 1));
        tab[gi] = to_fixed127(w);
      }
    }
    poff += (size_t)K * m;
  }
}

// exact sum of the limbs, as a double
static double limbs_value(const unsigned long long* limbs) {
  // signed limb sums -> carry-normalised 32-bit chunks (value >= 0)
  long long carry = 0;
  uint32_t chunk[kLimbs + 2];
  for (int i = 0; i < kLimbs; ++i) {
    const __int128 v = (__int128)(long long)limbs[i] + carry;
    chunk[i] = (uint32_t)(v & 0xffffffff);
    carry = (long long)(v >> 32);
  }
  chunk[kLimbs] = (uint32_t)(carry & 0xffffffff);
  chunk[kLimbs + 1] = (uint32_t)((carry >> 32) & 0xffffffff);
  dd s = dd{0.0, 0.0};
  for (int i = kLimbs + 1; i >= 0; --i)
    s = dd_add(s, dd_make(ldexp((double)chunk[i], 32 * i - kLimbScale)));
  return s.hi + s.lo;
}

int run_batched_bs(int G, const pbat_graph* graphs, int K, const double* p, const pbat_options& o,
                   cudaStream_t st, double* R_out, uint64_t* Nk_out, const std::string& key,
                   const DeviceInfo& dev, uint64_t* kernel_ns, const std::vector<std::string>* elig,
                   double* dRdp_out, std::vector<std::pair<int, int>>* coarse);

int run_batched(int G, const pbat_graph* graphs, int K, const double* p, pbat_options* opt,
                void* stream, double* R_out, uint64_t* Nk_out, double* dRdp_out) {
  clear_error();
  if (G < 1 || G > 4096) return fail(PBAT_ERANGE, "n_graphs=%d not in [1,4096]", G);
  if (K < 1 || K > 64) return fail(PBAT_ERANGE, "n_pvec=%d not in [1,64]", K);
  if (!graphs || !p || !R_out) return fail(PBAT_EINVAL, "graphs, p and R_out must not be NULL");
  pbat_options o;
  pbat_options_init(&o);
  if (opt) o = *opt;
  int rc;
  size_t ptotal = 0;
  for (int i = 0; i < G; ++i) {
    GraphIn g{graphs[i].n_nodes, graphs[i].n_arcs, graphs[i].tail, graphs[i].head,
              graphs[i].directed, graphs[i].source, graphs[i].sink};
    if ((rc = validate_graph(g))) return fail(rc, "network %d: %s", i, last_error());
    if ((rc = validate_p(p + ptotal, K * g.m))) return fail(rc, "network %d: %s", i, last_error());
    ptotal += (size_t)K * g.m;
  }
  if ((rc = validate_options(opt, 0))) return rc;
  if (o.range_bits != 0) return fail(PBAT_EINVAL, "range_bits is not supported for batches");
  DeviceInfo dev;
  if ((rc = device_info(dev))) return rc;
  cudaStream_t st = (cudaStream_t)stream;

  std::string key = batch_key(dev.device, G, graphs, K, o);
  if (o.algo != PBAT_ALGO_FRONTIER) {
    // bit-sliced batched module: R and N_k, or with the gradient the
    // gradient module (every p-vector's exact per-arc sums from one
    // connectivity pass per state); both one persistent launch
    std::vector<double> Rb((size_t)G * K);
    std::vector<uint64_t> Nb;
    std::vector<double> Gb;
    std::vector<std::string> elig;
    std::vector<std::pair<int, int>> coarse;
    int nk_total = 0;
    size_t ptotal2 = 0;
    for (int i = 0; i < G; ++i) nk_total += graphs[i].n_arcs + 1;
    Nb.resize(nk_total);
    if (dRdp_out) {
      // an arc may be a walk arc of the gradient module only if every
      // p-vector puts its p in [2^-20, 1 - 2^-20] (its sums are divided by
      // p and 1 - p)
      elig.resize(G);
      for (int i = 0; i < G; ++i) {
        const int m = graphs[i].n_arcs;
        elig[i].assign(m, '1');
        for (int k = 0; k < K; ++k)
          for (int a = 0; a < m; ++a) {
            const double x = p[ptotal2 + (size_t)k * m + a];
            if (!(x >= 0x1p-20 && x <= 1.0 - 0x1p-20)) elig[i][a] = '0';
          }
        ptotal2 += (size_t)K * m;
        key += "grad:" + elig[i];
      }
      Gb.resize(ptotal2);
    }
    uint64_t kns = 0;
    rc = run_batched_bs(G, graphs, K, p, o, st, Rb.data(), Nb.data(), key, dev, &kns,
                        dRdp_out ? &elig : nullptr, dRdp_out ? Gb.data() : nullptr,
                        o.algo == PBAT_ALGO_AUTO ? &coarse : nullptr);
    if (rc == PBAT_OK) {
      // pairs the fixed-point bounds cannot certify: exact single runs
      std::vector<size_t> poff(G);
      for (int i = 0, acc = 0; i < G; ++i) {
        poff[i] = (size_t)acc;
        acc += K * graphs[i].n_arcs;
      }
      for (const auto& ik : coarse) {
        const int i = ik.first, k = ik.second;
        GraphIn g{graphs[i].n_nodes, graphs[i].n_arcs, graphs[i].tail, graphs[i].head,
                  graphs[i].directed, graphs[i].source, graphs[i].sink};
        pbat_options oo = o;
        oo.algo = PBAT_ALGO_FRONTIER;
        rc = run_single(g, p + poff[i] + (size_t)k * g.m, dRdp_out != nullptr, &oo, stream,
                        &Rb[(size_t)i * K + k], nullptr,
                        dRdp_out ? Gb.data() + poff[i] + (size_t)k * g.m : nullptr);
        if (rc) return rc;
      }
      memcpy(R_out, Rb.data(), sizeof(double) * Rb.size());
      if (Nk_out) memcpy(Nk_out, Nb.data(), sizeof(uint64_t) * Nb.size());
      if (dRdp_out) memcpy(dRdp_out, Gb.data(), sizeof(double) * Gb.size());
      if (opt) {
        opt->stats[4] = kns;   // device time of the batched launch
        opt->stats[5] = 1;     // one persistent kernel for every p-vector
        opt->stats[7] = 1;
      }
      return PBAT_OK;
    }
    if (rc != PBAT_ENOTSUP || o.algo == PBAT_ALGO_BITSLICE) return rc;
    clear_error();
  }
  BatchEntry* E = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_bmu);
    for (auto* e : g_batches)
      if (!e->busy && e->key == key) { e->busy = true; E = e; break; }
  }
  if (!E) {
    std::unique_ptr<BatchEntry> ne(new BatchEntry());
    ne->key = key;
    ne->busy = true;
    if ((rc = batch_build(*ne, G, graphs, K, o, dev))) {
      if (ne->scr) scratch_release(ne->scr);
      return rc;
    }
    E = ne.release();
    std::lock_guard<std::mutex> lk(g_bmu);
    g_batches.push_back(E);
  }
  auto done = [&](int code) {
    std::lock_guard<std::mutex> lk(g_bmu);
    E->busy = false;
    return code;
  };
  batch_fill_tables(*E, graphs, p);
  char* d = (char*)E->scr->dmem;
  char* h = (char*)E->scr->hmem;
  if (cudaMemcpyAsync(d, h, E->upload_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return done(fail(PBAT_ECUDA, "upload failed: %s", cudaGetErrorString(cudaGetLastError())));
  if (!E->exec) {
    // capture the reset + kernels once; replay on later calls
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
      return done(fail(PBAT_ECUDA, "stream create failed"));
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int erc = ok ? batch_enqueue(*E, cs) : PBAT_ECUDA;
    ok = (cudaStreamEndCapture(cs, &graph) == cudaSuccess) && ok && erc == PBAT_OK;
    if (ok) ok = cudaGraphInstantiate(&E->exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (!ok) {
      E->exec = nullptr;
      return done(fail(PBAT_ECUDA, "CUDA graph capture of the batched launch failed: %s",
                       cudaGetErrorString(cudaGetLastError())));
    }
  }
  if (cudaGraphLaunch(E->exec, st) != cudaSuccess)
    return done(fail(PBAT_ECUDA, "graph launch failed: %s", cudaGetErrorString(cudaGetLastError())));
  if (cudaMemcpyAsync(h + E->o_limbs, d + E->o_limbs, E->d_total - E->o_limbs,
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return done(fail(PBAT_ECUDA, "batched run failed: %s", cudaGetErrorString(cudaGetLastError())));
  if (*(unsigned int*)(h + E->o_status) & 1u)
    return done(fail(PBAT_ETIMEOUT, "time budget ran out on the device"));
  const unsigned long long* limbs = (const unsigned long long*)(h + E->o_limbs);
  const unsigned long long* nk = (const unsigned long long*)(h + E->o_nk);
  std::vector<double> Rtmp((size_t)G * K);
  for (int i = 0; i < G; ++i)
    for (int k = 0; k < K; ++k) Rtmp[(size_t)i * K + k] = limbs_value(limbs + ((size_t)i * K + k) * kLimbs);
  std::vector<uint64_t> Ntmp(nk, nk + E->nk_total);
  if (opt) {
    opt->stats[5] = (unsigned long long)((E->K + kBatchChunk - 1) / kBatchChunk);  // kernels
  }
  done(PBAT_OK);
  if (dRdp_out) {
    // gradient: one fused enumeration per (network, p-vector)
    size_t poff = 0;
    for (int i = 0; i < G; ++i) {
      GraphIn g{graphs[i].n_nodes, graphs[i].n_arcs, graphs[i].tail, graphs[i].head,
                graphs[i].directed, graphs[i].source, graphs[i].sink};
      for (int k = 0; k < K; ++k) {
        double Rk;
        pbat_options oo = o;
        rc = run_single(g, p + poff + (size_t)k * g.m, true, &oo, stream, &Rk, nullptr,
                        dRdp_out + poff + (size_t)k * g.m);
        if (rc) return rc;
      }
      poff += (size_t)K * g.m;
    }
  }
  memcpy(R_out, Rtmp.data(), sizeof(double) * Rtmp.size());
  if (Nk_out) memcpy(Nk_out, Ntmp.data(), sizeof(uint64_t) * Ntmp.size());
  return PBAT_OK;
}

}  // namespace pbat

extern "C" int pbat_reliability_batched(int n_graphs, const pbat_graph* graphs, int n_pvec,
                                        const double* p, pbat_options* opt, void* cuda_stream,
                                        double* R_out, uint64_t* Nk_out, double* dRdp_out) {
  try {
    return pbat::run_batched(n_graphs, graphs, n_pvec, p, opt, cuda_stream, R_out, Nk_out,
                             dRdp_out);
  } catch (...) {
    return pbat::fail(PBAT_ENOMEM, "host exception");
  }
}
