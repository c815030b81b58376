// pbat_engine.cu -- host side of the PBAT engine behind the C ABI.
//
// Steps of one call (the PBAT driver of arXiv 2209.09711 Sec. 5.1, laid out
// for one GPU):
//   validate  -> reject what the problem statement excludes (Sec. 2.4)
//   plan      -> choose which arcs are prefix / walk / lane arcs and how many
//                of each (STEP 0-1: the equal division of Sec. 4.3)
//   tables    -> fixed-point walk masses, lane masses, prefix masses,
//                reciprocals
//   launch    -> the bit-sliced or the frontier kernel over all work items
//                (STEP 2); the bit-sliced kernels add their block sums into
//                256-bit fixed-point results with integer atomics, the
//                frontier kernel is followed by the fixed-order reduction of
//                its block partials (STEP 3)
//   read back -> R, N_k and dR/dp in input arc order (the fused bit-sliced
//                kernel's per-arc sums become dR/dp here)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "pbat.h"
#include "pbat_engine.h"
#include "pbat_internal.h"
#include "pbat_nvtx.h"

namespace pbat {

size_t frontier_smem_bytes(int n, int m, int L, int nthr, bool grad, bool wide);
const void* frontier_kernel_ptr(bool grad, bool wide);
cudaError_t launch_frontier(bool grad, bool wide, int grid, int nthr, size_t smem,
                            cudaStream_t st, const FrontierParams& P, const u128* wmid,
                            const DevWork& W);
cudaError_t launch_reduce(cudaStream_t st, const DevWork& W, int nblocks, int n_acc, int n_cnt);

struct BsLaunch;
void bs_finish_grad(const BsLaunch& bl, const dd* acc, int m, double* g_internal);
BsLaunch* bs_new();
void bs_delete(BsLaunch* b);
void bs_precompile(const GraphIn& g, const double* p, bool grad,
                   const std::vector<pbat_options>& opts, const DeviceInfo& dev);
int bs_prepare(const GraphIn& g, const double* p, bool grad, const pbat_options& o,
               const DeviceInfo& dev, BsLaunch& bl);
cudaError_t bs_launch(const BsLaunch& bl, int grid, cudaStream_t st, const unsigned long long* d_lane,
                      const unsigned long long* d_thr, const unsigned long long* d_wmid,
                      const void* d_ptab, const void* d_ptab_ex, const DevWork& W, int phase);
const std::vector<MxHost>& bs_ptab(const BsLaunch& bl);
const std::vector<MxHost>& bs_ptab_ex(const BsLaunch& bl);
const std::vector<unsigned long long>& bs_thr_tab(const BsLaunch& bl);
bool bs_grad(const BsLaunch& bl);
const std::vector<int>& bs_perm(const BsLaunch& bl);
unsigned long long bs_items(const BsLaunch& bl);
unsigned long long bs_item_states(const BsLaunch& bl);
int bs_per_sm(const BsLaunch& bl, int phase);
int bs_nthr(const BsLaunch& bl);
const std::vector<unsigned long long>& bs_lane_tab(const BsLaunch& bl);
const std::vector<unsigned long long>& bs_wmid(const BsLaunch& bl);
void bs_describe(const BsLaunch& bl, int* out6);
int bs_source_for(const GraphIn& g, const double* p, bool grad, const pbat_options& o,
                  std::string& out);
int bsb_source_for(int G, const pbat_graph* graphs, int K, const pbat_options& o,
                   const std::vector<std::string>* elig, std::string& out);

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string t_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_last_error = buf;
  return code;
}

void clear_error() { t_last_error.clear(); }

// Host-side fault injection, for failure-detection tests: PBAT_FAULT holds a
// comma-separated list of sites -- "plan", "compile", "alloc", "launch" --
// and a listed site fails the way its real call can, with the same error
// code, before any GPU work of that step.  Nothing on the device is faulted.
bool fault_at(const char* site) {
  const char* f = getenv("PBAT_FAULT");
  if (!f || !*f) return false;
  const size_t n = strlen(site);
  for (const char* q = f; (q = strstr(q, site)) != nullptr; q += n) {
    const bool starts = q == f || q[-1] == ',';
    const bool ends = q[n] == '\0' || q[n] == ',';
    if (starts && ends) return true;
  }
  return false;
}
const char* last_error() { return t_last_error.c_str(); }

#define PBAT_CUDA(call)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(PBAT_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                  __FILE__, __LINE__);                                                    \
  } while (0)

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
int validate_graph(const GraphIn& g) {
  if (g.n > kMaxNodes) return fail(PBAT_ERANGE, "n_nodes=%d exceeds %d", g.n, kMaxNodes);
  if (g.m > kMaxArcs) return fail(PBAT_ERANGE, "n_arcs=%d exceeds %d", g.m, kMaxArcs);
  if (g.n < 2) return fail(PBAT_EINVAL, "n_nodes=%d: need at least 2 nodes", g.n);
  if (g.m < 1) return fail(PBAT_EINVAL, "n_arcs=%d: need at least 1 arc", g.m);
  if (!g.tail || !g.head) return fail(PBAT_EINVAL, "tail/head must not be NULL");
  if (g.source < 0 || g.source >= g.n || g.sink < 0 || g.sink >= g.n)
    return fail(PBAT_EINVAL, "source=%d sink=%d out of [0,%d)", g.source, g.sink, g.n);
  if (g.source == g.sink) return fail(PBAT_EINVAL, "source == sink (%d)", g.source);
  for (int k = 0; k < g.m; ++k) {
    if (g.tail[k] < 0 || g.tail[k] >= g.n || g.head[k] < 0 || g.head[k] >= g.n)
      return fail(PBAT_EINVAL, "arc %d (%d,%d) has a node id out of [0,%d)", k, g.tail[k],
                  g.head[k], g.n);
    if (g.tail[k] == g.head[k]) return fail(PBAT_EINVAL, "arc %d is a loop at node %d", k, g.tail[k]);
  }
  return PBAT_OK;
}

int validate_p(const double* p, int m) {
  if (!p) return fail(PBAT_EINVAL, "p must not be NULL");
  for (int k = 0; k < m; ++k)
    if (!(p[k] >= 0.0 && p[k] <= 1.0))
      return fail(PBAT_EINVAL, "p[%d]=%g is not in [0,1]", k, p[k]);
  return PBAT_OK;
}

int validate_options(const pbat_options* o, int m) {
  if (!o) return PBAT_OK;
  if (o->struct_size != (int)sizeof(pbat_options))
    return fail(PBAT_EINVAL, "pbat_options.struct_size=%d, expected %d (call pbat_options_init)",
                o->struct_size, (int)sizeof(pbat_options));
  if (o->algo < PBAT_ALGO_AUTO || o->algo > PBAT_ALGO_BITSLICE)
    return fail(PBAT_EINVAL, "unknown algo %d", o->algo);
  if (o->range_bits < 0 || o->range_bits > m)
    return fail(PBAT_EINVAL, "range_bits=%d not in [0,%d]", o->range_bits, m);
  if (o->range_bits > 0) {
    const uint64_t lim = (uint64_t)1 << o->range_bits;
    if (o->range_lo > o->range_hi || o->range_hi > lim)
      return fail(PBAT_EINVAL, "range [%llu,%llu) not within [0,2^%d]",
                  (unsigned long long)o->range_lo, (unsigned long long)o->range_hi, o->range_bits);
  }
  if (o->block_threads != -1 &&
      (o->block_threads < 32 || o->block_threads > 256 || o->block_threads % 32))
    return fail(PBAT_EINVAL, "block_threads=%d must be -1 or a multiple of 32 in [32,256]",
                o->block_threads);
  if (o->prune < 0 || o->prune > 2) return fail(PBAT_EINVAL, "prune=%d not in {0,1,2}", o->prune);
  if (o->occupancy < -1 || o->occupancy > 8)
    return fail(PBAT_EINVAL, "occupancy=%d not in [-1,8]", o->occupancy);
  if (o->launches < 0 || o->launches > 2)
    return fail(PBAT_EINVAL, "launches=%d not in {0,1,2}", o->launches);
  if (!(o->time_budget_s >= 0.0)) return fail(PBAT_EINVAL, "time_budget_s must be >= 0");
  return PBAT_OK;
}

// ---------------------------------------------------------------------------
// fixed point and double-double helpers (host)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------
static bool walk_ok(double p) {  // the gradient divides walk masses by p and 1 - p
  return p >= 0x1p-20 && p <= 1.0 - 0x1p-20;
}

int make_plan(const GraphIn& g, const double* p, bool grad, const pbat_options& o,
              const DeviceInfo& dev, Plan& pl) {
  if (fault_at("plan")) return fail(PBAT_EINVAL, "injected fault: planning");
  const int m = g.m;
  const int r = o.range_bits;
  pl.grad = grad;
  pl.range_bits = r;
  pl.ell = std::min(kMaxLaneBits, m - r);
  const int free_bits = m - r - pl.ell;
  const int lmax = grad ? kMaxWalkBitsGrad : kMaxWalkBitsR;
  // enough work items to keep every warp of the persistent grid busy
  int want_items_log2 = 14;
  if (o.walk_bits >= 0) {
    pl.L = std::min(o.walk_bits, std::min(lmax, free_bits));
  } else if (o.prefix_bits >= 0) {
    const int d = std::max(o.prefix_bits, r);
    pl.L = std::max(0, std::min(lmax, m - pl.ell - d));
  } else {
    const int extra_prefix = std::max(0, want_items_log2 - r);
    pl.L = std::max(0, std::min(lmax, free_bits - extra_prefix));
  }
  pl.d = m - pl.ell - pl.L;
  // Internal arc order: internal position k holds input arc m-1-k, so the
  // state word equals the paper's state index (x_1 most significant, Eq. 2)
  // and the first range_bits input arcs are the top prefix bits.
  pl.perm.resize(m);
  for (int k = 0; k < m; ++k) pl.perm[k] = m - 1 - k;
  if (grad) {
    // walk arcs need p strictly inside (0, 1); swap offenders with a lane or
    // a free prefix arc
    const int w0 = pl.ell, w1 = pl.ell + pl.L;
    const int swap_hi = m - r;  // prefix positions [w1, m - r) are not range-fixed
    for (int k = w0; k < w1; ++k) {
      if (walk_ok(p[pl.perm[k]])) continue;
      int found = -1;
      for (int c = 0; c < swap_hi && found < 0; ++c) {
        if (c >= w0 && c < w1) continue;
        if (walk_ok(p[pl.perm[c]])) found = c;
      }
      if (found < 0) {
        // shrink the walk: move this arc's slot to the prefix side
        pl.L = k - w0;
        pl.d = m - pl.ell - pl.L;
        break;
      }
      std::swap(pl.perm[k], pl.perm[found]);
    }
  }
  uint64_t lo = 0, hi = (uint64_t)1 << pl.d;
  if (r > 0) {
    lo = o.range_lo << (pl.d - r);
    hi = o.range_hi << (pl.d - r);
  }
  if (pl.d >= 64) return fail(PBAT_ERANGE, "prefix of %d bits is too deep", pl.d);
  pl.task_lo = lo;
  pl.n_tasks = hi - lo;
  pl.wide = g.n > 32;
  pl.nthr = o.block_threads > 0 ? o.block_threads : 128;
  pl.smem = frontier_smem_bytes(g.n, m, pl.L, pl.nthr, grad, pl.wide);
  if (pl.smem > (size_t)dev.smem_optin)
    return fail(PBAT_ERANGE, "shared memory %zu B exceeds %d B (lower walk_bits)", pl.smem,
                dev.smem_optin);
  pl.prune = o.prune ? 1 : 0;
  return PBAT_OK;
}

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------

void build_params(const GraphIn& g, const double* p, const Plan& pl, const pbat_options& o,
                  FrontierParams& P, std::vector<u128>& wmid) {
  memset(&P, 0, sizeof P);
  const int m = g.m;
  P.n = g.n;
  P.m = m;
  P.directed = g.directed ? 1 : 0;
  P.source = g.source;
  P.sink = g.sink;
  P.lane_bits = pl.ell;
  P.walk_bits = pl.L;
  P.prefix_bits = pl.d;
  P.prune = pl.prune;
  P.task_lo = pl.task_lo;
  P.n_tasks = pl.n_tasks;
  P.budget_ns = o.time_budget_s > 0 ? (unsigned long long)(o.time_budget_s * 1e9) : 0ull;
  P.free_mask = pl.ell + pl.L >= 64 ? ~0ull : ((1ull << (pl.ell + pl.L)) - 1ull);
  for (int k = 0; k < m; ++k) {
    const int a = pl.perm[k];
    P.au[k] = (unsigned char)g.tail[a];
    P.av[k] = (unsigned char)g.head[a];
    P.p[k] = p[a];
    P.q[k] = dd_one_minus(p[a]);
    if (k >= pl.ell && k < pl.ell + pl.L) {
      P.inv_p[k] = dd_recip(p[a]);
      P.inv_q[k] = dd_recip_dd(P.q[k]);
    }
  }
  for (int k = 0; k < m; ++k) {
    unsigned long long gm = 0;
    const int a = pl.perm[k];
    for (int j = 0; j < m; ++j) {
      const int b = pl.perm[j];
      const bool same = g.directed ? (g.tail[a] == g.tail[b] && g.head[a] == g.head[b])
                                   : ((g.tail[a] == g.tail[b] && g.head[a] == g.head[b]) ||
                                      (g.tail[a] == g.head[b] && g.head[a] == g.tail[b]));
      if (same) gm |= 1ull << j;
    }
    P.grp[k] = gm;
  }
  const int nl = 1 << pl.ell;
  for (int j = 0; j < 32; ++j) {
    if (j >= nl) {
      P.lane_w[j] = dd{0.0, 0.0};
      for (int i = 0; i < kMaxLaneBits; ++i) P.lane_w_ex[i][j] = dd{0.0, 0.0};
      continue;
    }
    dd w = dd_make(1.0);
    for (int i = 0; i < pl.ell; ++i) w = dd_mul(w, arc_w(p, pl.perm[i], (j >> i) & 1));
    P.lane_w[j] = w;
    for (int x = 0; x < pl.ell; ++x) {
      dd we = dd_make(1.0);
      for (int i = 0; i < pl.ell; ++i)
        if (i != x) we = dd_mul(we, arc_w(p, pl.perm[i], (j >> i) & 1));
      P.lane_w_ex[x][j] = we;
    }
  }
  for (int j = 0; j < 64; ++j) P.binom[j] = binom_u64(pl.ell + pl.L, j);
  const int nW = 1 << pl.L;
  wmid.resize(nW);
  for (int gi = 0; gi < nW; ++gi) {
    dd w = dd_make(1.0);
    for (int b = 0; b < pl.L; ++b) w = dd_mul(w, arc_w(p, pl.perm[pl.ell + b], (gi >> b) & 1));
    wmid[gi] = to_fixed127(w);
  }
}

// ---------------------------------------------------------------------------
// device info and scratch pool
// ---------------------------------------------------------------------------
static std::mutex g_mu;
static std::vector<DeviceInfo> g_dev;

int device_info(DeviceInfo& out) {
  int d = 0;
  PBAT_CUDA(cudaGetDevice(&d));
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& x : g_dev)
    if (x.device == d) {
      out = x;
      return PBAT_OK;
    }
  DeviceInfo di;
  di.device = d;
  PBAT_CUDA(cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, d));
  PBAT_CUDA(cudaDeviceGetAttribute(&di.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d));
  PBAT_CUDA(cudaDeviceGetAttribute(&di.cc_major, cudaDevAttrComputeCapabilityMajor, d));
  PBAT_CUDA(cudaDeviceGetAttribute(&di.cc_minor, cudaDevAttrComputeCapabilityMinor, d));
  g_dev.push_back(di);
  out = di;
  return PBAT_OK;
}

static std::vector<Scratch*> g_pool;

int scratch_acquire(int device, size_t dbytes, size_t hbytes, Scratch** out) {
  if (fault_at("alloc")) return fail(PBAT_ENOMEM, "injected fault: device scratch allocation");
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto* s : g_pool) {
      if (!s->busy && s->device == device && s->dbytes >= dbytes && s->hbytes >= hbytes) {
        s->busy = true;
        *out = s;
        return PBAT_OK;
      }
    }
  }
  auto* s = new Scratch();
  s->device = device;
  s->dbytes = std::max<size_t>(dbytes, 1 << 20);
  s->hbytes = std::max<size_t>(hbytes, 1 << 16);
  if (cudaMalloc(&s->dmem, s->dbytes) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return fail(PBAT_ENOMEM, "cudaMalloc of %zu B failed", dbytes);
  }
  if (cudaMallocHost(&s->hmem, s->hbytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->dmem);
    delete s;
    return fail(PBAT_ENOMEM, "cudaMallocHost of %zu B failed", hbytes);
  }
  s->busy = true;
  std::lock_guard<std::mutex> lk(g_mu);
  g_pool.push_back(s);
  *out = s;
  return PBAT_OK;
}

void scratch_release(Scratch* s) {
  if (!s) return;
  std::lock_guard<std::mutex> lk(g_mu);
  s->busy = false;
}

// ---------------------------------------------------------------------------
// one planned enumeration (single network)
// ---------------------------------------------------------------------------
struct Job {
  GraphIn g;
  Plan pl;
  FrontierParams P;
  DeviceInfo dev;
  Scratch* scr = nullptr;
  int grid = 0;
  int n_acc = 0;   // accumulated sums: R, then per arc one (frontier) or two (fused bit-sliced)
  size_t reset_bytes = 64;
  unsigned long long* h_limbs = nullptr;
  char* h_region = nullptr;   // host mirror of the device result region
  DevWork W{};
  u128* d_wmid = nullptr;
  // host mirror in pinned memory
  dd* h_acc = nullptr;
  unsigned long long* h_n = nullptr;
  unsigned int* h_status = nullptr;
  unsigned long long* h_stats = nullptr;
  void* wmid_host_staging = nullptr;
  size_t wmid_bytes = 0;
  // CUDA events around the enumeration kernel of every execute since the
  // last read (so a caller can time many launches and read once)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs;
  size_t n_pending = 0;
  // bit-sliced kernel (R and N_k); null for the frontier kernel
  BsLaunch* bs = nullptr;
  unsigned long long* d_lane = nullptr;
  unsigned long long* d_thr = nullptr;
  unsigned long long* d_wmid64 = nullptr;
  void* d_ptab = nullptr;
  void* d_ptabx = nullptr;
  // absolute error bounds of R and of each dR/dp_k, in units of the
  // enumerated probability mass (the rounding of the fixed-point tables)
  double abs_err_bound = 0.0;
  double grad_err_bound = 0.0;
  double mass = 1.0;           // probability mass of the enumerated states
  std::vector<int> perm;       // internal arc position -> input arc
  unsigned long long item_states = 0, n_items = 0;
  int grid_nthr = 128;
  // two launches per enumeration: the first resolves what the prune can and
  // defers the items left to walk, the second walks them (bit-sliced kernels
  // with the prune on and many items)
  bool two_phase = false;
  int grid1 = 0, grid2 = 0;   // grids of the two launches
  // the inputs, kept to re-run the exact frontier kernel when R is too small
  // for the bit-sliced kernel's fixed-point error bound
  std::vector<int32_t> tail_copy, head_copy;
  std::vector<double> p_copy;
  pbat_options opt_copy;
};

static size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }

// Probability mass of the states an enumeration covers: 1 for the whole
// space, else the mass of the prefixes [range_lo, range_hi) of the first
// range_bits input arcs (a digit-by-digit sum, O(range_bits)).
double range_mass(int m, const double* p, const pbat_options& o) {
  (void)m;
  if (o.range_bits <= 0) return 1.0;
  const int r = o.range_bits;
  auto below = [&](unsigned long long x) {  // mass of prefixes < x (x <= 2^r)
    if (x >= (1ull << r)) return 1.0L;
    long double acc = 0.0L, run = 1.0L;
    for (int i = 0; i < r; ++i) {  // input arc i is bit r-1-i of the prefix
      const int bit = (int)((x >> (r - 1 - i)) & 1ull);
      if (bit) acc += run * (1.0L - (long double)p[i]);
      run *= bit ? (long double)p[i] : 1.0L - (long double)p[i];
    }
    return acc;
  };
  return (double)(below(o.range_hi) - below(o.range_lo));
}

int job_create(const GraphIn& g, const double* p, bool grad, pbat_options* opt, Job** out);
int job_upload(Job* J, cudaStream_t st);
int job_launch(Job* J, cudaStream_t st);
void job_destroy(Job* J);

// ---------------------------------------------------------------------------
// autotuner: planning mode, walk length L, block shape and occupancy of the
// bit-sliced kernel
// ---------------------------------------------------------------------------
// Candidates are timed on the real problem (CUDA events around the kernel,
// best of two launches) and the fastest is kept per network structure, mode
// and range -- in memory, and in the file named by PBAT_AUTOTUNE_CACHE if
// that is set ("key walk_bits block_threads prune occupancy launches" lines).  Only
// problems of at least 2^26 states are tuned: below that a launch is too
// short for the choice to matter.
struct TuneChoice {
  int L, nt, prune, occ, launches;
};
static std::mutex g_tune_mu;
static std::map<std::string, TuneChoice> g_tune;
static bool g_tune_loaded = false;

static std::string tune_key(const GraphIn& g, bool grad, const pbat_options& o, int device) {
  char head[180];
  snprintf(head, sizeof head, "d%d:g%d:n%d:m%d:dir%d:s%d:t%d:r%d:%llx:%llx:pr%d:oc%d:", device,
           grad ? 1 : 0, g.n, g.m, g.directed ? 1 : 0, g.source, g.sink, o.range_bits,
           (unsigned long long)o.range_lo, (unsigned long long)o.range_hi, o.prune,
           o.occupancy * 4 + o.launches);
  std::string k = head;
  for (int i = 0; i < g.m; ++i) {
    char e[24];
    snprintf(e, sizeof e, "%d-%d,", g.tail[i], g.head[i]);
    k += e;
  }
  return k;
}

static void tune_load_file() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("PBAT_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[4400];
  while (fgets(line, sizeof line, f)) {
    char key[4096];
    TuneChoice c{-1, 128, 1, 0, 1};
    if (sscanf(line, "%4095s %d %d %d %d %d", key, &c.L, &c.nt, &c.prune, &c.occ, &c.launches) == 6)
      g_tune[key] = c;
  }
  fclose(f);
}

static void tune_store_file(const std::string& key, const TuneChoice& c) {
  const char* path = getenv("PBAT_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), c.L, c.nt, c.prune, c.occ, c.launches);
  fclose(f);
}

static double log2_states(const GraphIn& g, const pbat_options& o) {
  double s = g.m;
  if (o.range_bits > 0) {
    const double frac = (double)(o.range_hi - o.range_lo) / ldexp(1.0, o.range_bits);
    s += frac > 0 ? log2(frac) : -1e9;
  }
  return s;
}

// Kernel time of one candidate (ms, best of two launches after its first),
// or a negative value if it cannot run.
static double tune_time(const GraphIn& g, const double* p, bool grad, pbat_options t,
                        cudaStream_t st) {
  t.autotune = 0;
  t.time_budget_s = 0;
  Job* J = nullptr;
  if (job_create(g, p, grad, &t, &J) != PBAT_OK) {
    clear_error();
    return -1.0;
  }
  double ms = 1e300;
  bool ok = !job_upload(J, st);
  for (int rep = 0; ok && rep < 3; ++rep) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    ok = !job_launch(J, st);
    cudaEventRecord(b, st);
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    float f = 0.f;
    if (ok && cudaEventElapsedTime(&f, a, b) == cudaSuccess && rep > 0) ms = std::min(ms, (double)f);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  job_destroy(J);
  if (!ok) {
    cudaGetLastError();
    clear_error();
    return -1.0;
  }
  return ms;
}

// Fill o.walk_bits / o.block_threads / o.prune / o.occupancy with the tuned
// choice when tuning applies.  Two stages: (1) with the prune on, the
// planning mode -- source/sink-near prefix arcs against prune-aware prefix
// arcs (prune = 2) -- at the planner's default shape, since the mode changes
// how many items the prune resolves and so the best shape; (2) walk length,
// block size and occupancy within the chosen mode.  Every choice gives the
// same exact results.
static int autotune(const GraphIn& g, const double* p, bool grad, pbat_options& o,
                    const DeviceInfo& dev) {
  if (!o.autotune || o.walk_bits >= 0 || o.block_threads > 0 || o.prefix_bits >= 0) return PBAT_OK;
  if (o.algo == PBAT_ALGO_FRONTIER || log2_states(g, o) < 26.0) return PBAT_OK;
  const std::string key = tune_key(g, grad, o, dev.device);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_file();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      o.walk_bits = it->second.L;
      o.block_threads = it->second.nt;
      o.prune = it->second.prune;
      o.occupancy = it->second.occ;
      o.launches = it->second.launches;
      return PBAT_OK;
    }
  }
  NvtxRange nv("pbat autotune");
  cudaStream_t st;
  PBAT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  // stage 1: planning mode
  int mode = o.prune;
  if (o.prune == 1) {
    pbat_options a = o, b = o;
    b.prune = 2;
    bs_precompile(g, p, grad, {a, b}, dev);
    const double ta = tune_time(g, p, grad, a, st), tb = tune_time(g, p, grad, b, st);
    if (tb > 0 && (ta < 0 || tb < ta)) mode = 2;
  }
  // stage 2: walk length x block size x occupancy x launches.  Candidates run the whole
  // problem: a block of the equal division is not a fair sample (which arcs
  // its range fixes changes how much the prune removes; the first block of
  // the 40-arc network favoured a shape 50% slower on the whole).  Large
  // problems try fewer candidates: long walks, no 64-thread blocks.
  const int lmax = std::min(10, std::max(0, g.m - o.range_bits - 10));
  const bool large = log2_states(g, o) > 34.0;
  std::vector<int> Ls, nts, occs;
  for (int L = std::max(0, lmax - (large ? 2 : 6)); L <= lmax; ++L) Ls.push_back(L);
  // warps per block need not be a power of two: on the 40-arc network 160
  // threads (3 blocks, 15 warps per SM) ran the fused kernel 12% faster
  // than 128 and 224 threads the R kernel 7% faster than 256
  if (!large) nts.push_back(64), nts.push_back(96);
  for (int nt : {128, 160, 192, 224, 256}) nts.push_back(nt);
  // a register cap of two blocks per SM: on GB300 the fused kernel of the
  // 40-arc network in prune-aware mode went from 26.0 to 24.7 ms with it
  if (o.occupancy >= 0) occs.push_back(o.occupancy);
  else occs = {0, 2};
  // one launch or two (with the prune on): the deferral pays where walked
  // items are long and few, or where the prune resolves nearly every item
  std::vector<int> launch_modes;
  if (o.launches) launch_modes.push_back(o.launches);
  else if (mode) launch_modes = {1, 2};
  else launch_modes.push_back(1);
  std::vector<pbat_options> cands;
  for (int L : Ls)
    for (int nt : nts)
      for (int oc : occs)
        for (int nl : launch_modes) {
          if (oc * nt > 2048) continue;
          pbat_options t = o;
          t.prune = mode;
          t.walk_bits = L;
          t.block_threads = nt;
          t.occupancy = oc;
          t.launches = nl;
          cands.push_back(t);
        }
  bs_precompile(g, p, grad, cands, dev);
  double best_ms = 1e300;
  TuneChoice best{-1, 128, mode, 0, 1};
  for (const pbat_options& t : cands) {
    const double ms = tune_time(g, p, grad, t, st);
    if (ms > 0 && ms < best_ms)
      best_ms = ms, best = TuneChoice{t.walk_bits, t.block_threads, t.prune, t.occupancy, t.launches};
  }
  cudaStreamDestroy(st);
  if (best.L < 0) return PBAT_OK;  // keep the planner's defaults
  o.walk_bits = best.L;
  o.block_threads = best.nt;
  o.prune = best.prune;
  o.occupancy = best.occ;
  o.launches = best.launches;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  tune_store_file(key, best);
  return PBAT_OK;
}

int job_create(const GraphIn& g, const double* p, bool grad, pbat_options* opt, Job** out) {
  NvtxRange nv("pbat plan and tables");
  pbat_options o;
  pbat_options_init(&o);
  if (opt) o = *opt;
  int rc;
  if ((rc = validate_graph(g))) return rc;
  if ((rc = validate_p(p, g.m))) return rc;
  if ((rc = validate_options(opt, g.m))) return rc;
  {
    DeviceInfo dv;
    if ((rc = device_info(dv))) return rc;
    if ((rc = autotune(g, p, grad, o, dv))) return rc;
  }
  const bool use_bs = o.algo == PBAT_ALGO_BITSLICE || o.algo == PBAT_ALGO_AUTO;
  // job_destroy also frees the bit-sliced launch if a later step fails
  std::unique_ptr<Job, void (*)(Job*)> J(new Job(), job_destroy);
  J->g = g;
  J->tail_copy.assign(g.tail, g.tail + g.m);
  J->head_copy.assign(g.head, g.head + g.m);
  J->g.tail = J->tail_copy.data();
  J->g.head = J->head_copy.data();
  J->p_copy.assign(p, p + g.m);
  J->opt_copy = o;
  J->mass = range_mass(g.m, p, o);
  if ((rc = device_info(J->dev))) return rc;
  std::vector<u128> wmid;
  int per_sm = 0, nthr = 128;
  unsigned long long n_items = 0;
  if (use_bs) {
    J->bs = bs_new();
    if ((rc = bs_prepare(g, p, grad, o, J->dev, *J->bs))) return rc;
    J->perm = bs_perm(*J->bs);
    per_sm = bs_per_sm(*J->bs, 0);
    nthr = bs_nthr(*J->bs);
    n_items = bs_items(*J->bs);
    J->item_states = bs_item_states(*J->bs);
    int d6[6];
    bs_describe(*J->bs, d6);
    // Per item, R is the sum over threads of thread mass x T (T: lane sums
    // times walk masses, summed over the walk) times the prefix mass.  Its
    // absolute error in units of the item's mass: the four byte-table
    // entries of a lane sum, each within 2^-63, give 2^-61; the 32 thread
    // masses, each within 2^-64 of exact and weighting a T <= 1, give 2^-59;
    // the R kernel's 64-bit walk masses, each within 2^-64, give 2^(L-64)
    // over 2^L walk states (the fused kernel's are 128-bit: negligible).
    // The prefix masses are relative (2^-62 per level): harmless at 1e-12.
    J->abs_err_bound = ldexp(1.0, -61) + ldexp(1.0, -59) + (grad ? 0.0 : ldexp(1.0, d6[2] - 64));
    // dR/dp_k of the fused kernel: the same two absolute terms for the
    // walk-arc sums A and B (whose terms all carry the arc's own factor, so
    // dividing by p or 1 - p does not amplify them) and the excluded-arc
    // tables of lane and thread arcs (2^-64 each, summed over 16 pairs with
    // weights summing to at most one): 2^-57 covers every role
    J->grad_err_bound = grad ? ldexp(1.0, -57) : 0.0;
    J->pl.grad = grad;
  } else {
    if ((rc = make_plan(g, p, grad, o, J->dev, J->pl))) return rc;
    build_params(g, p, J->pl, o, J->P, wmid);
    J->perm = J->pl.perm;
    const void* kfn = frontier_kernel_ptr(grad, J->pl.wide);
    PBAT_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)J->pl.smem));
    PBAT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, J->pl.nthr, J->pl.smem));
    if (per_sm < 1)
      return fail(PBAT_ERANGE, "frontier kernel cannot be resident (smem %zu B)", J->pl.smem);
    nthr = J->pl.nthr;
    n_items = J->pl.n_tasks;
    J->item_states = 1ull << (J->pl.ell + J->pl.L);
    J->abs_err_bound = ldexp(1.0, -100);
    J->grad_err_bound = ldexp(1.0, -98);
  }
  J->n_items = n_items;
  J->grid_nthr = nthr;
  // Deferring the walked items to a second launch lets the whole grid share
  // them at the end instead of meeting them in ticket order: with the
  // prune-aware plan of the 40-arc network 9% of the items are walked, each
  // about 10^5 instructions per warp, spread over the whole ticket range, so
  // the last ones otherwise start late (fused kernel on GB300: 22.7 -> 20.8
  // ms at the best shapes).  The first launch visits the items with a fixed
  // warp stride and appends deferred items 32 at a time.  The R kernel's
  // items are shorter and it stays faster in one launch (7.7 against 8.0
  // ms), so by default only the fused kernel defers; opt.launches (or the
  // autotuner) chooses otherwise.  Small item counts keep one launch by
  // default (the second costs a launch latency).
  const bool can_two = J->bs && o.prune && n_items <= (1ull << 24);
  J->two_phase = can_two && (o.launches == 2 ||
                             (o.launches == 0 && grad && n_items >= (1ull << 18)));
  // the list has a slot for every item (at most 128 MiB), so it never fills
  const unsigned long long list_cap = J->two_phase ? n_items : 0;
  const long long warps_per_block = nthr / 32;
  long long grid = (long long)per_sm * J->dev.sms;
  // never more warps than work items
  const long long need = ((long long)std::min<unsigned long long>(n_items, 1ull << 40) +
                          warps_per_block - 1) / warps_per_block;
  grid = std::max(1LL, std::min(grid, need));
  J->grid = (int)grid;
  if (J->bs) {
    // the two launches of a two-launch run fill the GPU at their own occupancy
    J->grid1 = (int)std::max(1LL, std::min((long long)bs_per_sm(*J->bs, 1) * J->dev.sms, need));
    J->grid2 = (int)std::max(1LL, std::min((long long)bs_per_sm(*J->bs, 2) * J->dev.sms, need));
  }
  const int m = g.m;
  // accumulators per block: the frontier kernel and the bit-sliced R kernel
  // write R and one value per arc (zeros for R only) or R alone; the fused
  // bit-sliced kernel writes R and two sums per arc
  J->n_acc = J->bs ? (bs_grad(*J->bs) ? 1 + 2 * m : 1) : 1 + m;
  const int n_acc = J->n_acc;

  // device scratch layout
  size_t off = 0;
  // counter, status, stats and the results sit together: one memset per launch
  const size_t o_counter = off; off = up16(off + 8);
  const size_t o_status = off; off = up16(off + 4);
  const size_t o_stats = off; off = up16(off + 3 * 8);
  const size_t o_list_n = off; off = up16(off + 8);     // deferred-item count and ticket
  const size_t o_counter2 = off; off = up16(off + 8);
  const size_t o_out_n = off; off = up16(off + (size_t)(m + 1) * 8);
  const size_t limbs_bytes = J->bs ? (size_t)n_acc * 8 * 8 : 0;
  const size_t o_out_limbs = off; off = up16(off + limbs_bytes);
  J->reset_bytes = off;
  // the frontier kernel: per-block partials and the fixed-order reduction
  const size_t part_bytes = J->bs ? 0 : (size_t)grid * n_acc * sizeof(dd);
  const size_t o_part_acc = off; off = up16(off + part_bytes);
  const size_t o_part_n = off; off = up16(off + (J->bs ? 0 : (size_t)grid * (m + 1) * 8));
  const size_t o_out_acc = off; off = up16(off + (size_t)n_acc * sizeof(dd));
  // per-warp slots of every block of the largest of the launches' grids
  const long long grid_max = std::max<long long>(grid, std::max(J->grid1, J->grid2));
  const size_t wacc_bytes =
      (J->bs && bs_grad(*J->bs)) ? (size_t)grid_max * (nthr / 32) * (1 + 2 * m) * 24 : 0;
  const size_t o_wacc = off; off = up16(off + wacc_bytes);
  const size_t o_wmid = off; off = up16(off + wmid.size() * sizeof(u128));
  size_t o_lane = 0, o_thr = 0, o_wmid64 = 0, o_ptab = 0, o_ptabx = 0, o_tab_end = 0;
  if (J->bs) {
    o_lane = off; off = up16(off + bs_lane_tab(*J->bs).size() * 8);
    o_thr = off; off = up16(off + bs_thr_tab(*J->bs).size() * 8);
    o_wmid64 = off; off = up16(off + bs_wmid(*J->bs).size() * 8);
    o_ptab = off; off = up16(off + bs_ptab(*J->bs).size() * sizeof(MxHost));
    o_ptabx = off; off = up16(off + bs_ptab_ex(*J->bs).size() * sizeof(MxHost));
    o_tab_end = off;
  }
  const size_t o_list = off; off = up16(off + (size_t)list_cap * 8);
  const size_t dbytes = off;
  // host (pinned) layout: results + staging of the walk table
  // the first reset_bytes mirror the device's result region (one copy back)
  size_t hoff = 0;
  const size_t h_region = hoff; hoff = up16(hoff + J->reset_bytes);
  const size_t h_status = h_region + o_status, h_stats = h_region + o_stats;
  const size_t h_n = h_region + o_out_n, h_limbs = h_region + o_out_limbs;
  const size_t h_acc = hoff; hoff = up16(hoff + (size_t)n_acc * sizeof(dd));
  const size_t h_wmid = hoff; hoff = up16(hoff + wmid.size() * sizeof(u128));
  size_t h_lane = 0;
  if (J->bs) {
    h_lane = hoff;
    hoff = up16(hoff + (o_tab_end - o_lane));  // same layout as the device tables
  }
  const size_t hbytes = hoff;
  if ((rc = scratch_acquire(J->dev.device, dbytes, hbytes, &J->scr))) return rc;
  char* d = (char*)J->scr->dmem;
  char* h = (char*)J->scr->hmem;
  J->W.counter = (unsigned long long*)(d + o_counter);
  J->W.status = (unsigned int*)(d + o_status);
  J->W.stats = (unsigned long long*)(d + o_stats);
  J->W.part_acc = (dd*)(d + o_part_acc);
  J->W.part_n = (unsigned long long*)(d + o_part_n);
  J->W.out_acc = (dd*)(d + o_out_acc);
  J->W.out_n = (unsigned long long*)(d + o_out_n);
  J->W.out_limbs = limbs_bytes ? (unsigned long long*)(d + o_out_limbs) : nullptr;
  J->W.wacc = wacc_bytes ? (void*)(d + o_wacc) : nullptr;
  J->W.list = list_cap ? (unsigned long long*)(d + o_list) : nullptr;
  J->W.list_cap = list_cap;
  J->W.list_n = (unsigned long long*)(d + o_list_n);
  J->W.counter2 = (unsigned long long*)(d + o_counter2);
  J->d_wmid = (u128*)(d + o_wmid);
  J->h_region = h + h_region;
  J->h_acc = (dd*)(h + h_acc);
  J->h_limbs = (unsigned long long*)(h + h_limbs);
  J->h_n = (unsigned long long*)(h + h_n);
  J->h_status = (unsigned int*)(h + h_status);
  J->h_stats = (unsigned long long*)(h + h_stats);
  memcpy(h + h_wmid, wmid.data(), wmid.size() * sizeof(u128));
  J->wmid_host_staging = h + h_wmid;
  J->wmid_bytes = wmid.size() * sizeof(u128);
  if (J->bs) {
    // one contiguous upload: lane tables then the walk table
    const auto& lt = bs_lane_tab(*J->bs);
    const auto& tt = bs_thr_tab(*J->bs);
    const auto& wm = bs_wmid(*J->bs);
    const auto& pt = bs_ptab(*J->bs);
    const auto& px = bs_ptab_ex(*J->bs);
    char* hb = h + h_lane - o_lane;  // host mirror of the device table block
    memcpy(hb + o_lane, lt.data(), lt.size() * 8);
    if (!tt.empty()) memcpy(hb + o_thr, tt.data(), tt.size() * 8);
    memcpy(hb + o_wmid64, wm.data(), wm.size() * 8);
    memcpy(hb + o_ptab, pt.data(), pt.size() * sizeof(MxHost));
    if (!px.empty()) memcpy(hb + o_ptabx, px.data(), px.size() * sizeof(MxHost));
    J->d_lane = (unsigned long long*)(d + o_lane);
    J->d_thr = (unsigned long long*)(d + o_thr);
    J->d_wmid64 = (unsigned long long*)(d + o_wmid64);
    J->d_ptab = (void*)(d + o_ptab);
    J->d_ptabx = (void*)(d + o_ptabx);
    J->wmid_host_staging = h + h_lane;
    J->wmid_bytes = o_tab_end - o_lane;
    J->d_wmid = (u128*)(d + o_lane);  // upload destination
  }
  *out = J.release();
  return PBAT_OK;
}

// Upload the walk table (host -> device, on the stream).
int job_upload(Job* J, cudaStream_t st) {
  PBAT_CUDA(cudaMemcpyAsync(J->d_wmid, J->wmid_host_staging, J->wmid_bytes,
                            cudaMemcpyHostToDevice, st));
  return PBAT_OK;
}

// Timing event pairs are pooled per device: a one-shot call would otherwise
// create and destroy two events every time.
static std::mutex g_ev_mu;
static std::map<int, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> g_ev_pool;

static int event_pair_acquire(int device, std::pair<cudaEvent_t, cudaEvent_t>* out) {
  {
    std::lock_guard<std::mutex> lk(g_ev_mu);
    auto& v = g_ev_pool[device];
    if (!v.empty()) {
      *out = v.back();
      v.pop_back();
      return PBAT_OK;
    }
  }
  cudaEvent_t a, b;
  PBAT_CUDA(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return fail(PBAT_ECUDA, "cudaEventCreate failed");
  }
  *out = {a, b};
  return PBAT_OK;
}

static void event_pairs_release(int device, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& evs) {
  std::lock_guard<std::mutex> lk(g_ev_mu);
  auto& v = g_ev_pool[device];
  for (auto& e : evs) v.push_back(e);
  evs.clear();
}

// Launch the enumeration (and, for the frontier kernel, the reduction);
// asynchronous.
int job_launch(Job* J, cudaStream_t st) {
  NvtxRange nv("pbat launch");
  if (fault_at("launch")) return fail(PBAT_ECUDA, "injected fault: kernel launch");
  PBAT_CUDA(cudaMemsetAsync(J->W.counter, 0, J->reset_bytes, st));  // counter, status, stats, results
  const bool timed = J->n_pending < 65536;
  if (timed && J->n_pending == J->evs.size()) {
    std::pair<cudaEvent_t, cudaEvent_t> e;
    const int rc = event_pair_acquire(J->dev.device, &e);
    if (rc) return rc;
    J->evs.push_back(e);
  }
  if (timed) PBAT_CUDA(cudaEventRecord(J->evs[J->n_pending].first, st));
  if (J->bs && !J->two_phase) {
    PBAT_CUDA(bs_launch(*J->bs, J->grid, st, J->d_lane, J->d_thr, J->d_wmid64, J->d_ptab,
                        J->d_ptabx, J->W, 0));
  } else if (J->bs) {
    PBAT_CUDA(bs_launch(*J->bs, J->grid1, st, J->d_lane, J->d_thr, J->d_wmid64, J->d_ptab,
                        J->d_ptabx, J->W, 1));
    PBAT_CUDA(bs_launch(*J->bs, J->grid2, st, J->d_lane, J->d_thr, J->d_wmid64, J->d_ptab,
                        J->d_ptabx, J->W, 2));
  }
  else
    PBAT_CUDA(launch_frontier(J->pl.grad, J->pl.wide, J->grid, J->pl.nthr, J->pl.smem, st, J->P,
                              J->d_wmid, J->W));
  if (timed) {
    PBAT_CUDA(cudaEventRecord(J->evs[J->n_pending].second, st));
    ++J->n_pending;
  }
  if (!J->bs) PBAT_CUDA(launch_reduce(st, J->W, J->grid, J->n_acc, J->g.m + 1));
  return PBAT_OK;
}

void job_destroy(Job* J);

// Copy results to the host and wait; convert to input arc order.
int job_read(Job* J, cudaStream_t st, double* R_out, uint64_t* Nk_out, double* dRdp_out,
             pbat_options* opt) {
  NvtxRange nv("pbat read");
  const int m = J->g.m;
  // one copy of counter, status, statistics, N_k and (bit-sliced) the
  // fixed-point results; the frontier kernel's sums come from the reduce
  if (!J->bs)
    PBAT_CUDA(cudaMemcpyAsync(J->h_acc, J->W.out_acc, (size_t)J->n_acc * sizeof(dd),
                              cudaMemcpyDeviceToHost, st));
  PBAT_CUDA(cudaMemcpyAsync(J->h_region, J->W.counter, J->reset_bytes, cudaMemcpyDeviceToHost, st));
  PBAT_CUDA(cudaStreamSynchronize(st));
  if (*J->h_status & 1u)
    return fail(PBAT_ETIMEOUT, "time budget of %.3f s ran out on the device",
                J->opt_copy.time_budget_s);
  if (J->bs)
    for (int i = 0; i < J->n_acc; ++i) J->h_acc[i] = limbs256_to_dd(J->h_limbs + 8 * i);
  if (opt) {
    const unsigned long long item = J->item_states;
    opt->stats[0] = J->h_stats[0] * item;
    opt->stats[1] = (J->h_stats[1] + J->h_stats[2]) * item;
    opt->stats[2] = J->wmid_bytes;
    opt->stats[3] = J->reset_bytes + (J->bs ? 0 : J->n_acc * sizeof(dd));
    double ns = 0.0;
    for (size_t i = 0; i < J->n_pending; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, J->evs[i].first, J->evs[i].second) == cudaSuccess)
        ns += ms * 1e6;
      else
        cudaGetLastError();
    }
    opt->stats[4] = (unsigned long long)ns;
    // one kernel per launch, two in two-phase runs; the frontier kernel adds its reduce
    opt->stats[5] = (J->bs ? (J->two_phase ? 2 : 1) : 2) * J->n_pending;
    opt->stats[6] = J->n_items;
    opt->stats[7] = J->n_pending;
  }
  J->n_pending = 0;
  const double R = J->h_acc[0].hi + J->h_acc[0].lo;
  std::vector<double> gi;
  if (J->bs && dRdp_out) {
    gi.resize(m);
    bs_finish_grad(*J->bs, J->h_acc, m, gi.data());
  }
  // The bit-sliced kernels' error bounds against the accuracy promised:
  // R within 1e-12 relative; each dR/dp_k within 1e-12 of max(|g_k|,
  // 1e-4 R) -- for an arc whose T1/T0 sums cancel, 1e-12 of |g_k| is below
  // what their rounding can resolve, so the floor 1e-4 R applies; where
  // they do not cancel (condition number below 2^53 * 1e-13) |g_k| exceeds
  // 1e-3 R, so 1e-12 * max(|g_k|, 1e-4 R) is met by the same test.
  bool too_coarse = false;
  if (J->bs && J->opt_copy.algo == PBAT_ALGO_AUTO) {
    too_coarse = R < 1e12 * J->abs_err_bound * J->mass;
    const double E = J->grad_err_bound * J->mass;
    for (size_t k = 0; k < gi.size() && !too_coarse; ++k)
      too_coarse = E > 1e-12 * std::max(std::fabs(gi[k]) - E, 1e-4 * R);
  }
  if (too_coarse) {
    // the fixed-point bounds of the bit-sliced kernel would not guarantee
    // that accuracy for so small an R (or gradient): run the frontier
    // kernel, whose tables are exact to 2^-100
    pbat_options o = J->opt_copy;
    o.algo = PBAT_ALGO_FRONTIER;
    Job* F = nullptr;
    int rc = job_create(J->g, J->p_copy.data(), J->pl.grad, &o, &F);
    if (!rc && !(rc = job_upload(F, st)) && !(rc = job_launch(F, st)))
      rc = job_read(F, st, R_out, Nk_out, J->pl.grad ? dRdp_out : nullptr, opt);
    job_destroy(F);
    return rc;
  }
  *R_out = R;
  if (Nk_out)
    for (int k = 0; k <= m; ++k) Nk_out[k] = J->h_n[k];
  if (dRdp_out) {
    if (J->bs) {
      for (int k = 0; k < m; ++k) dRdp_out[J->perm[k]] = gi[k];
    } else {
      for (int k = 0; k < m; ++k) {
        const dd v = J->h_acc[1 + k];
        dRdp_out[J->perm[k]] = v.hi + v.lo;
      }
    }
  }
  return PBAT_OK;
}

void job_destroy(Job* J) {
  if (!J) return;
  if (J->bs) bs_delete(J->bs);
  event_pairs_release(J->dev.device, J->evs);
  scratch_release(J->scr);
  delete J;
}

int run_single(const GraphIn& g, const double* p, bool grad, pbat_options* opt, void* stream,
               double* R_out, uint64_t* Nk_out, double* dRdp_out) {
  clear_error();
  if (!R_out) return fail(PBAT_EINVAL, "R_out must not be NULL");
  if (grad && !dRdp_out) return fail(PBAT_EINVAL, "dRdp_out must not be NULL");
  Job* J = nullptr;
  int rc = job_create(g, p, grad, opt, &J);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (!(rc = job_upload(J, st)) && !(rc = job_launch(J, st)))
    rc = job_read(J, st, R_out, Nk_out, grad ? dRdp_out : nullptr, opt);
  job_destroy(J);
  return rc;
}

}  // namespace pbat

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void pbat_options_init(pbat_options* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->struct_size = (int)sizeof(pbat_options);
  o->algo = PBAT_ALGO_AUTO;
  o->prefix_bits = -1;
  o->walk_bits = -1;
  o->block_threads = -1;
  o->prune = 1;
  o->autotune = 1;
  o->occupancy = -1;
  o->launches = 0;
}

int pbat_reliability(int n_nodes, int n_arcs, const int32_t* tail, const int32_t* head,
                     int directed, const double* p, int source, int sink, pbat_options* opt,
                     void* cuda_stream, double* R_out, uint64_t* Nk_out) {
  try {
    pbat::GraphIn g{n_nodes, n_arcs, tail, head, directed, source, sink};
    return pbat::run_single(g, p, false, opt, cuda_stream, R_out, Nk_out, nullptr);
  } catch (...) {
    return pbat::fail(PBAT_ENOMEM, "host exception");
  }
}

int pbat_reliability_grad(int n_nodes, int n_arcs, const int32_t* tail, const int32_t* head,
                          int directed, const double* p, int source, int sink, pbat_options* opt,
                          void* cuda_stream, double* R_out, uint64_t* Nk_out, double* dRdp_out) {
  try {
    pbat::GraphIn g{n_nodes, n_arcs, tail, head, directed, source, sink};
    return pbat::run_single(g, p, true, opt, cuda_stream, R_out, Nk_out, dRdp_out);
  } catch (...) {
    return pbat::fail(PBAT_ENOMEM, "host exception");
  }
}

int pbat_kernel_source(int n_nodes, int n_arcs, const int32_t* tail, const int32_t* head,
                       int directed, const double* p, int source, int sink, int want_grad,
                       const pbat_options* opt, char* buf, size_t cap) {
  try {
    pbat::clear_error();
    pbat::GraphIn g{n_nodes, n_arcs, tail, head, directed, source, sink};
    int rc;
    if ((rc = pbat::validate_graph(g)) || (rc = pbat::validate_options(opt, n_arcs))) return rc;
    if (p && (rc = pbat::validate_p(p, n_arcs))) return rc;
    pbat_options o;
    pbat_options_init(&o);
    if (opt) o = *opt;
    std::string src;
    if ((rc = pbat::bs_source_for(g, p, want_grad != 0, o, src))) return rc;
    if (buf && cap) {
      const size_t n = std::min(cap - 1, src.size());
      memcpy(buf, src.data(), n);
      buf[n] = '\0';
    }
    return (int)std::min<size_t>(src.size(), 0x7fffffff);
  } catch (...) {
    return pbat::fail(PBAT_ENOMEM, "host exception");
  }
}

static int batch_source(int n_graphs, const pbat_graph* graphs, int n_pvec, const double* p,
                        bool grad, const pbat_options* opt, char* buf, size_t cap) {
  try {
    pbat::clear_error();
    if (n_graphs < 1 || !graphs || n_pvec < 1 || n_pvec > 64)
      return pbat::fail(PBAT_EINVAL, "bad batch");
    std::vector<std::string> elig;
    size_t poff = 0;
    for (int i = 0; i < n_graphs; ++i) {
      pbat::GraphIn g{graphs[i].n_nodes, graphs[i].n_arcs, graphs[i].tail, graphs[i].head,
                      graphs[i].directed, graphs[i].source, graphs[i].sink};
      int rc = pbat::validate_graph(g);
      if (rc) return rc;
      if (grad) {
        // walk arcs of the gradient module: p in [2^-20, 1 - 2^-20] under
        // every p-vector (every arc when p is NULL)
        elig.emplace_back(g.m, '1');
        if (p)
          for (int k = 0; k < n_pvec; ++k)
            for (int a = 0; a < g.m; ++a) {
              const double x = p[poff + (size_t)k * g.m + a];
              if (!(x >= 0x1p-20 && x <= 1.0 - 0x1p-20)) elig.back()[a] = '0';
            }
        poff += (size_t)n_pvec * g.m;
      }
    }
    pbat_options o;
    pbat_options_init(&o);
    if (opt) o = *opt;
    std::string src;
    int rc = pbat::bsb_source_for(n_graphs, graphs, n_pvec, o, grad ? &elig : nullptr, src);
    if (rc) return rc;
    if (buf && cap) {
      const size_t n = std::min(cap - 1, src.size());
      memcpy(buf, src.data(), n);
      buf[n] = '\0';
    }
    return (int)std::min<size_t>(src.size(), 0x7fffffff);
  } catch (...) {
    return pbat::fail(PBAT_ENOMEM, "host exception");
  }
}

int pbat_batch_kernel_source(int n_graphs, const pbat_graph* graphs, int n_pvec,
                             const pbat_options* opt, char* buf, size_t cap) {
  return batch_source(n_graphs, graphs, n_pvec, nullptr, false, opt, buf, cap);
}

int pbat_batch_grad_kernel_source(int n_graphs, const pbat_graph* graphs, int n_pvec,
                                  const double* p, const pbat_options* opt, char* buf, size_t cap) {
  return batch_source(n_graphs, graphs, n_pvec, p, true, opt, buf, cap);
}

struct pbat_plan_s {
  pbat::Job* job;
  pbat_options opt;
};

int pbat_plan_create(int n_nodes, int n_arcs, const int32_t* tail, const int32_t* head,
                     int directed, const double* p, int source, int sink, int want_grad,
                     pbat_options* opt, void* cuda_stream, pbat_plan* plan_out) {
  try {
    pbat::clear_error();
    if (!plan_out) return pbat::fail(PBAT_EINVAL, "plan_out must not be NULL");
    pbat::GraphIn g{n_nodes, n_arcs, tail, head, directed, source, sink};
    pbat::Job* J = nullptr;
    int rc = pbat::job_create(g, p, want_grad != 0, opt, &J);
    if (rc) return rc;
    if ((rc = pbat::job_upload(J, (cudaStream_t)cuda_stream)) ||
        (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess &&
         (rc = pbat::fail(PBAT_ECUDA, "table upload failed")))) {
      pbat::job_destroy(J);
      return rc;
    }
    pbat_plan pl = new pbat_plan_s();
    pl->job = J;
    pbat_options_init(&pl->opt);
    if (opt) pl->opt = *opt;
    *plan_out = pl;
    return PBAT_OK;
  } catch (...) {
    return pbat::fail(PBAT_ENOMEM, "host exception");
  }
}

int pbat_plan_execute(pbat_plan plan, void* cuda_stream) {
  pbat::clear_error();
  if (!plan) return pbat::fail(PBAT_EINVAL, "plan must not be NULL");
  return pbat::job_launch(plan->job, (cudaStream_t)cuda_stream);
}

int pbat_plan_read(pbat_plan plan, void* cuda_stream, double* R_out, uint64_t* Nk_out,
                   double* dRdp_out) {
  pbat::clear_error();
  if (!plan || !R_out) return pbat::fail(PBAT_EINVAL, "plan and R_out must not be NULL");
  return pbat::job_read(plan->job, (cudaStream_t)cuda_stream, R_out, Nk_out,
                        plan->job->pl.grad ? dRdp_out : nullptr, &plan->opt);
}

int pbat_plan_describe(pbat_plan plan, int* out8) {
  pbat::clear_error();
  if (!plan || !out8) return pbat::fail(PBAT_EINVAL, "plan and out8 must not be NULL");
  const pbat::Job* J = plan->job;
  if (J->bs) {
    int d6[6];
    pbat::bs_describe(*J->bs, d6);
    out8[0] = PBAT_ALGO_BITSLICE;
    for (int i = 0; i < 4; ++i) out8[1 + i] = d6[i];
  } else {
    out8[0] = PBAT_ALGO_FRONTIER;
    out8[1] = J->pl.ell;
    out8[2] = 0;
    out8[3] = J->pl.L;
    out8[4] = J->pl.d;
  }
  out8[5] = J->grid_nthr;
  out8[6] = J->grid;
  out8[7] = J->pl.grad ? 1 : 0;
  return PBAT_OK;
}

int pbat_plan_stats(pbat_plan plan, uint64_t* stats_out) {
  pbat::clear_error();
  if (!plan || !stats_out) return pbat::fail(PBAT_EINVAL, "plan and stats_out must not be NULL");
  for (int i = 0; i < 8; ++i) stats_out[i] = plan->opt.stats[i];
  return PBAT_OK;
}

void pbat_plan_destroy(pbat_plan plan) {
  if (!plan) return;
  pbat::job_destroy(plan->job);
  delete plan;
}

const char* pbat_last_error(void) { return pbat::last_error(); }

int pbat_version(void) { return 1 * 10000 + 0 * 100 + 0; }

}  // extern "C"
