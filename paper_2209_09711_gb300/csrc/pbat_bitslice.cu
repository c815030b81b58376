// pbat_bitslice.cu -- launcher of the bit-sliced enumeration kernels: the
// NVRTC compile cache, the per-network tables and parameters, the launch,
// the host finish of the fused gradient, and the batched module.  The
// planner and the generated connectivity program are in pbat_bs_plan.cu.

#include <cuda_runtime.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <string>
#include <thread>
#include <vector>

#include "pbat.h"
#include "pbat_bs_plan.h"
#include "pbat_bs_template.h"
#include "pbat_engine.h"
#include "pbat_internal.h"
#include "pbat_nvtx.h"

namespace pbat {

// Host mirror of BsParams in the kernel source (same field order and types).
struct BsParamsHost {
  unsigned long long task_lo, n_tasks, budget_ns;
  int prune, nlev, ex_shift, pad;
  int lev_bits[10];
  int lev_off[10];
  unsigned long long thw[32];
  unsigned long long binom[64];
};

// ---------------------------------------------------------------------------
// NVRTC compile cache
// ---------------------------------------------------------------------------
struct JitEntry {
  cudaLibrary_t lib = nullptr;
  cudaKernel_t kernel = nullptr;
  // the two launches of a two-launch run (single-network kernels only)
  cudaKernel_t kernel_p1 = nullptr, kernel_p2 = nullptr;
  int regs = 0;
};
static std::mutex g_jit_mu;
static std::map<std::string, JitEntry> g_jit;

static std::mutex g_cubin_mu;
static std::map<std::string, std::vector<char>> g_cubin;   // compiled ahead, not yet loaded

// NVRTC only -- no CUDA call, so any host thread may run it.  On failure
// `err` holds the compiler's error lines.
static bool nvrtc_cubin(const std::string& src, int cc, std::vector<char>& cubin, std::string& err) {
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "pbat_bitslice_gen.cu", 0, nullptr, nullptr) !=
      NVRTC_SUCCESS) {
    err = "nvrtcCreateProgram failed";
    return false;
  }
  const std::string arch = "-arch=sm_" + std::to_string(cc) + "a";
  const char* opts[] = {arch.c_str(), "-std=c++17", "-lineinfo", "-diag-suppress=177"};
  const nvrtcResult rc = nvrtcCompileProgram(prog, 4, opts);
  if (rc != NVRTC_SUCCESS) {
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    std::string all(ls, '\0');
    if (ls) nvrtcGetProgramLog(prog, &all[0]);
    nvrtcDestroyProgram(&prog);
    // keep the error lines only
    err = std::string(nvrtcGetErrorString(rc)) + " ";
    size_t at = 0;
    while (at < all.size()) {
      size_t nl = all.find('\n', at);
      if (nl == std::string::npos) nl = all.size();
      const std::string line = all.substr(at, nl - at);
      if (line.find("error") != std::string::npos) err += line + " | ";
      at = nl + 1;
    }
    if (err.size() > 400) err.resize(400);
    return false;
  }
  size_t cs = 0;
  nvrtcGetCUBINSize(prog, &cs);
  cubin.resize(cs);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  return true;
}

// Compile several sources at once on host threads (the autotuner's
// candidates); the cubins wait for jit_compile.  A failure is left for
// jit_compile to report when that source is needed.
static void jit_precompile(const std::vector<std::string>& srcs, int cc) {
  NvtxRange nv("pbat NVRTC precompile");
  std::vector<const std::string*> todo;
  {
    std::lock_guard<std::mutex> lj(g_jit_mu);
    std::lock_guard<std::mutex> lc(g_cubin_mu);
    for (const auto& src : srcs)
      if (!g_jit.count(src) && !g_cubin.count(src)) todo.push_back(&src);
  }
  if (todo.empty()) return;
  std::atomic<size_t> next{0};
  auto work = [&]() {
    for (;;) {
      const size_t i = next++;
      if (i >= todo.size()) return;
      std::vector<char> cubin;
      std::string err;
      if (!nvrtc_cubin(*todo[i], cc, cubin, err)) continue;
      std::lock_guard<std::mutex> lc(g_cubin_mu);
      g_cubin.emplace(*todo[i], std::move(cubin));
    }
  };
  const int nthreads =
      std::max(1, std::min({(int)todo.size(), 16, (int)std::thread::hardware_concurrency()}));
  std::vector<std::thread> pool;
  for (int t = 1; t < nthreads; ++t) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
}

static int jit_compile(const std::string& src, const DeviceInfo& dev, const char* kname,
                       JitEntry* out) {
  if (fault_at("compile")) return fail(PBAT_ECUDA, "injected fault: NVRTC compile");
  std::lock_guard<std::mutex> lk(g_jit_mu);
  auto it = g_jit.find(src);
  if (it != g_jit.end()) {
    *out = it->second;
    return PBAT_OK;
  }
  std::vector<char> cubin;
  {
    std::lock_guard<std::mutex> lc(g_cubin_mu);
    auto c = g_cubin.find(src);
    if (c != g_cubin.end()) {
      cubin.swap(c->second);
      g_cubin.erase(c);
    }
  }
  if (cubin.empty()) {
    NvtxRange nv("pbat NVRTC compile");
    std::string err;
    if (!nvrtc_cubin(src, dev.cc_major * 10 + dev.cc_minor, cubin, err))
      return fail(PBAT_ECUDA, "NVRTC compile of the bit-sliced kernel failed: %s", err.c_str());
  }
  JitEntry e;
  cudaError_t ce = cudaLibraryLoadData(&e.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
  if (ce != cudaSuccess) return fail(PBAT_ECUDA, "cudaLibraryLoadData: %s", cudaGetErrorString(ce));
  ce = cudaLibraryGetKernel(&e.kernel, e.lib, kname);
  if (ce != cudaSuccess) return fail(PBAT_ECUDA, "cudaLibraryGetKernel: %s", cudaGetErrorString(ce));
  // optional per-phase entry points: absent from the batched modules
  if (cudaLibraryGetKernel(&e.kernel_p1, e.lib, (std::string(kname) + "_p1").c_str()) != cudaSuccess ||
      cudaLibraryGetKernel(&e.kernel_p2, e.lib, (std::string(kname) + "_p2").c_str()) != cudaSuccess) {
    cudaGetLastError();
    e.kernel_p1 = e.kernel_p2 = nullptr;
  }
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, (const void*)e.kernel) == cudaSuccess) e.regs = fa.numRegs;
  else cudaGetLastError();
  g_jit.emplace(src, e);
  *out = e;
  return PBAT_OK;
}

// ---------------------------------------------------------------------------
// tables and launch
// ---------------------------------------------------------------------------
struct BsGradParamsHost {
  unsigned long long thw_ex[5][32];
  unsigned long long lw_ex[5][32];
  dd inv_p[64], inv_q[64];
};

struct BsLaunch {
  BsPlan plan;
  BsParamsHost P;
  BsGradParamsHost Q;
  std::vector<unsigned long long> thr_tab;   // [4][256] (fused kernel)
  std::vector<unsigned long long> wmid128;   // [2^L][2] (fused kernel)
  std::vector<MxHost> ptab;                  // prefix masses per level
  std::vector<MxHost> ptab_ex;               // [prefix arc][2^11]: its level without it
  std::vector<unsigned long long> lane_tab;  // [4][256][2]: lane mass, packed class counts
  std::vector<unsigned long long> wmid;      // [2^L]
  JitEntry jit;
  int nthr = 128;
  size_t smem = 0;
  int per_sm = 1;                     // resident blocks per SM: one-launch kernel
  int per_sm1 = 1, per_sm2 = 1;       // the two launches of a two-launch run
  size_t smem1 = 0;                   // shared memory of the first of two fused launches
};

// out[v] = product over x < n of (bit x of v ? p : 1 - p) of arc arcs[x], for
// every v < 2^n, built by doubling: two double-double products per entry.

// Byte-table sums from 32 pattern masses w[]: entry (b, v) is the sum of
// w[8b + x] over the set bits x of v, rounded to 2^62 fixed point.  The
// masses are rounded once to 2^126 and the subset sums are exact 128-bit
// integer additions (one per entry, by the lowest set bit).


static const int kNkShift[6] = {0, 8, 19, 31, 43, 54};

// packed N_k counts of a word whose every lane state is connected
static unsigned long long full_counts(int ell) {
  unsigned long long n = 0;
  for (int j = 0; j < (1 << ell); ++j) n += 1ull << kNkShift[__builtin_popcount((unsigned)j)];
  return n;
}

// The fused kernel keeps each lane's accumulators in registers when the
// item is short (the per-item global update would be a large share of it)
// or the per-word connectivity program is small (registers to spare); on
// GB300: 3x6 grid (L = 5) 70.5 -> 66.7 us, 34-arc directed network (12
// operations per word) 1.54 -> 1.43 ms, but the 40-arc network (260
// operations per word) 144.7 -> 157.6 ms, so that one keeps global slots.
static bool acc_in_registers(const BsPlan& bp) { return bp.L <= 6 || bp.ops_var <= 128; }

// Walk arcs unrolled per step (2^in_bits words with compile-time walk words):
// three give more independent words to the R kernel (GB300: 40-arc network
// 106.5 -> 87.8 ms, 34-arc directed 541 -> 495 us) and to the fused kernel
// when its accumulators are in registers (34-arc 1437 -> 1385 us), but the
// fused kernel with a large program loses registers to them (40-arc 147.4 ->
// 154 ms) and keeps two.  The R kernel of a short program (at most 64
// operations per word) takes four (prune-aware 40-arc plan, 27 operations:
// 7.69 -> 7.45 ms); the fused kernel measured slower with four (18.7 -> 22.7
// ms).
static int walk_unroll_bits(const BsPlan& bp) {
  if (!bp.grad) return bp.ops_var <= 64 ? 4 : 3;
  return acc_in_registers(bp) ? 3 : 2;
}

static std::string bs_source(const GraphIn& g, const BsPlan& bp, int nthr) {
  char defs[700];
  const unsigned lane_mask = bp.ell >= 5 ? 0xffffffffu : ((1u << (1 << bp.ell)) - 1u);
  snprintf(defs, sizeof defs,
           "#define BS_M %d\n#define BS_ELL %d\n#define BS_TB %d\n#define BS_L %d\n#define BS_D %d\n"
           "#define BS_NTHR %d\n#define BS_WALK0 %d\n#define BS_TOP %d\n#define BS_NCORE %d\n"
           "#define BS_LANE_MASK 0x%08xu\n#define BS_FULL_COUNTS 0x%016llxull\n#define BS_GRAD %d\n"
           "#define BS_ACC_REG %d\n#define BS_IN_BITS %d\n#define BS_THR_MASK 0x%08xu\n"
           "#define BS_MINB %d\n#define BS_PEX_MASK 0x%016llxull\n",
           g.m, bp.ell, bp.tb, bp.L, bp.d, nthr, bp.ell + bp.tb, bp.ell + bp.tb + bp.L, bp.ncore,
           lane_mask, full_counts(bp.ell), bp.grad ? 1 : 0, acc_in_registers(bp) ? 1 : 0,
           walk_unroll_bits(bp), bp.tb >= 5 ? 0xffffffffu : ((1u << (1 << bp.tb)) - 1u), bp.minb,
           bp.pex);
  const std::string tmpl = kBsTemplate;
  const size_t cut = tmpl.find("//@@GENERATED@@");
  // only this plan's kernel: the other kernel's section is left out, so that
  // a change to one kernel leaves the other's generated source unchanged
  std::string tail = tmpl.substr(cut);
  const size_t r0 = tail.find("#if !BS_GRAD\n"), f0 = tail.find("#if BS_GRAD\n");
  const size_t f1 = tail.rfind("#endif");
  if (r0 != std::string::npos && f0 != std::string::npos && f1 != std::string::npos && r0 < f0 && f0 < f1) {
    if (bp.grad) tail.erase(r0, f0 - r0);
    else tail.erase(f0, f1 + 6 - f0);
  }
  return std::string(defs) + tmpl.substr(0, cut) + bp.gen + tail;
}

// Generated source for a network (no device needed); see pbat_kernel_source.
int bs_source_for(const GraphIn& g, const double* p, bool grad, const pbat_options& o,
                  std::string& out) {
  BsPlan bp;
  const int nthr = o.block_threads > 0 ? o.block_threads : 128;
  std::vector<double> half;
  if (grad && !p) {
    half.assign(g.m, 0.5);
    p = half.data();
  }
  int rc = bs_make_plan(g, o, nthr, bp, grad ? p : nullptr);
  if (rc) return rc;
  char perm[64 * 4 + 64] = "// internal arc -> input arc:";
  for (int k = 0; k < g.m; ++k) snprintf(perm + strlen(perm), 8, " %d", bp.perm[k]);
  out = std::string(perm) + "\n" + bs_source(g, bp, nthr);
  return PBAT_OK;
}

// Plans (and their compiled kernels) depend on the network's structure, the
// options and -- for the fused kernel -- which arcs may be walk arcs; they
// are cached so that repeated calls only rebuild the p-dependent tables.
struct BsCached {
  BsPlan plan;
  JitEntry jit;
  size_t smem = 0;   // shared memory the kernel attribute was set for
  int per_sm = 0;    // resident blocks per SM at that size (one-launch kernel)
  int per_sm1 = 0, per_sm2 = 0;   // the two launches of a two-launch run
};
static std::mutex g_bsplan_mu;
static std::map<std::string, BsCached> g_bsplan;

static std::string bs_plan_key(const GraphIn& g, const double* p, bool grad, const pbat_options& o,
                               int nthr, int device) {
  std::string k;
  auto put = [&](long long v) { k.append((const char*)&v, sizeof v); };
  put(device); put(g.n); put(g.m); put(g.directed); put(g.source); put(g.sink); put(grad);
  put(o.walk_bits); put(o.prefix_bits); put(o.range_bits); put(nthr); put(o.prune == 2);
  put(std::max(0, o.occupancy));
  k.append((const char*)g.tail, sizeof(int32_t) * g.m);
  k.append((const char*)g.head, sizeof(int32_t) * g.m);
  if (grad)
    for (int a = 0; a < g.m; ++a) k.push_back(bs_walk_ok(p, a) ? '1' : '0');
  return k;
}

// Compile the kernels of several option sets ahead of bs_prepare, on host
// threads (the autotuner's candidates: one NVRTC compile each, which would
// otherwise run one after another).  Plans that fail are skipped here and
// reported when bs_prepare meets them.
void bs_precompile(const GraphIn& g, const double* p, bool grad,
                   const std::vector<pbat_options>& opts, const DeviceInfo& dev) {
  std::vector<std::string> srcs;
  for (const pbat_options& o : opts) {
    const int nthr = o.block_threads > 0 ? o.block_threads : 128;
    {
      std::lock_guard<std::mutex> lk(g_bsplan_mu);
      if (g_bsplan.count(bs_plan_key(g, p, grad, o, nthr, dev.device))) continue;
    }
    BsPlan bp;
    if (bs_make_plan(g, o, nthr, bp, grad ? p : nullptr)) {
      clear_error();
      continue;
    }
    srcs.push_back(bs_source(g, bp, nthr));
  }
  jit_precompile(srcs, dev.cc_major * 10 + dev.cc_minor);
}

int bs_prepare(const GraphIn& g, const double* p, bool grad, const pbat_options& o,
               const DeviceInfo& dev, BsLaunch& bl) {
  bl.nthr = o.block_threads > 0 ? o.block_threads : 128;
  int rc;
  const std::string key = bs_plan_key(g, p, grad, o, bl.nthr, dev.device);
  bool cached = false;
  {
    std::lock_guard<std::mutex> lk(g_bsplan_mu);
    auto it = g_bsplan.find(key);
    if (it != g_bsplan.end()) {
      bl.plan = it->second.plan;
      bl.jit = it->second.jit;
      cached = true;
    }
  }
  if (!cached) {
    if ((rc = bs_make_plan(g, o, bl.nthr, bl.plan, grad ? p : nullptr))) return rc;
    const std::string src = bs_source(g, bl.plan, bl.nthr);
    if ((rc = jit_compile(src, dev, grad ? "bs_kernel_grad" : "bs_kernel", &bl.jit))) return rc;
    std::lock_guard<std::mutex> lk(g_bsplan_mu);
    g_bsplan[key] = BsCached{bl.plan, bl.jit, 0, 0};
  }
  const BsPlan& bp = bl.plan;
  const int m = g.m, top = bp.ell + bp.tb + bp.L;
  // parameters
  BsParamsHost& P = bl.P;
  memset(&P, 0, sizeof P);
  P.prune = o.prune ? 1 : 0;
  P.budget_ns = o.time_budget_s > 0 ? (unsigned long long)(o.time_budget_s * 1e9) : 0ull;
  dd tw[32];
  for (int j = 0; j < 32; ++j) {
    tw[j] = dd{0.0, 0.0};
    if (j >= (1 << bp.tb)) continue;
    dd w = dd_make(1.0);
    for (int i = 0; i < bp.tb; ++i) w = dd_mul(w, arc_w(p, bp.perm[bp.ell + i], (j >> i) & 1));
    tw[j] = w;
    P.thw[j] = fixed_u64(w, 63);
  }
  for (int j = 0; j < 64; ++j) P.binom[j] = binom_u64(top, j);
  unsigned long long lo = 0, hi = 1ull << bp.d;
  if (bp.r > 0) {
    lo = o.range_lo << (bp.d - bp.r);
    hi = o.range_hi << (bp.d - bp.r);
  }
  P.task_lo = lo;
  P.n_tasks = hi - lo;
  // prefix masses: the d prefix arcs in levels of at most 6 bits (fused
  // kernel: the per-arc excluded tables stay small) or 8 bits (R only); each
  // entry is the double-double product over the level's arcs, rounded to
  // the kernels' integer floating point, and a level product on the device
  // is one integer multiply
  const int max_bits = grad ? 6 : 8;
  P.nlev = (bp.d + max_bits - 1) / max_bits;
  P.ex_shift = max_bits;
  bl.ptab.clear();
  bl.ptab_ex.assign(grad ? (size_t)bp.d << max_bits : 0, MxHost{0, 0, 0});
  for (int l = 0, sh = 0; l < P.nlev; ++l) {
    const int bits = bp.d / P.nlev + (l < bp.d % P.nlev ? 1 : 0);
    P.lev_bits[l] = bits;
    P.lev_off[l] = (int)bl.ptab.size();
    std::vector<dd> tab((size_t)1 << bits);
    product_table(p, bp.perm.data() + top + sh, bits, tab.data());
    for (int v = 0; v < (1 << bits); ++v) bl.ptab.push_back(to_mx(tab[v]));
    if (grad)
      for (int jj = 0; jj < bits; ++jj) {
        // the level's product without arc jj: a table over the other arcs,
        // indexed by v with bit jj removed
        int others[12];
        for (int x = 0, n = 0; x < bits; ++x)
          if (x != jj) others[n++] = bp.perm[top + sh + x];
        product_table(p, others, bits - 1, tab.data());
        for (int v = 0; v < (1 << bits); ++v) {
          const int u = (v & ((1 << jj) - 1)) | ((v >> (jj + 1)) << jj);
          bl.ptab_ex[((size_t)(sh + jj) << max_bits) + v] = to_mx(tab[u]);
        }
      }
    sh += bits;
  }
  if (bl.ptab.empty()) bl.ptab.push_back(to_mx(dd_make(1.0)));
  // lane tables: byte position b, value v -> lane mass (scale 2^62) and the
  // counts of its set lanes by lane popcount class, packed in fields of
  // 8, 11, 12, 12, 11, 8 bits
  bl.lane_tab.assign(4 * 256 * 2, 0ull);
  dd lw[32];
  for (int j = 0; j < 32; ++j) lw[j] = dd{0.0, 0.0};
  product_table(p, bp.perm.data(), bp.ell, lw);
  byte_table_sums(lw, 1 << bp.ell, bl.lane_tab.data(), 2);
  for (int b = 0; b < 4; ++b) {
    // counts by the lowest set bit: one addition per entry
    unsigned long long nb[256];
    nb[0] = 0;
    for (int v = 1; v < 256; ++v) {
      const int j = 8 * b + __builtin_ctz((unsigned)v);
      nb[v] = nb[v & (v - 1)] + (j < (1 << bp.ell) ? 1ull << kNkShift[__builtin_popcount((unsigned)j)] : 0ull);
      bl.lane_tab[(b * 256 + v) * 2 + 1] = nb[v];
    }
  }
  const int L_in = std::min(bp.L, walk_unroll_bits(bp)), L_out = bp.L - L_in;
  if (!grad) {
    bl.wmid.resize((size_t)1 << bp.L);
    std::vector<dd> wt((size_t)1 << bp.L);
    product_table(p, bp.perm.data() + bp.ell + bp.tb, bp.L, wt.data());
    for (int gi = 0; gi < (1 << bp.L); ++gi) bl.wmid[gi] = fixed_u64(wt[gi], 63);
    bl.smem = (size_t)(4 * 256 * 2 + (1 << bp.L) + (bp.L + 1) * bl.nthr) * 8 +
              (size_t)(bl.nthr / 32) * 24 + (size_t)(m + 1) * 8;
  } else {
    // fused kernel: thread-pattern masses, 128-bit walk masses, fixed-point
    // excluded-arc masses, reciprocals of the walk arcs' p and 1 - p
    memset(&bl.Q, 0, sizeof bl.Q);
    bl.thr_tab.assign(4 * 256, 0ull);
    byte_table_sums(tw, 1 << bp.tb, bl.thr_tab.data(), 1);
    bl.wmid128.resize((size_t)2 << bp.L);
    std::vector<dd> wt((size_t)1 << bp.L);
    product_table(p, bp.perm.data() + bp.ell + bp.tb, bp.L, wt.data());
    for (int gi = 0; gi < (1 << bp.L); ++gi) {
      const u128 f = to_fixed127(wt[gi]);
      bl.wmid128[2 * gi] = f.lo;
      bl.wmid128[2 * gi + 1] = f.hi;
    }
    // pattern masses without arc x: a product table over the other arcs,
    // indexed by the pattern with bit x removed
    auto excluded = [&](const int* arcs, int n, unsigned long long (*out)[32]) {
      for (int x = 0; x < n; ++x) {
        int others[5];
        for (int i = 0, c = 0; i < n; ++i)
          if (i != x) others[c++] = arcs[i];
        dd tab[16];
        product_table(p, others, n - 1, tab);
        for (int j = 0; j < (1 << n); ++j)
          out[x][j] = fixed_u64(tab[(j & ((1 << x) - 1)) | ((j >> (x + 1)) << x)], 63);
      }
    };
    excluded(bp.perm.data() + bp.ell, bp.tb, bl.Q.thw_ex);
    excluded(bp.perm.data(), bp.ell, bl.Q.lw_ex);
    // 1/p and 1/(1 - p) of the walk arcs and of the prefix arcs whose sums
    // carry their own factor (every prefix arc not in pex)
    for (int k = bp.ell + bp.tb; k < m; ++k) {
      if (k >= top && ((bp.pex >> k) & 1ull)) continue;
      const double pk = p[bp.perm[k]];
      bl.Q.inv_p[k] = dd_recip(pk);
      bl.Q.inv_q[k] = dd_recip_dd(dd_one_minus(pk));
    }
    bl.smem = (size_t)(4 * 256 * 2 + 2 * (1 << bp.L) + 4 * 256 + (bp.L + 1) * bl.nthr) * 8 +
              (size_t)std::max(L_out, 1) * bl.nthr * 16 + (size_t)(m + 1) * 8;
  }
  if (bl.smem > (size_t)dev.smem_optin)
    return fail(PBAT_ERANGE, "bit-sliced kernel needs %zu B of shared memory", bl.smem);
  {
    // the shared-memory attribute and the occupancy of a cached kernel are
    // known after its first preparation
    std::lock_guard<std::mutex> lk(g_bsplan_mu);
    auto it = g_bsplan.find(key);
    if (it != g_bsplan.end() && it->second.per_sm > 0 && it->second.smem == bl.smem) {
      bl.per_sm = it->second.per_sm;
      bl.per_sm1 = it->second.per_sm1;
      bl.per_sm2 = it->second.per_sm2;
      bl.smem1 = grad ? (size_t)(m + 1) * 8 : bl.smem;
      return PBAT_OK;
    }
  }
  // shared-memory attribute and resident blocks per SM of each entry point
  // (the first of two fused launches needs only the N_k counts)
  bl.smem1 = grad ? (size_t)(m + 1) * 8 : bl.smem;
  auto setup = [&](cudaKernel_t k, size_t smem, int* per_sm) -> int {
    *per_sm = 1;
    if (!k) return PBAT_OK;
    cudaError_t e = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return fail(PBAT_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, (const void*)k, bl.nthr, smem);
    if (e != cudaSuccess || *per_sm < 1) {
      cudaGetLastError();
      *per_sm = 1;
    }
    return PBAT_OK;
  };
  if ((rc = setup(bl.jit.kernel, bl.smem, &bl.per_sm)) ||
      (rc = setup(bl.jit.kernel_p1, bl.smem1, &bl.per_sm1)) ||
      (rc = setup(bl.jit.kernel_p2, bl.smem, &bl.per_sm2)))
    return rc;
  std::lock_guard<std::mutex> lk(g_bsplan_mu);
  auto it = g_bsplan.find(key);
  if (it != g_bsplan.end()) {
    it->second.smem = bl.smem;
    it->second.per_sm = bl.per_sm;
    it->second.per_sm1 = bl.per_sm1;
    it->second.per_sm2 = bl.per_sm2;
  }
  return PBAT_OK;
}

// Launch with the device copies of the tables (see bs_tables for the order).
// phase 0: the one-launch kernel; 1, 2: the two launches of a two-launch run.
cudaError_t bs_launch(const BsLaunch& bl, int grid, cudaStream_t st, const unsigned long long* d_lane,
                      const unsigned long long* d_thr, const unsigned long long* d_wmid,
                      const void* d_ptab, const void* d_ptab_ex, const DevWork& W, int phase) {
  const BsParamsHost& P = bl.P;
  const cudaKernel_t k = phase == 1 ? bl.jit.kernel_p1 : phase == 2 ? bl.jit.kernel_p2 : bl.jit.kernel;
  if (!k) return cudaErrorInvalidDeviceFunction;
  if (bl.plan.grad) {
    const BsGradParamsHost& Q = bl.Q;
    void* args[] = {(void*)&P, (void*)&Q, (void*)&d_lane, (void*)&d_thr, (void*)&d_wmid,
                    (void*)&d_ptab, (void*)&d_ptab_ex, (void*)&W};
    return cudaLaunchKernel((const void*)k, dim3(grid), dim3(bl.nthr), args,
                            phase == 1 ? bl.smem1 : bl.smem, st);
  }
  void* args[] = {(void*)&P, (void*)&d_lane, (void*)&d_wmid, (void*)&d_ptab, (void*)&W};
  return cudaLaunchKernel((const void*)k, dim3(grid), dim3(bl.nthr), args, bl.smem, st);
}

// accessors used by the engine
const std::vector<int>& bs_perm(const BsLaunch& bl) { return bl.plan.perm; }
unsigned long long bs_items(const BsLaunch& bl) { return bl.P.n_tasks; }
unsigned long long bs_item_states(const BsLaunch& bl) {
  return 1ull << (bl.plan.ell + bl.plan.tb + bl.plan.L);
}
int bs_per_sm(const BsLaunch& bl, int phase) {
  return phase == 1 ? bl.per_sm1 : phase == 2 ? bl.per_sm2 : bl.per_sm;
}
int bs_nthr(const BsLaunch& bl) { return bl.nthr; }
const std::vector<unsigned long long>& bs_lane_tab(const BsLaunch& bl) { return bl.lane_tab; }
const std::vector<unsigned long long>& bs_wmid(const BsLaunch& bl) {
  return bl.plan.grad ? bl.wmid128 : bl.wmid;
}
const std::vector<unsigned long long>& bs_thr_tab(const BsLaunch& bl) { return bl.thr_tab; }
const std::vector<MxHost>& bs_ptab(const BsLaunch& bl) { return bl.ptab; }
const std::vector<MxHost>& bs_ptab_ex(const BsLaunch& bl) { return bl.ptab_ex; }
bool bs_grad(const BsLaunch& bl) { return bl.plan.grad; }

// The fused kernel's result holds R, then A_k and B_k for every internal arc
// k: the gradient is A / p - B / (1 - p) for walk arcs and for prefix arcs
// with p in [2^-20, 1 - 2^-20] (their sums carry the arc's own factor), A - B
// for the other prefix arcs (masses without the arc, working minus failed),
// and A for lane and thread arcs (exact pair differences).
void bs_finish_grad(const BsLaunch& bl, const dd* acc, int m, double* g_internal) {
  const BsPlan& bp = bl.plan;
  const int walk0 = bp.ell + bp.tb, top = walk0 + bp.L;
  for (int k = 0; k < m; ++k) {
    const dd a = acc[1 + 2 * k], b = acc[2 + 2 * k];
    dd v;
    if (k >= top && ((bp.pex >> k) & 1ull))
      v = dd_sub(a, b);
    else if (k >= walk0)
      v = dd_sub(dd_mul(a, bl.Q.inv_p[k]), dd_mul(b, bl.Q.inv_q[k]));
    else
      v = a;
    g_internal[k] = v.hi + v.lo;
  }
}
BsLaunch* bs_new() { return new BsLaunch(); }
void bs_delete(BsLaunch* b) { delete b; }
void bs_describe(const BsLaunch& bl, int* out6) {
  out6[0] = bl.plan.ell; out6[1] = bl.plan.tb; out6[2] = bl.plan.L; out6[3] = bl.plan.d;
  out6[4] = bl.plan.ops_inv; out6[5] = bl.plan.ops_var;
}

}  // namespace pbat

// ---------------------------------------------------------------------------
// Batched bit-sliced enumeration: one module, one persistent kernel.
// ---------------------------------------------------------------------------
namespace pbat {

struct BGraphHost {
  unsigned long long task_begin, n_tasks;
  int gidx, m, nlev, prune;
  int lev_bits[8], lev_off[8];
  int lt_off, nt_off, wm_off, pt_off, pt_size, thw_off, nk_off, tb;
  int L, top;
  unsigned lane_mask;
  int pad0;
  int wm2_off, tt_off, lwex_off, thwex_off, ptex_off, out_off, ell, d;
  unsigned thr_mask;
  int pad1;
  unsigned long long full_counts;
  unsigned long long pex_mask;
  unsigned long long binom[64];
};

constexpr int kBsbThreads = 128;
constexpr int kBsbMinBlocks = 4;  // default launch bounds: 4 blocks of 128 threads, <= 128 registers
constexpr int kBsbMaxWalk = 5;  // 2^L connectivity words per thread staged in shared memory
constexpr int kBsbLimbs = 8;    // 32-bit chunks of a 256-bit value at scale 2^250, in 64-bit atomics
constexpr int kBsbMaxGraphs = 256;

struct BsBatch {
  std::string key;
  bool busy = false;
  int device = -1, G = 0, K = 0, Kp = 0, grid = 0, lmax = 0;
  int minb = 4;                     // launch bounds: blocks per SM the registers must allow
  size_t smem = 0;
  JitEntry jit;
  std::vector<BsPlan> plans;        // input order
  std::vector<int> order;           // launch order -> input index
  std::vector<BGraphHost> bg;       // launch order
  unsigned long long total = 0;
  int nk_total = 0;
  size_t n_lt = 0, n_nt = 0, n_wm = 0, n_pt = 0, n_thw = 0;
  Scratch* scr = nullptr;
  size_t o_graphs, o_lt, o_nt, o_wm, o_pt, o_thw, o_upload_end, o_limbs, o_nk, o_counter, o_status, o_end;
  cudaGraphExec_t exec = nullptr;
  // the gradient module (bs_batch_grad): which arcs of each network may be
  // walk arcs (p in [2^-20, 1 - 2^-20] for every p-vector), its extra tables
  // and the size of its results (R, then A_k and B_k of every arc, per
  // network and p-vector)
  bool grad = false;
  std::vector<std::string> elig;   // input order, one '0'/'1' per arc
  size_t o_wm2 = 0, o_tt = 0, o_lwex = 0, o_thwex = 0, o_ptex = 0, n_out = 0;
};

static std::mutex g_bsb_mu;
static std::vector<BsBatch*> g_bsb;

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

static int bsb_layout(BsBatch& E, int G, const pbat_graph* graphs, int K, const pbat_options& o,
                      const DeviceInfo& dev, const std::vector<unsigned long long>& items);

// Plans every network, orders them by work, and writes the module source.
static int bsb_source(BsBatch& E, int G, const pbat_graph* graphs, int K, const pbat_options& o,
                      std::vector<unsigned long long>& items, std::string& src_out);

static int bsb_build(BsBatch& E, int G, const pbat_graph* graphs, int K, const pbat_options& o,
                     const DeviceInfo& dev) {
  E.device = dev.device;
  std::vector<unsigned long long> items;
  std::string src;
  int rc = bsb_source(E, G, graphs, K, o, items, src);
  if (rc) return rc;
  if ((rc = jit_compile(src, dev, E.grad ? "bs_batch_grad" : "bs_batch", &E.jit))) return rc;
  return bsb_layout(E, G, graphs, K, o, dev, items);
}

static int bsb_source(BsBatch& E, int G, const pbat_graph* graphs, int K, const pbat_options& o,
                      std::vector<unsigned long long>& items, std::string& src_out) {
  E.G = G;
  E.K = K;
  E.plans.resize(G);
  items.assign(G, 0ull);
  for (int i = 0; i < G; ++i) {
    GraphIn g{graphs[i].n_nodes, graphs[i].n_arcs, graphs[i].tail, graphs[i].head,
              graphs[i].directed, graphs[i].source, graphs[i].sink};
    pbat_options oo;
    pbat_options_init(&oo);
    oo.walk_bits = std::min(o.walk_bits >= 0 ? o.walk_bits : kBsbMaxWalk, kBsbMaxWalk);
    oo.prune = o.prune;   // prune == 2: prune-aware prefix arcs
    // the gradient module divides walk-arc sums by p and 1 - p: only arcs
    // eligible under every p-vector may be walk arcs
    std::vector<double> pe;
    if (E.grad) {
      pe.resize(g.m);
      for (int a = 0; a < g.m; ++a) pe[a] = E.elig[i][a] == '1' ? 0.5 : 0.0;
    }
    int rc = bs_make_plan(g, oo, kBsbThreads, E.plans[i], E.grad ? pe.data() : nullptr);
    if (rc) return rc;
    items[i] = 1ull << E.plans[i].d;
    E.lmax = std::max(E.lmax, E.plans[i].L);
  }
  E.order.resize(G);
  for (int i = 0; i < G; ++i) E.order[i] = i;
  std::stable_sort(E.order.begin(), E.order.end(), [&](int a, int b) { return items[a] > items[b]; });
  // source: prelude, one struct per network (launch order), item template, kernel
  const std::string tmpl = kBsTemplate;
  E.minb = o.occupancy > 0 ? o.occupancy : kBsbMinBlocks;
  std::string src = "#define BSB_NTHR " + std::to_string(kBsbThreads) + "\n#define BSB_LMAX " +
                    std::to_string(E.lmax) + "\n#define BSB_MINB " + std::to_string(E.minb) + "\n" +
                    tmpl.substr(0, tmpl.find("//@@GENERATED@@"));
  for (int r = 0; r < G; ++r) {
    const BsPlan& bp = E.plans[E.order[r]];
    std::string gen = bp.gen;
    auto rep = [&](const std::string& a, const std::string& b) {
      const size_t at = gen.find(a);
      if (at != std::string::npos) gen.replace(at, a.size(), b);
    };
    rep("__device__ __forceinline__ void bs_inv(", "static __device__ __forceinline__ void inv(");
    rep("__device__ __forceinline__ u32 bs_var(", "static __device__ __forceinline__ u32 var(");
    const int m = graphs[E.order[r]].n_arcs;
    const unsigned lane_mask = bp.ell >= 5 ? 0xffffffffu : ((1u << (1 << bp.ell)) - 1u);
    char head[400];
    snprintf(head, sizeof head,
             "struct G%d {\n  static constexpr int M = %d, ELL = %d, TB = %d, L = %d, D = %d, NCORE = %d,"
             " WALK0 = %d, TOP = %d;\n  static constexpr u32 LANE_MASK = 0x%08xu;\n",
             r, m, bp.ell, bp.tb, bp.L, bp.d, bp.ncore, bp.ell + bp.tb, bp.ell + bp.tb + bp.L, lane_mask);
    src += head + gen + "};\n";
  }
  // shared memory: per-thread N_k bins, the item's connectivity words (and,
  // in the gradient module, their lane transposes), per-warp N_k counts
  std::string kern = E.grad ?
      "extern \"C\" __global__ void __launch_bounds__(BSB_NTHR, BSB_MINB)\n"
      "bs_batch_grad(const BGraph* __restrict__ graphs, int G, int K, int Kp, u64 total,\n"
      "         const u64* __restrict__ lt, const u64* __restrict__ nt, const u64* __restrict__ wm2,\n"
      "         const mx* __restrict__ pt, const u64* __restrict__ thw, const u64* __restrict__ tt,\n"
      "         const u64* __restrict__ lwex, const u64* __restrict__ thwex,\n"
      "         const mx* __restrict__ ptex, u64* limbs, u64* nk,\n"
      "         u64* counter, u32* status, u64 budget_ns) {\n"
      "  extern __shared__ __align__(16) u64 s_bins[];\n"
      "  const int lane = threadIdx.x & 31;\n"
      "  const BsTr tr = bs_tr_init(lane);\n"
      "  u64* bins = s_bins + threadIdx.x;\n"
      "  u32* cw = (u32*)(s_bins + (BSB_LMAX + 1) * BSB_NTHR) + threadIdx.x;\n"
      "  u32* ctw = (u32*)(s_bins + (BSB_LMAX + 1) * BSB_NTHR) + ((size_t)1 << BSB_LMAX) * BSB_NTHR +\n"
      "             threadIdx.x;\n"
      "  u64* nkw = s_bins + (BSB_LMAX + 1) * BSB_NTHR + ((size_t)1 << BSB_LMAX) * BSB_NTHR +\n"
      "             (threadIdx.x >> 5) * 65;\n"
      "  for (int i = lane; i < 65; i += 32) nkw[i] = 0ull;\n"
    :
      "extern \"C\" __global__ void __launch_bounds__(BSB_NTHR, BSB_MINB)\n"
      "bs_batch(const BGraph* __restrict__ graphs, int G, int K, int Kp, u64 total,\n"
      "         const u64* __restrict__ lt, const u64* __restrict__ nt, const u64* __restrict__ wm,\n"
      "         const mx* __restrict__ pt, const u64* __restrict__ thw, u64* limbs, u64* nk,\n"
      "         u64* counter, u32* status, u64 budget_ns) {\n"
      "  extern __shared__ __align__(16) u64 s_bins[];\n"
      "  const int lane = threadIdx.x & 31;\n"
      "  u64* bins = s_bins + threadIdx.x;\n"
      "  u32* cw = (u32*)(s_bins + (BSB_LMAX + 1) * BSB_NTHR) + threadIdx.x;\n"
      "  u64* nkw = s_bins + (BSB_LMAX + 1) * BSB_NTHR + (((size_t)1 << BSB_LMAX) * BSB_NTHR) / 2 +\n"
      "             (threadIdx.x >> 5) * 65;\n"
      "  for (int i = lane; i < 65; i += 32) nkw[i] = 0ull;\n";
  kern +=
      "  int cur = -1;   // network whose counts nkw holds\n"
      "  const u64 t0 = bs_timer();\n"
      "  for (;;) {\n"
      "    u64 task = 0;\n"
      "    if (lane == 0) {\n"
      "      task = atomicAdd(counter, 1ull);\n"
      "      if (budget_ns && bs_timer() - t0 > budget_ns) { atomicOr(status, 1u); task = ~0ull; }\n"
      "    }\n"
      "    task = __shfl_sync(0xffffffffu, task, 0);\n"
      "    if (task >= total) break;\n"
      "    int lo = 0, hi = G - 1;\n"
      "    while (lo < hi) { const int mid = (lo + hi + 1) >> 1; if (graphs[mid].task_begin <= task) lo = mid; else hi = mid - 1; }\n"
      "    const BGraph* __restrict__ Bp = graphs + lo;\n"
      "    if (lo != cur) {\n"
      "      __syncwarp();\n"
      "      if (cur >= 0) bsb_flush_counts(graphs + cur, nkw, nk, lane);\n"
      "      cur = lo;\n"
      "    }\n"
      "    const u64 prefix = task - Bp->task_begin;\n"
      "    const int prune = Bp->prune;\n"
      "    int st = 0;\n"
      "    switch (lo) {\n";
  for (int r = 0; r < G; ++r)
    kern += "      case " + std::to_string(r) + ": st = bsb_conn<G" + std::to_string(r) +
            ">(prefix, lane, prune, cw); break;\n";
  kern += "    }\n";
  kern += E.grad ?
          "    if (st) bsb_finish_grad(Bp, st, prefix, lane, K, Kp, lt, nt, wm2, pt, thw, tt, lwex, thwex,\n"
          "                            ptex, limbs, nkw, bins, cw, ctw, tr);\n" :
          "    if (st) bsb_finish(Bp, st, prefix, lane, K, Kp, lt, nt, wm, pt, thw, limbs, nkw, bins, cw);\n";
  kern +=
          "    __syncwarp();\n  }\n"
          "  __syncwarp();\n"
          "  if (cur >= 0) bsb_flush_counts(graphs + cur, nkw, nk, lane);\n}\n";
  std::string bt = kBsBatchTemplate;
  const size_t cut = bt.find("//@@BATCH_KERNEL@@");
  src += bt.substr(0, cut) + kern;
  src_out = src;
  return PBAT_OK;
}

// Descriptors, table layout (launch order), scratch and launch shape.
static int bsb_layout(BsBatch& E, int G, const pbat_graph* graphs, int K, const pbat_options& o,
                      const DeviceInfo& dev, const std::vector<unsigned long long>& items) {
  int rc;
  E.bg.resize(G);
  E.Kp = (K + 15) & ~15;   // whole chunks of 16 p-vectors per table row
  const int Kp = E.Kp;
  unsigned long long begin = 0;
  size_t lt = 0, nt = 0, wm = 0, pt = 0, th = 0;
  size_t wm2 = 0, tt = 0, lwex = 0, thwex = 0, ptex = 0, outl = 0;   // gradient module
  int nk_off = 0;
  std::vector<int> nk_offs(G);
  for (int i = 0; i < G; ++i) {
    nk_offs[i] = nk_off;
    nk_off += graphs[i].n_arcs + 1;
  }
  E.nk_total = nk_off;
  for (int r = 0; r < G; ++r) {
    const int i = E.order[r];
    const BsPlan& bp = E.plans[i];
    BGraphHost& b = E.bg[r];
    memset(&b, 0, sizeof b);
    b.task_begin = begin;
    b.n_tasks = items[i];
    begin += items[i];
    b.gidx = i;
    b.m = graphs[i].n_arcs;
    b.prune = o.prune ? 1 : 0;
    b.nlev = (bp.d + 6) / 7;   // levels of at most 7 bits: small per-p-vector tables
    int off = 0;
    for (int l = 0; l < b.nlev; ++l) {
      b.lev_bits[l] = bp.d / b.nlev + (l < bp.d % b.nlev ? 1 : 0);
      b.lev_off[l] = off;
      off += 1 << b.lev_bits[l];
    }
    b.pt_size = std::max(off, 1);
    for (int j = 0; j < 64; ++j) b.binom[j] = binom_u64(bp.ell + bp.tb + bp.L, j);
    b.lt_off = (int)lt; lt += (size_t)1024 * Kp;
    b.nt_off = (int)nt; nt += 1024;
    b.wm_off = (int)wm; wm += ((size_t)1 << bp.L) * Kp;
    b.pt_off = (int)pt; pt += (size_t)b.pt_size * K;
    b.thw_off = (int)th; th += (size_t)32 * Kp;
    b.nk_off = nk_offs[i];
    b.tb = bp.tb;
    b.L = bp.L;
    b.top = bp.ell + bp.tb + bp.L;
    b.lane_mask = bp.ell >= 5 ? 0xffffffffu : ((1u << (1 << bp.ell)) - 1u);
    b.full_counts = full_counts(bp.ell);
    b.ell = bp.ell;
    b.d = bp.d;
    b.thr_mask = bp.tb >= 5 ? 0xffffffffu : ((1u << (1 << bp.tb)) - 1u);
    b.pex_mask = bp.pex;
    if (E.grad) {
      b.wm2_off = (int)wm2; wm2 += (size_t)2 * ((size_t)1 << bp.L) * Kp;
      b.tt_off = (int)tt; tt += (size_t)1024 * Kp;
      b.lwex_off = (int)lwex; lwex += (size_t)5 * 32 * Kp;
      b.thwex_off = (int)thwex; thwex += (size_t)5 * 32 * Kp;
      b.ptex_off = (int)ptex; ptex += (size_t)K * bp.d * 128;
      b.out_off = (int)outl; outl += (size_t)K * (1 + 2 * b.m) * kBsbLimbs;
    }
  }
  E.total = begin;
  E.n_out = E.grad ? outl : (size_t)kBsbLimbs * G * K;
  E.n_lt = lt; E.n_nt = nt; E.n_wm = wm; E.n_pt = pt; E.n_thw = th;
  size_t off = 0;
  E.o_graphs = off; off = a256(off + sizeof(BGraphHost) * G);
  E.o_lt = off; off = a256(off + 8 * lt);
  E.o_nt = off; off = a256(off + 8 * nt);
  E.o_wm = off; off = a256(off + 8 * wm);
  E.o_pt = off; off = a256(off + sizeof(MxHost) * pt);
  E.o_thw = off; off = a256(off + 8 * th);
  E.o_wm2 = off; off = a256(off + 8 * wm2);
  E.o_tt = off; off = a256(off + 8 * tt);
  E.o_lwex = off; off = a256(off + 8 * lwex);
  E.o_thwex = off; off = a256(off + 8 * thwex);
  E.o_ptex = off; off = a256(off + sizeof(MxHost) * ptex);
  E.o_upload_end = off;
  E.o_limbs = off; off = a256(off + 8 * E.n_out);
  E.o_nk = off; off = a256(off + 8 * (size_t)E.nk_total);
  E.o_counter = off; off = a256(off + 8);
  E.o_status = off; off = a256(off + 4);
  E.o_end = off;
  if ((rc = scratch_acquire(dev.device, E.o_end, E.o_end, &E.scr))) return rc;
  memcpy((char*)E.scr->hmem + E.o_graphs, E.bg.data(), sizeof(BGraphHost) * G);
  E.smem = (size_t)(E.lmax + 1) * kBsbThreads * 8 +
           ((size_t)1 << E.lmax) * kBsbThreads * 4 * (E.grad ? 2 : 1) +
           (size_t)(kBsbThreads / 32) * 65 * 8;
  cudaError_t e = cudaFuncSetAttribute((const void*)E.jit.kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)E.smem);
  if (e != cudaSuccess) return fail(PBAT_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)E.jit.kernel, kBsbThreads,
                                                    E.smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const long long need = (long long)((E.total + kBsbThreads / 32 - 1) / (kBsbThreads / 32));
  E.grid = (int)std::max(1LL, std::min((long long)per_sm * dev.sms, need));
  return PBAT_OK;
}

static void bsb_tables(BsBatch& E, const pbat_graph* graphs, const double* p) {
  char* h = (char*)E.scr->hmem;
  unsigned long long* lt = (unsigned long long*)(h + E.o_lt);
  unsigned long long* nt = (unsigned long long*)(h + E.o_nt);
  unsigned long long* wm = (unsigned long long*)(h + E.o_wm);
  MxHost* pt = (MxHost*)(h + E.o_pt);
  unsigned long long* th = (unsigned long long*)(h + E.o_thw);
  unsigned long long* wm2t = (unsigned long long*)(h + E.o_wm2);
  unsigned long long* ttt = (unsigned long long*)(h + E.o_tt);
  unsigned long long* lwx = (unsigned long long*)(h + E.o_lwex);
  unsigned long long* thx = (unsigned long long*)(h + E.o_thwex);
  MxHost* ptx = (MxHost*)(h + E.o_ptex);
  const int K = E.K, Kp = E.Kp;
  std::vector<size_t> poff(E.G);
  size_t acc = 0;
  for (int i = 0; i < E.G; ++i) {
    poff[i] = acc;
    acc += (size_t)K * graphs[i].n_arcs;
  }
  // networks write disjoint table regions: build them on several host threads
  const int nthreads = std::max(1, std::min({E.G, 16, (int)std::thread::hardware_concurrency()}));
  auto build_range = [&](int r0, int r1) {
  for (int r = r0; r < r1; ++r) {
    const BGraphHost& b = E.bg[r];
    const int i = b.gidx, m = b.m;
    const BsPlan& bp = E.plans[i];
    const int top = bp.ell + bp.tb + bp.L;
    for (int v = 0; v < 1024; ++v) {  // packed N counts by lane class (same for every p-vector)
      const int by = v >> 8, val = v & 255;
      unsigned long long n = 0;
      for (int k = 0; k < 8; ++k) {
        const int j = 8 * by + k;
        if (!((val >> k) & 1) || j >= (1 << bp.ell)) continue;
        n += 1ull << kNkShift[__builtin_popcount((unsigned)j)];
      }
      nt[b.nt_off + v] = n;
    }
    for (int k = K; k < Kp; ++k) {  // padding p-vector: zero mass
      for (int v = 0; v < 1024; ++v) lt[b.lt_off + (size_t)v * Kp + k] = 0;
      for (int gi = 0; gi < (1 << bp.L); ++gi) wm[b.wm_off + (size_t)gi * Kp + k] = 0;
      for (int t = 0; t < 32; ++t) th[b.thw_off + (size_t)t * Kp + k] = 0;
    }
    for (int k = 0; k < K; ++k) {
      const double* pv = p + poff[i] + (size_t)k * m;
      dd lw[32], tw[32];
      for (int j = 0; j < 32; ++j) lw[j] = tw[j] = dd{0.0, 0.0};
      product_table(pv, bp.perm.data(), bp.ell, lw);
      byte_table_sums(lw, 1 << bp.ell, lt + b.lt_off + k, Kp);
      dd wtab[32];
      product_table(pv, bp.perm.data() + bp.ell + bp.tb, bp.L, wtab);
      for (int gi = 0; gi < (1 << bp.L); ++gi) wm[b.wm_off + (size_t)gi * Kp + k] = fixed_u64(wtab[gi], 63);
      product_table(pv, bp.perm.data() + bp.ell, bp.tb, tw);
      for (int t = 0; t < 32; ++t)
        th[b.thw_off + (size_t)t * Kp + k] = t < (1 << bp.tb) ? fixed_u64(tw[t], 63) : 0ull;
      MxHost* ptk = pt + b.pt_off + (size_t)k * b.pt_size;
      if (b.nlev == 0) ptk[0] = to_mx(dd_make(1.0));
      for (int l = 0, sh = 0; l < b.nlev; ++l) {
        dd tab[1 << 7];
        product_table(pv, bp.perm.data() + top + sh, b.lev_bits[l], tab);
        for (int v = 0; v < (1 << b.lev_bits[l]); ++v) ptk[b.lev_off[l] + v] = to_mx(tab[v]);
        if (E.grad)
          for (int jj = 0; jj < b.lev_bits[l]; ++jj) {
            if (!((bp.pex >> (top + sh + jj)) & 1ull)) continue;   // divided by p on the host
            // the level's product without prefix arc sh + jj, indexed by the
            // level value with that arc's bit removed
            int others[8];
            for (int x = 0, c = 0; x < b.lev_bits[l]; ++x)
              if (x != jj) others[c++] = bp.perm[top + sh + x];
            dd ex[1 << 6];
            product_table(pv, others, b.lev_bits[l] - 1, ex);
            MxHost* row = ptx + b.ptex_off + (((size_t)k * bp.d + sh + jj) << 7);
            for (int v = 0; v < (1 << b.lev_bits[l]); ++v)
              row[v] = to_mx(ex[(v & ((1 << jj) - 1)) | ((v >> (jj + 1)) << jj)]);
          }
        sh += b.lev_bits[l];
      }
      if (E.grad) {
        // 128-bit walk masses, thread-pattern byte tables, and the lane and
        // thread pattern masses without each of their arcs
        dd w2[32];
        product_table(pv, bp.perm.data() + bp.ell + bp.tb, bp.L, w2);
        for (int gi = 0; gi < (1 << bp.L); ++gi) {
          const u128 f = to_fixed127(w2[gi]);
          wm2t[b.wm2_off + ((size_t)gi * Kp + k) * 2] = f.lo;
          wm2t[b.wm2_off + ((size_t)gi * Kp + k) * 2 + 1] = f.hi;
        }
        byte_table_sums(tw, 1 << bp.tb, ttt + b.tt_off + k, Kp);
        auto excluded = [&](const int* arcs, int n, unsigned long long* out) {
          for (int x = 0; x < 5; ++x)
            for (int j = 0; j < 32; ++j) out[((size_t)(x * 32 + j)) * Kp + k] = 0ull;
          for (int x = 0; x < n; ++x) {
            int oth[5];
            for (int i = 0, c = 0; i < n; ++i)
              if (i != x) oth[c++] = arcs[i];
            dd tab[16];
            product_table(pv, oth, n - 1, tab);
            for (int j = 0; j < (1 << n); ++j)
              out[((size_t)(x * 32 + j)) * Kp + k] =
                  fixed_u64(tab[(j & ((1 << x) - 1)) | ((j >> (x + 1)) << x)], 63);
          }
        };
        excluded(bp.perm.data(), bp.ell, lwx + b.lwex_off);
        excluded(bp.perm.data() + bp.ell, bp.tb, thx + b.thwex_off);
      }
    }
  }
  };
  if (nthreads == 1) {
    build_range(0, E.G);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t)
    pool.emplace_back(build_range, E.G * t / nthreads, E.G * (t + 1) / nthreads);
  for (auto& th_ : pool) th_.join();
}

static int bsb_enqueue(BsBatch& E, cudaStream_t st, unsigned long long budget_ns) {
  char* d = (char*)E.scr->dmem;
  cudaError_t e = cudaMemsetAsync(d + E.o_limbs, 0, E.o_end - E.o_limbs, st);
  if (e != cudaSuccess) return fail(PBAT_ECUDA, "memset: %s", cudaGetErrorString(e));
  const void* graphs = d + E.o_graphs;
  const void *lt = d + E.o_lt, *nt = d + E.o_nt, *wm = d + E.o_wm, *pt = d + E.o_pt, *thw = d + E.o_thw;
  void *limbs = d + E.o_limbs, *nk = d + E.o_nk, *counter = d + E.o_counter, *status = d + E.o_status;
  int G = E.G, K = E.K, Kp = E.Kp;
  unsigned long long total = E.total, bud = budget_ns;
  const void *wm2 = d + E.o_wm2, *tt = d + E.o_tt, *lwex = d + E.o_lwex, *thwex = d + E.o_thwex;
  const void* ptex = d + E.o_ptex;
  void* args[] = {(void*)&graphs, &G, &K, &Kp, &total, (void*)&lt, (void*)&nt, (void*)&wm,
                  (void*)&pt, (void*)&thw, &limbs, &nk, &counter, &status, &bud};
  void* gargs[] = {(void*)&graphs, &G, &K, &Kp, &total, (void*)&lt, (void*)&nt, (void*)&wm2,
                   (void*)&pt, (void*)&thw, (void*)&tt, (void*)&lwex, (void*)&thwex, (void*)&ptex,
                   &limbs, &nk, &counter, &status, &bud};
  e = cudaLaunchKernel((const void*)E.jit.kernel, dim3(E.grid), dim3(kBsbThreads),
                       E.grad ? gargs : args, E.smem, st);
  if (e != cudaSuccess) return fail(PBAT_ECUDA, "batched launch: %s", cudaGetErrorString(e));
  return PBAT_OK;
}

static double bsb_limbs_value(const unsigned long long* limbs) {
  const dd v = limbs256_to_dd(limbs);
  return v.hi + v.lo;
}

// Source of the batched module (diagnostic; no device needed).
int bsb_source_for(int G, const pbat_graph* graphs, int K, const pbat_options& o,
                   const std::vector<std::string>* elig, std::string& out) {
  if (G > kBsbMaxGraphs) return fail(PBAT_ERANGE, "at most %d networks per bit-sliced batch", kBsbMaxGraphs);
  BsBatch E;
  if (elig) {
    E.grad = true;
    E.elig = *elig;
  }
  std::vector<unsigned long long> items;
  return bsb_source(E, G, graphs, K, o, items, out);
}

// The batch's walk length (split depth: each network's items are its
// prefixes of d = m - 10 - L arcs) and, with the prune on, its planning mode
// (source/sink-near or prune-aware prefix arcs): every candidate builds its
// module and runs the batch once; the fastest launch wins.  The gradient
// module (elig given) is tuned the same way.  The register cap is not
// tuned: on GB300 the 64-network workload ran fastest at the default launch
// bounds of 4 blocks per SM (R module 5.42 ms; 3, 6 and 2 blocks: 5.61, 6.82
// and 5.91 ms).  Returns false when no candidate ran (the planner's
// defaults are kept).
static bool bsb_tune(int G, const pbat_graph* graphs, int K, const double* p, const pbat_options& o,
                     cudaStream_t st, const DeviceInfo& dev, const std::vector<std::string>* elig,
                     int* best_L, int* best_prune, int* best_occ) {
  double best_ms = 1e300;
  bool found = false;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    cudaGetLastError();
    return false;
  }
  auto new_batch = [&](BsBatch& T) {
    if (elig) {
      T.grad = true;
      T.elig = *elig;
    }
  };
  // the candidates' modules compile at once on host threads
  auto precompile = [&](const std::vector<pbat_options>& cands) {
    std::vector<std::string> srcs;
    for (const pbat_options& t : cands) {
      BsBatch T;
      new_batch(T);
      std::vector<unsigned long long> items;
      std::string src;
      if (bsb_source(T, G, graphs, K, t, items, src) == PBAT_OK) srcs.push_back(std::move(src));
      else clear_error();
    }
    jit_precompile(srcs, dev.cc_major * 10 + dev.cc_minor);
  };
  auto run = [&](const pbat_options& t) {
    BsBatch T;
    new_batch(T);
    if (bsb_build(T, G, graphs, K, t, dev) != PBAT_OK) {
      if (T.scr) scratch_release(T.scr);
      clear_error();
      return;
    }
    bsb_tables(T, graphs, p);
    bool ok = cudaMemcpyAsync(T.scr->dmem, T.scr->hmem, T.o_upload_end, cudaMemcpyHostToDevice, st) ==
              cudaSuccess;
    ok = ok && cudaEventRecord(a, st) == cudaSuccess && bsb_enqueue(T, st, 0) == PBAT_OK &&
         cudaEventRecord(b, st) == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
    float ms = 0.f;
    if (ok && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      *best_L = t.walk_bits;
      *best_prune = t.prune;
      *best_occ = t.occupancy;
      found = true;
    }
    if (!ok) {
      cudaGetLastError();
      clear_error();
    }
    scratch_release(T.scr);
  };
  std::vector<pbat_options> cands;
  for (int mode : (o.prune == 1 ? std::vector<int>{1, 2} : std::vector<int>{o.prune}))
    for (int L = 3; L <= kBsbMaxWalk; ++L) {
      pbat_options t = o;
      t.walk_bits = L;
      t.prune = mode;
      t.occupancy = o.occupancy > 0 ? o.occupancy : 0;
      t.time_budget_s = 0;
      cands.push_back(t);
    }
  precompile(cands);
  for (const pbat_options& t : cands) run(t);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return found;
}

// R (and N_k) of a batch with the bit-sliced batched kernel; with `elig`
// (one string of '0'/'1' walk-arc eligibility per network) the gradient
// module also returns dR/dp in dRdp_out (the layout of p), and lists in
// *coarse the (network, p-vector) pairs whose R or gradient the
// fixed-point error bounds cannot certify to 1e-12 (the caller re-runs them
// exactly).  Returns PBAT_ENOTSUP when the batch is outside the module's
// limits (the caller then uses the frontier kernel).
int run_batched_bs(int G, const pbat_graph* graphs, int K, const double* p, const pbat_options& o,
                   cudaStream_t st, double* R_out, uint64_t* Nk_out, const std::string& key,
                   const DeviceInfo& dev, uint64_t* kernel_ns, const std::vector<std::string>* elig,
                   double* dRdp_out, std::vector<std::pair<int, int>>* coarse) {
  NvtxRange nv("pbat batched");
  if (G > kBsbMaxGraphs) return PBAT_ENOTSUP;
  BsBatch* E = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_bsb_mu);
    for (auto* e : g_bsb)
      if (!e->busy && e->key == key) { e->busy = true; E = e; break; }
  }
  if (!E) {
    pbat_options ob = o;
    if (o.autotune && o.walk_bits < 0) {
      int L = -1, mode = o.prune, occ = o.occupancy;
      if (bsb_tune(G, graphs, K, p, o, st, dev, elig, &L, &mode, &occ)) {
        ob.walk_bits = L;
        ob.prune = mode;
        ob.occupancy = occ;
      }
    }
    std::unique_ptr<BsBatch> ne(new BsBatch());
    ne->key = key;
    ne->busy = true;
    if (elig) {
      ne->grad = true;
      ne->elig = *elig;
    }
    int rc = bsb_build(*ne, G, graphs, K, ob, dev);
    if (rc) {
      if (ne->scr) scratch_release(ne->scr);
      return rc;
    }
    E = ne.release();
    std::lock_guard<std::mutex> lk(g_bsb_mu);
    g_bsb.push_back(E);
  }
  auto done = [&](int code) {
    std::lock_guard<std::mutex> lk(g_bsb_mu);
    E->busy = false;
    return code;
  };
  const unsigned long long budget = o.time_budget_s > 0 ? (unsigned long long)(o.time_budget_s * 1e9) : 0ull;
  bsb_tables(*E, graphs, p);
  char* d = (char*)E->scr->dmem;
  char* h = (char*)E->scr->hmem;
  if (cudaMemcpyAsync(d, h, E->o_upload_end, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return done(fail(PBAT_ECUDA, "upload failed: %s", cudaGetErrorString(cudaGetLastError())));
  if (!E->exec) {
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
      return done(fail(PBAT_ECUDA, "stream create failed"));
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const int erc = ok ? bsb_enqueue(*E, cs, budget) : PBAT_ECUDA;
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
  if (fault_at("launch")) return done(fail(PBAT_ECUDA, "injected fault: kernel launch"));
  // CUDA events around the replayed graph (its reset and kernel) give the
  // device time the caller can read from the statistics
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (kernel_ns && (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess)) {
    cudaGetLastError();
    if (ev0) cudaEventDestroy(ev0);
    ev0 = ev1 = nullptr;
  }
  if (ev0) cudaEventRecord(ev0, st);
  if (cudaGraphLaunch(E->exec, st) != cudaSuccess) {
    if (ev0) cudaEventDestroy(ev0), cudaEventDestroy(ev1);
    return done(fail(PBAT_ECUDA, "graph launch failed: %s", cudaGetErrorString(cudaGetLastError())));
  }
  if (ev0) cudaEventRecord(ev1, st);
  if (cudaMemcpyAsync(h + E->o_limbs, d + E->o_limbs, E->o_end - E->o_limbs, cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    if (ev0) cudaEventDestroy(ev0), cudaEventDestroy(ev1);
    return done(fail(PBAT_ECUDA, "batched run failed: %s", cudaGetErrorString(cudaGetLastError())));
  }
  if (ev0) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) *kernel_ns = (uint64_t)(ms * 1e6);
    else cudaGetLastError();
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
  }
  if (*(unsigned int*)(h + E->o_status) & 1u) return done(fail(PBAT_ETIMEOUT, "time budget ran out on the device"));
  const unsigned long long* limbs = (const unsigned long long*)(h + E->o_limbs);
  const unsigned long long* nk = (const unsigned long long*)(h + E->o_nk);
  if (!E->grad) {
    for (int r = 0; r < G; ++r) {
      const int i = E->bg[r].gidx;
      // absolute error of R: lane sums 2^-61, thread masses 2^-59, 64-bit
      // walk masses 2^(L-64), in units of the enumerated mass
      const double bound = ldexp(1.0, -61) + ldexp(1.0, -59) + ldexp(1.0, E->bg[r].L - 64);
      for (int k = 0; k < K; ++k) {
        const double R = bsb_limbs_value(limbs + ((size_t)i * K + k) * kBsbLimbs);
        R_out[(size_t)i * K + k] = R;
        if (coarse && R < 1e12 * bound) coarse->push_back({i, k});
      }
    }
  } else {
    // R, then A_q and B_q of every internal arc q per (network, p-vector):
    // dR/dp is A / p - B / (1 - p) for walk arcs and prefix arcs, except A -
    // B for prefix arcs outside [2^-20, 1 - 2^-20], and A for lane and
    // thread arcs (as for the single-network fused kernel)
    std::vector<size_t> poff(G);
    for (int i = 0, acc = 0; i < G; ++i) {
      poff[i] = (size_t)acc;
      acc += K * graphs[i].n_arcs;
    }
    for (int r = 0; r < G; ++r) {
      const BGraphHost& b = E->bg[r];
      const int i = b.gidx, m = b.m, top = b.top, walk0 = b.ell + b.tb;
      const BsPlan& bp = E->plans[i];
      for (int k = 0; k < K; ++k) {
        const unsigned long long* base = limbs + b.out_off + (size_t)k * (1 + 2 * m) * kBsbLimbs;
        const double* pk = p + poff[i] + (size_t)k * m;
        const dd Rd = limbs256_to_dd(base);
        const double R = Rd.hi + Rd.lo;
        R_out[(size_t)i * K + k] = R;
        // the single-network fused kernel's bounds: R within 2^-61 + 2^-59,
        // each gradient entry within 2^-57 (walk masses are 128-bit here)
        bool bad = R < 1e12 * (ldexp(1.0, -61) + ldexp(1.0, -59));
        const double Eg = ldexp(1.0, -57);
        for (int q = 0; q < m; ++q) {
          const dd A = limbs256_to_dd(base + (size_t)(1 + 2 * q) * kBsbLimbs);
          const dd B = limbs256_to_dd(base + (size_t)(2 + 2 * q) * kBsbLimbs);
          const int a = bp.perm[q];
          dd v;
          if (q >= top && ((bp.pex >> q) & 1ull))
            v = dd_sub(A, B);
          else if (q >= walk0)
            v = dd_sub(dd_mul(A, dd_recip(pk[a])), dd_mul(B, dd_recip_dd(dd_one_minus(pk[a]))));
          else
            v = A;
          const double g = v.hi + v.lo;
          dRdp_out[poff[i] + (size_t)k * m + a] = g;
          bad = bad || Eg > 1e-12 * std::max(std::fabs(g) - Eg, 1e-4 * R);
        }
        if (bad && coarse) coarse->push_back({i, k});
      }
    }
  }
  if (Nk_out) memcpy(Nk_out, nk, sizeof(uint64_t) * E->nk_total);
  return done(PBAT_OK);
}

}  // namespace pbat
