// pbat_noalloc.cu -- R and N_k without any device or pinned allocation.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// a framework's caching allocator or capped per process, and latency-critical
// paths that cannot afford the device-wide synchronisation an allocation may
// cause.  This entry point runs the same frontier enumeration kernel as
// pbat_reliability, but its scratch (work ticket, status, per-block
// partials, the walk-mass table, the reduced results) lives in one
// file-scope __device__ array of fixed size that every GPU loading this
// library keeps until the process exits.  Inputs and outputs are the
// caller's host arrays, as for pbat_reliability.
//
// Host code must not pass `g_noalloc_scratch` itself to a kernel: in host
// code that name is only a host-side stand-in.  Every call looks up its
// device address with cudaGetSymbolAddress, with the caller's device current
// (cheap, and it allocates nothing), so the address stays right even after
// the caller resets the device and the module is loaded again.
//
// All calls share the one array and it keeps the last call's contents; the
// ticket, status and statistics are cleared at the start of every call.
// Calls whose work overlapped on the GPU would race on the array, so the
// library holds one lock for the whole of each call (the call waits for its
// stream before it returns): calls from several host threads run one after
// another.  The walk-mass table is staged in a static host buffer under the
// same lock, so a call needs only a few KiB of the caller's stack.
//
// The call copies through host memory and waits for its stream, which stream
// capture does not allow: it refuses to run while its stream is capturing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "pbat.h"
#include "pbat_engine.h"
#include "pbat_internal.h"

namespace pbat {

size_t frontier_smem_bytes(int n, int m, int L, int nthr, bool grad, bool wide);
const void* frontier_kernel_ptr(bool grad, bool wide);
cudaError_t launch_frontier(bool grad, bool wide, int grid, int nthr, size_t smem,
                            cudaStream_t st, const FrontierParams& P, const u128* wmid,
                            const DevWork& W);
cudaError_t launch_reduce(cudaStream_t st, const DevWork& W, int nblocks, int n_acc, int n_cnt);

constexpr size_t kNoAllocScratchBytes = (size_t)512 << 10;  // 512 KiB
constexpr int kNoAllocMaxWalkBits = 12;                     // walk table <= 64 KiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
  void* base = nullptr;  // device address of g_noalloc_scratch on this device
  int sms = 0;
};
static int g_na_sms[kNoAllocMaxDevices];   // SM count per device, 0 = not yet read
static std::mutex g_na_mu;                 // held for the whole of every call
static u128 g_na_wmid[1 << kNoAllocMaxWalkBits];   // host staging of the walk table

// Fixed layout of the static scratch (byte offsets).
constexpr size_t kNaCounter = 0;     // u64 ticket; status at 16; stats at 32..55
constexpr size_t kNaOutAcc = 64;     // (1 + m) double-doubles, m <= 63
constexpr size_t kNaOutN = 1088;     // (m + 1) u64
constexpr size_t kNaWmid = 2048;     // 2^L u128 walk masses

// The scratch's device address on the current device (looked up on every
// call, with that device current) and its SM count (read once).  Called with
// g_na_mu held.
static int na_setup(int device, NoAllocDevice* out) {
  if (device < 0 || device >= kNoAllocMaxDevices)
    return fail(PBAT_ERANGE, "device %d is beyond the %d devices this entry point serves", device,
                kNoAllocMaxDevices);
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr)
    return fail(PBAT_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                cudaGetErrorString(e));
  if (!g_na_sms[device]) {
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return fail(PBAT_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    g_na_sms[device] = sms;
  }
  out->base = ptr;
  out->sms = g_na_sms[device];
  return PBAT_OK;
}

static int run_noalloc(const GraphIn& g, const double* p, const pbat_options* opt, void* stream,
                       double* R_out, uint64_t* Nk_out) {
  clear_error();
  if (!R_out) return fail(PBAT_EINVAL, "R_out must not be NULL");
  pbat_options o;
  pbat_options_init(&o);
  if (opt) o = *opt;
  int rc;
  if ((rc = validate_graph(g))) return rc;
  if ((rc = validate_p(p, g.m))) return rc;
  if ((rc = validate_options(opt, g.m))) return rc;
  if (o.algo == PBAT_ALGO_BITSLICE)
    return fail(PBAT_ENOTSUP, "this entry point runs the frontier kernel only");
  const int m = g.m, r = o.range_bits;
  // equal division (Sec. 4.3): lane, walk and prefix arcs; identity order,
  // so the state word is the paper's state index (Eq. 2)
  const int ell = std::min(kMaxLaneBits, m - r);
  const int free_bits = m - r - ell;
  int L;
  if (o.walk_bits >= 0) {
    if (o.walk_bits > kNoAllocMaxWalkBits)
      return fail(PBAT_ERANGE,
                  "walk_bits=%d needs a 2^%d-entry walk table; the static scratch holds at most "
                  "2^%d entries",
                  o.walk_bits, o.walk_bits, kNoAllocMaxWalkBits);
    L = std::min(o.walk_bits, free_bits);
  } else if (o.prefix_bits >= 0) {
    L = std::max(0, std::min(kNoAllocMaxWalkBits, m - ell - std::max(o.prefix_bits, r)));
  } else {
    L = std::max(0, std::min(kNoAllocMaxWalkBits, free_bits - std::max(0, 14 - r)));
  }
  const int d = m - ell - L;
  if (d >= 64) return fail(PBAT_ERANGE, "prefix of %d bits is too deep", d);

  cudaStream_t st = (cudaStream_t)stream;
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
      cudaGetLastError();
      return fail(PBAT_ECUDA, "cudaStreamIsCapturing failed");
    }
    if (cs != cudaStreamCaptureStatusNone)
      return fail(PBAT_ENOTSUP, "cannot run while its stream is being captured (the call copies "
                                "through host memory and waits for the stream)");
  }
  // one call at a time: the static device array and host staging are shared
  std::lock_guard<std::mutex> lk(g_na_mu);
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess)
    return fail(PBAT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(cudaGetLastError()));
  NoAllocDevice nd;
  if ((rc = na_setup(device, &nd))) return rc;

  // scratch budget: fixed header + walk table + per-block partials
  const size_t wmid_bytes = ((size_t)1 << L) * sizeof(u128);
  const size_t part_off = (kNaWmid + wmid_bytes + 255) & ~(size_t)255;
  const size_t per_block_acc = (size_t)(1 + m) * sizeof(dd);
  const size_t per_block = per_block_acc + (size_t)(m + 1) * 8;
  if (part_off + per_block > kNoAllocScratchBytes)
    return fail(PBAT_ERANGE, "needs more than the %zu B of static scratch", kNoAllocScratchBytes);
  const long long max_grid = (long long)((kNoAllocScratchBytes - part_off) / per_block);

  // kernel parameters on the host stack, the walk table in the static host
  // staging buffer (under the lock)
  FrontierParams P;
  memset(&P, 0, sizeof P);
  P.n = g.n;
  P.m = m;
  P.directed = g.directed ? 1 : 0;
  P.source = g.source;
  P.sink = g.sink;
  P.lane_bits = ell;
  P.walk_bits = L;
  P.prefix_bits = d;
  P.prune = o.prune ? 1 : 0;
  unsigned long long lo = 0, hi = 1ull << d;
  if (r > 0) {
    lo = o.range_lo << (d - r);
    hi = o.range_hi << (d - r);
  }
  P.task_lo = lo;
  P.n_tasks = hi - lo;
  P.budget_ns = o.time_budget_s > 0 ? (unsigned long long)(o.time_budget_s * 1e9) : 0ull;
  P.free_mask = ell + L >= 64 ? ~0ull : ((1ull << (ell + L)) - 1ull);
  for (int k = 0; k < m; ++k) {
    const int a = m - 1 - k;
    P.au[k] = (unsigned char)g.tail[a];
    P.av[k] = (unsigned char)g.head[a];
    P.p[k] = p[a];
    P.q[k] = dd_one_minus(p[a]);
  }
  for (int k = 0; k < m; ++k) {
    unsigned long long gm = 0;
    for (int j = 0; j < m; ++j) {
      const bool same = g.directed ? (P.au[k] == P.au[j] && P.av[k] == P.av[j])
                                   : ((P.au[k] == P.au[j] && P.av[k] == P.av[j]) ||
                                      (P.au[k] == P.av[j] && P.av[k] == P.au[j]));
      if (same) gm |= 1ull << j;
    }
    P.grp[k] = gm;
  }
  for (int j = 0; j < 32; ++j) {
    if (j >= (1 << ell)) {
      P.lane_w[j] = dd{0.0, 0.0};
      continue;
    }
    dd w = dd_make(1.0);
    for (int i = 0; i < ell; ++i) w = dd_mul(w, arc_w(p, m - 1 - i, (j >> i) & 1));
    P.lane_w[j] = w;
  }
  for (int j = 0; j < 64; ++j) P.binom[j] = binom_u64(ell + L, j);
  u128* wmid = g_na_wmid;
  for (int gi = 0; gi < (1 << L); ++gi) {
    dd w = dd_make(1.0);
    for (int b = 0; b < L; ++b) w = dd_mul(w, arc_w(p, m - 1 - (ell + b), (gi >> b) & 1));
    wmid[gi] = to_fixed127(w);
  }

  // launch shape: persistent grid, clamped to the partials that fit
  const bool wide = g.n > 32;
  const int nthr = o.block_threads > 0 ? o.block_threads : 128;
  const size_t smem = frontier_smem_bytes(g.n, m, L, nthr, false, wide);
  const void* kfn = frontier_kernel_ptr(false, wide);
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return fail(PBAT_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, nthr, smem);
  if (e != cudaSuccess || per_sm < 1)
    return fail(PBAT_ERANGE, "frontier kernel cannot be resident (smem %zu B)", smem);
  const long long need = (long long)((std::min<unsigned long long>(P.n_tasks, 1ull << 40) +
                                      nthr / 32 - 1) / (nthr / 32));
  const int grid = (int)std::max(1LL, std::min({(long long)per_sm * nd.sms, need, max_grid}));

  char* base = (char*)nd.base;
  DevWork W{};
  W.counter = (unsigned long long*)(base + kNaCounter);
  W.status = (unsigned int*)(base + kNaCounter + 16);
  W.stats = (unsigned long long*)(base + kNaCounter + 32);
  W.out_acc = (dd*)(base + kNaOutAcc);
  W.out_n = (unsigned long long*)(base + kNaOutN);
  W.part_acc = (dd*)(base + part_off);
  W.part_n = (unsigned long long*)(base + part_off + (size_t)grid * per_block_acc);
  W.wacc = nullptr;   // the frontier kernel keeps its accumulators in registers
  W.out_limbs = nullptr;
  const u128* d_wmid = (const u128*)(base + kNaWmid);

  // the copy from this pageable buffer returns once the buffer has been staged
  if ((e = cudaMemcpyAsync((void*)d_wmid, wmid, wmid_bytes, cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemsetAsync(base + kNaCounter, 0, 64, st)) ||
      (e = launch_frontier(false, wide, grid, nthr, smem, st, P, d_wmid, W)) ||
      (e = launch_reduce(st, W, grid, 1 + m, m + 1)))
    return fail(PBAT_ECUDA, "enqueue failed: %s", cudaGetErrorString(e));
  dd acc[1 + kMaxArcs];
  unsigned long long nk[kMaxArcs + 1];
  unsigned int status = 0;
  if ((e = cudaMemcpyAsync(acc, W.out_acc, sizeof(dd), cudaMemcpyDeviceToHost, st)) ||
      (e = cudaMemcpyAsync(nk, W.out_n, (size_t)(m + 1) * 8, cudaMemcpyDeviceToHost, st)) ||
      (e = cudaMemcpyAsync(&status, W.status, 4, cudaMemcpyDeviceToHost, st)) ||
      (e = cudaStreamSynchronize(st)))
    return fail(PBAT_ECUDA, "enumeration failed: %s", cudaGetErrorString(e));
  if (status & 1u) return fail(PBAT_ETIMEOUT, "time budget ran out on the device");
  *R_out = acc[0].hi + acc[0].lo;
  if (Nk_out)
    for (int k = 0; k <= m; ++k) Nk_out[k] = nk[k];
  return PBAT_OK;
}

}  // namespace pbat

extern "C" int pbat_reliability_noalloc(int n_nodes, int n_arcs, const int32_t* tail,
                                        const int32_t* head, int directed, const double* p,
                                        int source, int sink, const pbat_options* opt,
                                        void* cuda_stream, double* R_out, uint64_t* Nk_out) {
  try {
    pbat::GraphIn g{n_nodes, n_arcs, tail, head, directed, source, sink};
    return pbat::run_noalloc(g, p, opt, cuda_stream, R_out, Nk_out);
  } catch (...) {
    return pbat::fail(PBAT_ENOMEM, "host exception");
  }
}
