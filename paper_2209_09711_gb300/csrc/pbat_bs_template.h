// pbat_bs_template.h -- CUDA source of the bit-sliced enumeration kernels.
//
// The engine prepends a block of #defines and the graph-specific
// connectivity functions (bs_inv / bs_var, written by the planner in
// pbat_bs_plan.cu) and compiles the result with NVRTC for sm_103a.
//
// State layout: bit j of a thread's 32-bit word is the state whose BS_ELL
// lane arcs follow the bits of j; the BS_TB thread arcs follow the bits of
// the warp lane id; the BS_L walk arcs follow the walk index g; the BS_D
// prefix arcs are fixed per work item (one item per warp, from an atomic
// ticket: the equal division of Sec. 4.3).  The walk visits g in reflected
// Gray order over its upper BS_L - BS_IN bits and, for each such step, all
// 2^BS_IN settings of its lowest bits in an unrolled block whose walk words
// are compile-time constants that fold through the connectivity program.
//
// Per word the connectivity of its 32 states is c = bs_var(inv, walk words):
// bit j set iff the sink is reachable from the source in state j (the PLSA
// answer of Sec. 3.2).  R (Eq. 1) accumulates exactly: the lane mass of the
// connected bits comes from four byte tables (u64, scale 2^62, each entry
// paired with the bit counts of its lane-popcount classes so that one 16-byte
// load serves R and N_k), times the walk mass of g, into a 128-bit integer T
// per thread (scale 2^125); the thread-arc and prefix masses are applied once
// per item, in integer arithmetic (the FP64 rate of this part is 1/64 of its
// FP32 rate, so no per-item work uses FP64).
#pragma once

namespace pbat {

static const char* kBsTemplate = R"PBAT(
typedef unsigned int u32;
typedef unsigned long long u64;

#define BS_IN (BS_L >= BS_IN_BITS ? BS_IN_BITS : BS_L)
// launch bounds of the single-network kernels: with BS_MINB blocks per SM
// requested, the compiler keeps registers within 65536 / (BS_MINB * BS_NTHR)
#if defined(BS_MINB) && BS_MINB > 0
#define KERNEL_BOUNDS __launch_bounds__(BS_NTHR, BS_MINB)
#else
#define KERNEL_BOUNDS __launch_bounds__(BS_NTHR)
#endif
// the first of two launches (prune and closed-form sums, no walk) is compiled
// for at least 24 resident warps per SM: on GB300 it needs about 80 registers
// then, without spills
#if defined(BS_MINB) && BS_MINB > 768 / BS_NTHR
#define KERNEL_BOUNDS_P1 __launch_bounds__(BS_NTHR, BS_MINB)
#else
#define KERNEL_BOUNDS_P1 __launch_bounds__(BS_NTHR, (768 / BS_NTHR > 0 ? 768 / BS_NTHR : 1))
#endif
#define BS_OUT (BS_L - BS_IN)

struct dd { double hi, lo; };   // host-side double-double (only carried, never computed here)

struct u128 { u64 lo, hi; };
__device__ __forceinline__ void u128_add(u128& a, u64 blo, u64 bhi) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(blo), "l"(bhi));
}
__device__ __forceinline__ u128 u128_sub(u128 a, u128 b) {
  u128 r;
  asm("sub.cc.u64 %0, %2, %4;\n\tsubc.u64 %1, %3, %5;" : "=l"(r.lo), "=l"(r.hi) : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
  return r;
}
// (a * b) >> 64 for a 64-bit a and a 128-bit b (the lowest 64 bits dropped)
__device__ __forceinline__ u128 mul64x128_shr64(u64 a, u64 blo, u64 bhi) {
  const u64 h0 = __umul64hi(a, blo);
  const u64 l1 = a * bhi;
  const u64 h1 = __umul64hi(a, bhi);
  u128 r;
  asm("add.cc.u64 %0, %2, %3;\n\taddc.u64 %1, %4, 0;" : "=l"(r.lo), "=l"(r.hi) : "l"(l1), "l"(h0), "l"(h1));
  return r;
}
__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int m) {
  u128 r;
  r.lo = __shfl_xor_sync(0xffffffffu, v.lo, m);
  r.hi = __shfl_xor_sync(0xffffffffu, v.hi, m);
  return r;
}
// exact sum over the warp (every lane gets it)
#if defined(BS_GRAD) && BS_GRAD && !BS_ACC_REG
// the fused kernel with a large connectivity program: five rounds of 128-bit
// shuffles (the hardware reductions below measured 2% slower there)
__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const u128 w = shfl_xor_u128(v, o);
    u128_add(v, w.lo, w.hi);
  }
  return v;
}
#else
// the value in five chunks of at most 26 bits, whose 32-lane sums fit 31
// bits, one hardware warp reduction each, recombined in 128-bit arithmetic
// (GB300, against five rounds of 128-bit shuffles: 40-arc R kernel 87.7 ->
// 73.0 ms, 34-arc directed 490 -> 472 us)
__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
  const u32 c0 = (u32)(v.lo & 0x3ffffffull), c1 = (u32)((v.lo >> 26) & 0x3ffffffull);
  const u32 c2 = (u32)(((v.lo >> 52) | (v.hi << 12)) & 0x3ffffffull);
  const u32 c3 = (u32)((v.hi >> 14) & 0x3ffffffull), c4 = (u32)(v.hi >> 40);
  const u64 s0 = __reduce_add_sync(0xffffffffu, c0), s1 = __reduce_add_sync(0xffffffffu, c1);
  const u64 s2 = __reduce_add_sync(0xffffffffu, c2), s3 = __reduce_add_sync(0xffffffffu, c3);
  const u64 s4 = __reduce_add_sync(0xffffffffu, c4);
  u128 r = u128{s0, 0ull};
  u128_add(r, s1 << 26, 0ull);
  u128_add(r, s2 << 52, s2 >> 12);
  u128_add(r, 0ull, s3 << 14);
  u128_add(r, 0ull, s4 << 40);
  return r;
}
#endif

__device__ __forceinline__ u128 u128_shr(u128 v, int s) {
  if (s <= 0) return v;
  if (s >= 128) return u128{0ull, 0ull};
  if (s >= 64) return u128{v.hi >> (s - 64), 0ull};
  return u128{(v.lo >> s) | (v.hi << (64 - s)), v.hi >> s};
}

// Products of arc reliabilities (the prefix masses) as integer floating
// point: value m * 2^(-63 - e), m in [2^63, 2^64) or m = 0, e >= 0.  A
// product keeps 63 significant bits.
struct mx { u64 m; int e; int pad; };
__device__ __forceinline__ mx mx_mul(mx a, mx b) {
  u64 h = __umul64hi(a.m, b.m);
  int e = a.e + b.e - 1;
  if (!(h >> 63)) { h <<= 1; ++e; }
  return mx{h, e, 0};
}
// x times a 128-bit value v at scale 2^124 is mx_prod(x, v) * 2^(-123 - x.e)
// (truncated; below 2^124)
__device__ __forceinline__ u128 mx_prod(mx x, u128 v) { return mul64x128_shr64(x.m, v.lo, v.hi); }

// Floating 128-bit accumulator: value v * 2^(-123 - E) with v < 2^126, so a
// sum of items keeps about 125 significant bits relative to its own size,
// whatever the mass of the enumerated range.
struct facc { u128 v; int E; int pad; };
__device__ __forceinline__ void facc_add(facc& a, u128 P, int e) {
  if (!(P.lo | P.hi)) return;
  if (!(a.v.lo | a.v.hi)) { a.v = P; a.E = e; return; }
  if (e >= a.E) {
    const u128 q = u128_shr(P, e - a.E);
    u128_add(a.v, q.lo, q.hi);
  } else {
    a.v = u128_shr(a.v, a.E - e);
    a.E = e;
    u128_add(a.v, P.lo, P.hi);
  }
  if (a.v.hi >> 62) { a.v = u128_shr(a.v, 1); a.E -= 1; }
}

// add v * 2^(s - 250) to a 256-bit fixed-point number held as 32-bit chunks
// in eight 64-bit limbs (the upper halves absorb the carries); v < 2^127 and
// s <= 129 keep it below 2^256
__device__ __forceinline__ void bs_limb_add(u64* limbs, u128 v, int s) {
  if (s < 0) {
    v = u128_shr(v, -s);
    s = 0;
  }
  if (!(v.lo | v.hi)) return;
  const int c0 = s >> 5, r = s & 31;
  const u64 q0 = v.lo << r;
  const u64 q1 = r ? ((v.hi << r) | (v.lo >> (64 - r))) : v.hi;
  const u64 q2 = r ? (v.hi >> (64 - r)) : 0ull;
  const u64 c[5] = {q0 & 0xffffffffull, q0 >> 32, q1 & 0xffffffffull, q1 >> 32, q2};
#pragma unroll
  for (int i = 0; i < 5; ++i)
    if (c[i] && c0 + i < 8) atomicAdd(&limbs[c0 + i], c[i]);
}

// N_k counts of one word, packed by lane-popcount class cl = 0..5 into
// fields of 8, 11, 12, 12, 11 and 8 bits: wide enough for one item's sum
// over 2^L words with L <= 10 (at most C(10,5) * C(5,cl) per field).
#define BS_NK_SHIFTS {0, 8, 19, 31, 43, 54}
#define BS_NK_WIDTHS {8, 11, 12, 12, 11, 8}

struct BsParams {
  u64 task_lo, n_tasks, budget_ns;
  int prune, nlev;       // prefix-mass table levels
  int ex_shift, pad;     // log2 of the excluded-arc table's row length
  int lev_bits[10];      // prefix bits per level (low level first)
  int lev_off[10];       // first entry of each level in the prefix table
  u64 thw[32];           // thread-pattern masses, fixed point 2^63
  u64 binom[64];
};
struct facc;
struct BsWork {
  u64* counter; u32* status; u64* stats;
  dd* part_acc; u64* part_n; dd* out_acc; u64* out_n;
  facc* wacc;       // fused kernel: per warp, R and the two sums of every arc
  u64* out_limbs;   // [n_acc][8]: 256-bit fixed point at scale 2^250, 32 bits per limb
  u64* list;        // two-launch runs: items deferred to the walking launch
  u64 list_cap;     // 0: one-launch run
  u64* list_n;
  u64* counter2;    // ticket of the walking launch
};

// Work items of a launch.  One-launch runs (phase 0) take items by the
// atomic ticket over [0, n_tasks).  Two-launch runs: the first (phase 1)
// takes items 16 at a time -- a warp's first 16 fixed by its index, the
// rest by an atomic ticket (its items are short: one ticket per item would
// pack 2^21 atomics on one counter into the launch, and a fixed warp stride
// gave warps runs of alike items that end unevenly) -- resolves what the
// prune can and defers the items left to walk; the second (phase 2) takes
// the deferred items by a ticket over the list.  ~0: no item left.
__device__ __forceinline__ u64 bs_list_task(const BsWork& W) {
  const u64 i = atomicAdd(W.counter2, 1ull);
  return i < *W.list_n ? W.list[i] : ~0ull;
}
// The walking launch: true (in every thread of the block) when no deferred
// item is left for it -- the list is empty, or blocks that started earlier
// have taken every ticket -- so the block returns before it stages tables or
// clears accumulators (it would add nothing to the results).
__device__ __forceinline__ bool bs_list_done(const BsWork& W) {
  __shared__ int s_done;
  if (threadIdx.x == 0)
    s_done = *(volatile const u64*)W.counter2 >= *(volatile const u64*)W.list_n;
  __syncthreads();
  return s_done != 0;
}

// Phase 1: a warp collects its deferred items one per lane (entry j in lane
// j) and appends them to the list 32 at a time, with one atomic per batch.
// The list holds every item (list_cap = n_tasks), so it cannot overflow.
__device__ __forceinline__ void bs_flush_deferred(const BsWork& W, u64 pend, int npend, int lane) {
  if (!npend) return;
  u64 base = 0;
  if (lane == 0) base = atomicAdd(W.list_n, (u64)npend);
  base = __shfl_sync(0xffffffffu, base, 0);
  if (lane < npend) W.list[base + lane] = pend;
}

__device__ __forceinline__ u64 bs_timer() {
  u64 t; asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t)); return t;
}

// Mass of the prefix arcs of `prefix`: product over table levels.
__device__ __forceinline__ mx bs_prefix_mass(const BsParams& P, const mx* __restrict__ ptab, u64 prefix) {
  mx w = mx{1ull << 63, 0, 0};
  int sh = 0;
  for (int l = 0; l < P.nlev; ++l) {
    const u64 v = (prefix >> sh) & ((1ull << P.lev_bits[l]) - 1ull);
    const mx t = ptab[P.lev_off[l] + v];
    w = l ? mx_mul(w, t) : t;
    sh += P.lev_bits[l];
  }
  return w;
}
// Per-lane constants of the 32x32 bit transpose below: byte selectors of the
// 16- and 8-bit rounds, rotate amounts and keep-masks of the 4-, 2- and
// 1-bit rounds.
struct BsTr { u32 sel16, sel8, rot4, rot2, rot1, keep4, keep2, keep1; };
__device__ __forceinline__ BsTr bs_tr_init(int lane) {
  BsTr t;
  t.sel16 = (lane & 16) ? 0x3276u : 0x5410u;
  t.sel8 = (lane & 8) ? 0x3715u : 0x6240u;
  t.rot4 = (lane & 4) ? 28u : 4u;
  t.rot2 = (lane & 2) ? 30u : 2u;
  t.rot1 = (lane & 1) ? 31u : 1u;
  t.keep4 = (lane & 4) ? 0xF0F0F0F0u : 0x0F0F0F0Fu;
  t.keep2 = (lane & 2) ? 0xCCCCCCCCu : 0x33333333u;
  t.keep1 = (lane & 1) ? 0xAAAAAAAAu : 0x55555555u;
  return t;
}
// Round with distance sh: lanes with bit sh clear keep the low half of
// every 2sh-bit group and take the partner's low halves into their high
// halves; lanes with the bit set keep the high halves and take the
// partner's high halves into their low halves.  Byte-sized rounds are one
// byte permute; smaller ones a rotate and a bit select.
__device__ __forceinline__ u32 bs_transpose32(u32 x, const BsTr& t) {
  u32 y = __shfl_xor_sync(0xffffffffu, x, 16);
  x = __byte_perm(x, y, t.sel16);
  y = __shfl_xor_sync(0xffffffffu, x, 8);
  x = __byte_perm(x, y, t.sel8);
  y = __shfl_xor_sync(0xffffffffu, x, 4);
  x = (x & t.keep4) | (__funnelshift_l(y, y, t.rot4) & ~t.keep4);
  y = __shfl_xor_sync(0xffffffffu, x, 2);
  x = (x & t.keep2) | (__funnelshift_l(y, y, t.rot2) & ~t.keep2);
  y = __shfl_xor_sync(0xffffffffu, x, 1);
  x = (x & t.keep1) | (__funnelshift_l(y, y, t.rot1) & ~t.keep1);
  return x;
}

//@@GENERATED@@
// connectivity of one uniform state (every word 0 or ~0): the prune test
__device__ __forceinline__ u32 bs_uniform(const u32* a) {
  u32 e[BS_NCORE > 0 ? BS_NCORE : 1];
  bs_inv(a, e);
  u32 w[BS_L > 0 ? BS_L : 1];
#pragma unroll
  for (int b = 0; b < BS_L; ++b) w[b] = a[BS_WALK0 + b];
  return bs_var(e, w);
}

__device__ __forceinline__ void bs_init_arcs(u32* a, int lane) {
#pragma unroll
  for (int i = 0; i < BS_ELL; ++i)
    a[i] = i == 0 ? 0xAAAAAAAAu : i == 1 ? 0xCCCCCCCCu : i == 2 ? 0xF0F0F0F0u : i == 3 ? 0xFF00FF00u : 0xFFFF0000u;
#pragma unroll
  for (int i = 0; i < BS_TB; ++i) a[BS_ELL + i] = 0u - (u32)((lane >> i) & 1);
#pragma unroll
  for (int b = 0; b < BS_L; ++b) a[BS_WALK0 + b] = 0u;
}

// 0: walk the item, 1: every state disconnected, 2: every state connected.
// One bit-sliced evaluation answers both extremes: bit 0 has every arc below
// the prefix working, bit 1 every such arc failed (the prefix arcs are the
// same in every bit).
__device__ __forceinline__ int bs_prune(const u32* a) {
  u32 u[BS_M];
#pragma unroll
  for (int k = 0; k < BS_M; ++k) u[k] = k < BS_TOP ? 1u : a[k];
  const u32 ext = bs_uniform(u);
  if (!(ext & 1u)) return 1;
  return (ext & 2u) ? 2 : 0;
}

__device__ __forceinline__ void bs_flush_bins(u64* bins, u64* s_nbins, int base) {
  constexpr int sh[6] = BS_NK_SHIFTS, wd[6] = BS_NK_WIDTHS;
#pragma unroll 1
  for (int r = 0; r <= BS_L; ++r) {
    const u64 n = bins[r * BS_NTHR];
#pragma unroll
    for (int cl = 0; cl < 6; ++cl) {
      const u64 c = (n >> sh[cl]) & ((1ull << wd[cl]) - 1ull);
      if (c) atomicAdd(&s_nbins[base + r + cl], c);
    }
  }
}

// End of a block: entry i combines the warps' floating accumulators
// s_acc[w * stride + i] in integer arithmetic and adds the sum to the result
// with integer atomics (every sum is non-negative, and integer addition is
// exact, so the order of the blocks does not matter); then the block's N_k
// counts.  The host converts the result once.
__device__ __forceinline__ void bs_write_out(const BsWork& W, const facc* s_acc, int stride, int n_acc,
                                             const u64* s_nbins) {
  for (int i = threadIdx.x; i < n_acc; i += BS_NTHR) {
    facc t = s_acc[i];
    for (int w = 1; w < BS_NTHR / 32; ++w) facc_add(t, s_acc[w * stride + i].v, s_acc[w * stride + i].E);
    bs_limb_add(W.out_limbs + 8 * i, t.v, 127 - t.E);   // v * 2^(-123 - E) at scale 2^250
  }
  for (int i = threadIdx.x; i <= BS_M; i += BS_NTHR)
    if (s_nbins[i]) atomicAdd(&W.out_n[i], s_nbins[i]);
}

// ---------------------------------------------------------------------------
// R + N_k
// ---------------------------------------------------------------------------
#if !BS_GRAD
// PHASE 0: a one-launch run; 1 and 2: the two launches of a two-launch run
// (the first resolves what the prune can and defers the items left to walk,
// the second walks them).  One entry point per phase, so that a one-launch
// kernel carries none of the two-launch state in its registers.
template <int PHASE>
__device__ __forceinline__ void bs_kernel_body(const BsParams& P, const u64* __restrict__ lane_tab,
                                               const u64* __restrict__ wmid_tab,
                                               const mx* __restrict__ ptab, const BsWork& W) {
  extern __shared__ __align__(16) unsigned char smem[];
  ulonglong2* s_lt = (ulonglong2*)smem;                     // [4][256] {lane mass 2^62, packed counts}
  u64* s_wmid = (u64*)(s_lt + 4 * 256);                     // [2^L], scale 2^63
  u64* s_bins = s_wmid + (1 << BS_L);                       // [L + 1][NTHR]
  facc* s_acc = (facc*)(s_bins + (BS_L + 1) * BS_NTHR);     // [warps]: each warp's R
  u64* s_nbins = (u64*)(s_acc + BS_NTHR / 32);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if constexpr (PHASE == 2) {
    if (bs_list_done(W)) return;
  }
  for (int i = tid; i < 4 * 256; i += BS_NTHR) s_lt[i] = ((const ulonglong2*)lane_tab)[i];
  for (int i = tid; i < (1 << BS_L); i += BS_NTHR) s_wmid[i] = wmid_tab[i];
  for (int i = tid; i <= BS_M; i += BS_NTHR) s_nbins[i] = 0ull;
  __syncthreads();
  u64* bins = s_bins + tid;
  const bool thr_on = lane < (1 << BS_TB);
  const int pc_thr = __popc(lane & ((1 << BS_TB) - 1));
  const u64 thw = thr_on ? P.thw[lane] : 0ull;
  const u64 t_start = bs_timer();
  u64 n_walk = 0, n_full = 0, n_dead = 0;
  facc accR = facc{u128{0ull, 0ull}, 0, 0};   // this warp's R (the same in every lane)
  u32 a[BS_M];
  bs_init_arcs(a, lane);
  constexpr int phase = PHASE;
  // phase 1: this warp's chunk of items -- its first chunk is its own (no
  // ticket at the start of a short launch), the later ones come by ticket
  u64 chunk_next = ((u64)blockIdx.x * (BS_NTHR / 32) + warp) * 16, chunk_end = chunk_next + 16;
  u64 pend = 0;   // phase 1: this warp's deferred items, entry j in lane j
  int npend = 0;

  for (;;) {
    u64 task = 0;
    if constexpr (phase == 1) {
      if (chunk_next == chunk_end) {   // the next 16 items, by one atomic ticket
        u64 base = 0;
        if (lane == 0) base = (u64)gridDim.x * (BS_NTHR / 32) * 16 + atomicAdd(W.counter, 16ull);
        chunk_next = __shfl_sync(0xffffffffu, base, 0);
        chunk_end = chunk_next + 16;
      }
      task = chunk_next++;
    }
    if (lane == 0) {
      if constexpr (phase == 2) task = bs_list_task(W);
      else if constexpr (phase == 0) task = atomicAdd(W.counter, 1ull);
      if (P.budget_ns && bs_timer() - t_start > P.budget_ns) { atomicOr(W.status, 1u); task = ~0ull; }
    }
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= P.n_tasks) break;
    const u64 prefix = P.task_lo + task;
#pragma unroll
    for (int j = 0; j < BS_D; ++j) a[BS_TOP + j] = 0u - (u32)((prefix >> j) & 1ull);
    const int pc_pre = __popcll((long long)prefix);
    if ((P.prune && phase == 0) || phase == 1) {   // two-launch runs always prune
      const int pr = bs_prune(a);
      if (pr == 1) { ++n_dead; continue; }
      if (pr == 2) {
        ++n_full;
        for (int j = lane; j <= BS_TOP; j += 32) atomicAdd(&s_nbins[pc_pre + j], P.binom[j]);
        const mx w = bs_prefix_mass(P, ptab, prefix);
        facc_add(accR, mx_prod(w, u128{0ull, 1ull << 60}), w.e);
        continue;
      }
    }
    if constexpr (phase == 1) {   // left to walk: deferred to the second launch
      if (lane == npend) pend = task;
      if (++npend == 32) { bs_flush_deferred(W, pend, npend, lane); npend = 0; }
      continue;
    }
    ++n_walk;
    u32 e[BS_NCORE > 0 ? BS_NCORE : 1];
    bs_inv(a, e);
#pragma unroll
    for (int r = 0; r <= BS_L; ++r) bins[r * BS_NTHR] = 0ull;
    u128 T = u128{0ull, 0ull};
    u32 gout = 0;
    int pco = 0;
#pragma unroll 1
    for (u32 s = 0; s < (1u << BS_OUT); ++s) {
      if (s) {
        const int b = __ffs(s) - 1;
        gout ^= 1u << b;
        pco += ((gout >> b) & 1u) ? 1 : -1;
      }
      u32 w[BS_L > 0 ? BS_L : 1];
#pragma unroll
      for (int b = 0; b < BS_OUT; ++b) w[BS_IN + b] = 0u - ((gout >> b) & 1u);
#pragma unroll
      for (int r = 0; r < (1 << BS_IN); ++r) {
#pragma unroll
        for (int b = 0; b < BS_IN; ++b) w[b] = ((r >> b) & 1) ? ~0u : 0u;
        const u32 c = bs_var(e, w) & BS_LANE_MASK;
        // one warp vote, as in the fused kernel: when some word of the warp
        // is partly connected every word reads its lane-table entries (a
        // cut word the zero entries); otherwise each word is cut or fully
        // connected
        if (__any_sync(0xffffffffu, c != 0u && c != BS_LANE_MASK)) {
          const u32 g = (gout << BS_IN) | (u32)r;
          const int pc = pco + __popc(r);
          const ulonglong2 t0 = s_lt[0 * 256 + (c & 0xffu)], t1 = s_lt[1 * 256 + ((c >> 8) & 0xffu)];
          const ulonglong2 t2 = s_lt[2 * 256 + ((c >> 16) & 0xffu)], t3 = s_lt[3 * 256 + (c >> 24)];
          const u64 sR = t0.x + t1.x + t2.x + t3.x;
          const u64 wm = s_wmid[g];
          u128_add(T, sR * wm, __umul64hi(sR, wm));
          bins[pc * BS_NTHR] += t0.y + t1.y + t2.y + t3.y;
        } else if (c) {
          // every lane state connected: the lane mass is exactly 1
          const u64 wm = s_wmid[(gout << BS_IN) | (u32)r];
          u128_add(T, wm << 62, wm >> 2);
          bins[(pco + __popc(r)) * BS_NTHR] += BS_FULL_COUNTS;
        }
      }
    }
    if (thr_on) bs_flush_bins(bins, s_nbins, pc_pre + pc_thr);
    // item total: exact warp sum of T x thread mass (scale 2^124), times the
    // prefix mass, once per item
    const u128 S = warp_sum_u128(mul64x128_shr64(thw, T.lo, T.hi));
    const mx w = bs_prefix_mass(P, ptab, prefix);
    facc_add(accR, mx_prod(w, S), w.e);
  }
  if constexpr (phase == 1) bs_flush_deferred(W, pend, npend, lane);
  if (lane == 0) {
    atomicAdd(&W.stats[0], n_walk); atomicAdd(&W.stats[1], n_full); atomicAdd(&W.stats[2], n_dead);
    s_acc[warp] = accR;
  }
  __syncthreads();
  bs_write_out(W, s_acc, 1, 1, s_nbins);
}

#define KERNEL_R_ARGS const __grid_constant__ BsParams P, const u64* __restrict__ lane_tab, \
                  const u64* __restrict__ wmid_tab, const mx* __restrict__ ptab, const BsWork W
extern "C" __global__ void KERNEL_BOUNDS bs_kernel(KERNEL_R_ARGS) { bs_kernel_body<0>(P, lane_tab, wmid_tab, ptab, W); }
extern "C" __global__ void KERNEL_BOUNDS_P1 bs_kernel_p1(KERNEL_R_ARGS) { bs_kernel_body<1>(P, lane_tab, wmid_tab, ptab, W); }
extern "C" __global__ void KERNEL_BOUNDS bs_kernel_p2(KERNEL_R_ARGS) { bs_kernel_body<2>(P, lane_tab, wmid_tab, ptab, W); }
#endif

#if BS_GRAD
// ---------------------------------------------------------------------------
// Fused R + N_k + dR/dp.  Every gradient term is a difference of two exact
// integer sums over the two halves of state pairs (X, X + e_i) that carry
// identical weights, so it is exact and non-negative:
//   thread arcs: per-thread totals T of warp lanes t and t ^ 2^i;
//   lane arcs: the 32x32 bit matrix (threads x lanes) of a word is
//     transposed across the warp, so lane j holds the states of lane pattern
//     j; its total T2 (thread-pattern masses from byte tables) pairs lanes j
//     and j ^ 2^i in the same way;
//   walk arcs: A_b, the part of T collected while walk arc b works, against
//     T - A_b; both are summed over items and divided by p_b and 1 - p_b once,
//     at the end;
//   prefix arcs: item totals times the prefix mass without that arc, summed
//     apart for the arc working and failed.
// Per item every quantity is first summed exactly over the warp in 128-bit
// integers with fixed-point per-lane weights; then the lane that owns an arc
// (lanes k and k - 32 own internal arc k) scales it by the item's prefix
// mass (integer floating point) and adds it to that arc's two floating
// 128-bit accumulators in shared memory.  Walk masses are 128-bit (scale
// 2^127).
struct BsGradParams {
  u64 thw_ex[5][32];    // thread-pattern masses without thread arc i (2^63)
  u64 lw_ex[5][32];     // lane-pattern masses without lane arc i (2^63)
  dd inv_p[64], inv_q[64];
};

static_assert(BS_TOP <= 32, "lane k owns internal arc k");

// The prefix factor of internal arc k for this item.  Internal arcs, and
// prefix arcs with p in [2^-20, 1 - 2^-20], take the whole prefix mass: a
// prefix arc's two sums then carry its own factor p or 1 - p, which the
// host divides out once (as for walk arcs) -- the sums' errors are relative
// to their terms, so the division does not amplify them.  Prefix arcs with
// p outside that range (bits set in BS_PEX_MASK) take the item's prefix
// mass without their own factor, from the excluded-arc table.
__device__ __forceinline__ mx bs_arc_factor(const BsParams& P, const mx* __restrict__ ptab,
                                            const mx* __restrict__ ptab_ex, u64 prefix, int k, mx wpre) {
  if (k < BS_TOP || !((BS_PEX_MASK >> k) & 1ull)) return wpre;
  const int j = k - BS_TOP;
  int l = 0, sh = 0;
  while (sh + P.lev_bits[l] <= j) { sh += P.lev_bits[l]; ++l; }
  mx f = wpre;
  int s2 = 0;
  for (int q = 0; q < P.nlev; ++q) {
    const u64 bits = (prefix >> s2) & ((1ull << P.lev_bits[q]) - 1ull);
    const mx t = q == l ? ptab_ex[((size_t)j << P.ex_shift) + bits] : ptab[P.lev_off[q] + bits];
    f = q ? mx_mul(f, t) : t;
    s2 += P.lev_bits[q];
  }
  return f;
}

template <int PHASE>
__device__ __forceinline__ void bs_kernel_grad_body(
    const BsParams& P, const BsGradParams& Q, const u64* __restrict__ lane_tab,
    const u64* __restrict__ thr_tab, const u64* __restrict__ wmid128, const mx* __restrict__ ptab,
    const mx* __restrict__ ptab_ex, const BsWork& W) {
  extern __shared__ __align__(16) unsigned char smem[];
  ulonglong2* s_lt = (ulonglong2*)smem;                     // [4][256] {lane mass 2^62, packed counts}
  ulonglong2* s_wm = s_lt + 4 * 256;                        // [2^L] walk masses {lo, hi} (2^127)
  u64* s_tt = (u64*)(s_wm + (1 << BS_L));                   // [4][256] thread-pattern masses (2^62)
  u64* s_bins = s_tt + 4 * 256;                             // [L + 1][NTHR]
  u128* s_A = (u128*)(s_bins + (BS_L + 1) * BS_NTHR);       // [BS_OUT][NTHR]
  // the first of two launches walks nothing: it holds only the N_k counts,
  // so it is launched with (m + 1) * 8 bytes of shared memory
  u64* s_nbins = PHASE == 1 ? (u64*)smem : (u64*)(s_A + (BS_OUT > 0 ? BS_OUT : 1) * BS_NTHR);
  // per warp, in global scratch: R, then A_k and B_k of every arc k
  facc* g_acc = W.wacc + (size_t)blockIdx.x * (BS_NTHR / 32) * (1 + 2 * BS_M);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if constexpr (PHASE == 2) {
    if (bs_list_done(W)) return;
  }
  if constexpr (PHASE != 1) {
    for (int i = tid; i < 4 * 256; i += BS_NTHR) s_lt[i] = ((const ulonglong2*)lane_tab)[i];
    for (int i = tid; i < 4 * 256; i += BS_NTHR) s_tt[i] = thr_tab[i];
    for (int i = tid; i < (1 << BS_L); i += BS_NTHR) s_wm[i] = ((const ulonglong2*)wmid128)[i];
  }
  for (int i = tid; i < (BS_NTHR / 32) * (1 + 2 * BS_M); i += BS_NTHR) g_acc[i] = facc{u128{0ull, 0ull}, 0, 0};
  for (int i = tid; i <= BS_M; i += BS_NTHR) s_nbins[i] = 0ull;
  __syncthreads();
  facc* acc = g_acc + warp * (1 + 2 * BS_M);
  u64* bins = s_bins + tid;
  u128* A = s_A + tid;
  const BsTr tr = bs_tr_init(lane);
  const bool thr_on = lane < (1 << BS_TB);
  const int pc_thr = __popc(lane & ((1 << BS_TB) - 1));
  const u64 thw = thr_on ? P.thw[lane] : 0ull;
  const u64 t_start = bs_timer();
  u64 n_walk = 0, n_full = 0, n_dead = 0;
#if BS_ACC_REG
  // short items: this lane's accumulators -- R and the two sums of internal
  // arcs `lane` and `lane + 32` -- in registers, so an item costs no global
  // round trip.  Long items keep them all in the global slots: registers are
  // worth more to the walk.
  facc accR = facc{u128{0ull, 0ull}, 0, 0}, accA = accR, accB = accR;
#if BS_M > 32
  facc accA2 = accR, accB2 = accR;
#endif
#endif
  u32 a[BS_M];
  bs_init_arcs(a, lane);
  constexpr int phase = PHASE;
  // phase 1: this warp's chunk of items -- its first chunk is its own (no
  // ticket at the start of a short launch), the later ones come by ticket
  u64 chunk_next = ((u64)blockIdx.x * (BS_NTHR / 32) + warp) * 16, chunk_end = chunk_next + 16;
  u64 pend = 0;   // phase 1: this warp's deferred items, entry j in lane j
  int npend = 0;

  for (;;) {
    u64 task = 0;
    if constexpr (phase == 1) {
      if (chunk_next == chunk_end) {   // the next 16 items, by one atomic ticket
        u64 base = 0;
        if (lane == 0) base = (u64)gridDim.x * (BS_NTHR / 32) * 16 + atomicAdd(W.counter, 16ull);
        chunk_next = __shfl_sync(0xffffffffu, base, 0);
        chunk_end = chunk_next + 16;
      }
      task = chunk_next++;
    }
    if (lane == 0) {
      if constexpr (phase == 2) task = bs_list_task(W);
      else if constexpr (phase == 0) task = atomicAdd(W.counter, 1ull);
      if (P.budget_ns && bs_timer() - t_start > P.budget_ns) { atomicOr(W.status, 1u); task = ~0ull; }
    }
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= P.n_tasks) break;
    const u64 prefix = P.task_lo + task;
#pragma unroll
    for (int j = 0; j < BS_D; ++j) a[BS_TOP + j] = 0u - (u32)((prefix >> j) & 1ull);
    const int pc_pre = __popcll((long long)prefix);
    int pr = 0;
    if ((P.prune && phase == 0) || phase == 1) {   // two-launch runs always prune
      pr = bs_prune(a);
      if (pr == 1) { ++n_dead; continue; }
    }
    if constexpr (phase == 1) {
      if (pr == 0) {   // left to walk: deferred to the second launch
        if (lane == npend) pend = task;
        if (++npend == 32) { bs_flush_deferred(W, pend, npend, lane); npend = 0; }
        continue;
      }
    }
#if BS_ACC_REG
    // the prefix factors of an item that is not cut off, before its walk so
    // that their table loads overlap it (a cut-off item needs none: with
    // prune-aware prefix arcs most items are cut off or fully connected)
    const mx wpre = bs_prefix_mass(P, ptab, prefix);
    const mx f0 = bs_arc_factor(P, ptab, ptab_ex, prefix, lane, wpre);
    const mx f1 = lane + 32 < BS_M ? bs_arc_factor(P, ptab, ptab_ex, prefix, lane + 32, wpre) : wpre;
#endif
    u128 S;      // sum over the warp of T x thread mass, scale 2^124
    // warp sums of the internal arc this lane owns (internal arcs are below
    // 32): the exact pair difference, or for a walk arc A and T - A
    u128 myX = u128{0ull, 0ull}, myY = u128{0ull, 0ull};
    if (pr == 2 || phase == 1) {   // (the first of two launches walks nothing)
      ++n_full;
      for (int j = lane; j <= BS_TOP; j += 32) atomicAdd(&s_nbins[pc_pre + j], P.binom[j]);
      S = u128{0ull, 1ull << 60};   // the whole item: mass 1 at scale 2^124
    } else {
      ++n_walk;
      u32 e[BS_NCORE > 0 ? BS_NCORE : 1];
      bs_inv(a, e);
#pragma unroll
      for (int r = 0; r <= BS_L; ++r) bins[r * BS_NTHR] = 0ull;
#pragma unroll
      for (int b = 0; b < BS_OUT; ++b) A[b * BS_NTHR] = u128{0ull, 0ull};
      u128 T = u128{0ull, 0ull}, T2 = u128{0ull, 0ull};
      u128 Ain[BS_IN > 0 ? BS_IN : 1];
#pragma unroll
      for (int b = 0; b < BS_IN; ++b) Ain[b] = u128{0ull, 0ull};
      u32 gout = 0;
      int pco = 0;
#pragma unroll 1
      for (u32 s = 0; s < (1u << BS_OUT); ++s) {
        if (s) {
          const int b = __ffs(s) - 1;
          gout ^= 1u << b;
          const bool on = (gout >> b) & 1u;
          pco += on ? 1 : -1;
          // outer walk arc b: A collects the growth of T while the arc works
          u128 ab = A[b * BS_NTHR];
          if (on) ab = u128_sub(ab, T); else u128_add(ab, T.lo, T.hi);
          A[b * BS_NTHR] = ab;
        }
        u32 w[BS_L > 0 ? BS_L : 1];
#pragma unroll
        for (int b = 0; b < BS_OUT; ++b) w[BS_IN + b] = 0u - ((gout >> b) & 1u);
        // the inner words' packed counts by inner popcount, in registers
        u64 nb[BS_IN + 1];
#pragma unroll
        for (int j = 0; j <= BS_IN; ++j) nb[j] = 0ull;
#pragma unroll
        for (int r = 0; r < (1 << BS_IN); ++r) {
#pragma unroll
          for (int b = 0; b < BS_IN; ++b) w[b] = ((r >> b) & 1) ? ~0u : 0u;
          const u32 g = (gout << BS_IN) | (u32)r;
          const u32 c = bs_var(e, w) & BS_LANE_MASK;
          const ulonglong2 wv = s_wm[g];
          if (__any_sync(0xffffffffu, c != 0u && c != BS_LANE_MASK)) {
            // some word of the warp is partly connected: no branch on the
            // word's class (a cut word reads the zero entries, a connected
            // one the mass of all its lanes), and the lane transpose
            const ulonglong2 t0 = s_lt[0 * 256 + (c & 0xffu)], t1 = s_lt[1 * 256 + ((c >> 8) & 0xffu)];
            const ulonglong2 t2 = s_lt[2 * 256 + ((c >> 16) & 0xffu)], t3 = s_lt[3 * 256 + (c >> 24)];
            const u128 x = mul64x128_shr64(t0.x + t1.x + t2.x + t3.x, wv.x, wv.y);
            u128_add(T, x.lo, x.hi);
#pragma unroll
            for (int b = 0; b < BS_IN; ++b)
              if ((r >> b) & 1) u128_add(Ain[b], x.lo, x.hi);
            nb[__popc(r)] += t0.y + t1.y + t2.y + t3.y;
            const u32 ct = bs_transpose32(c, tr);
            const u64 s2 = s_tt[ct & 0xffu] + s_tt[256 + ((ct >> 8) & 0xffu)] +
                           s_tt[512 + ((ct >> 16) & 0xffu)] + s_tt[768 + (ct >> 24)];
            const u128 x2 = mul64x128_shr64(s2, wv.x, wv.y);
            u128_add(T2, x2.lo, x2.hi);
          } else if (c) {
            // every word of the warp is cut or fully connected (no lane-arc
            // pair differs): a connected word's lane mass is exactly 1, the
            // walk mass at scale 2^125
            const u128 x = u128{(wv.x >> 2) | (wv.y << 62), wv.y >> 2};
            u128_add(T, x.lo, x.hi);
#pragma unroll
            for (int b = 0; b < BS_IN; ++b)
              if ((r >> b) & 1) u128_add(Ain[b], x.lo, x.hi);
            nb[__popc(r)] += BS_FULL_COUNTS;
          }
        }
#pragma unroll
        for (int j = 0; j <= BS_IN; ++j) bins[(pco + j) * BS_NTHR] += nb[j];
      }
#pragma unroll
      for (int b = 0; b < BS_OUT; ++b)
        if ((gout >> b) & 1u) { u128 ab = A[b * BS_NTHR]; u128_add(ab, T.lo, T.hi); A[b * BS_NTHR] = ab; }
      if (thr_on) bs_flush_bins(bins, s_nbins, pc_pre + pc_thr);
      // ---- exact warp sums; slot k of `red` holds internal arc k's value
      S = warp_sum_u128(mul64x128_shr64(thw, T.lo, T.hi));
#pragma unroll
      for (int i = 0; i < BS_ELL; ++i) {
        const u128 o = shfl_xor_u128(T2, 1 << i);
        const u128 d2 = u128_sub(T2, o);
        const u128 v = ((lane >> i) & 1) ? mul64x128_shr64(Q.lw_ex[i][lane], d2.lo, d2.hi) : u128{0ull, 0ull};
        const u128 sv = warp_sum_u128(v);
        if (lane == i) myX = sv;
      }
#pragma unroll
      for (int i = 0; i < BS_TB; ++i) {
        const u128 o = shfl_xor_u128(T, 1 << i);
        const u128 d1 = u128_sub(T, o);
        const u128 v = (((lane >> i) & 1) && thr_on) ? mul64x128_shr64(Q.thw_ex[i][lane], d1.lo, d1.hi)
                                                     : u128{0ull, 0ull};
        const u128 sv = warp_sum_u128(v);
        if (lane == BS_ELL + i) myX = sv;
      }
#pragma unroll
      for (int b = 0; b < BS_L; ++b) {
        const u128 Ab = b < BS_IN ? Ain[b < BS_IN ? b : 0] : A[(b >= BS_IN ? b - BS_IN : 0) * BS_NTHR];
        const u128 sa = warp_sum_u128(mul64x128_shr64(thw, Ab.lo, Ab.hi));
        // the failed half: S - sa, the lanes' truncated products of T less
        // those of A (each lane's difference is that of T - A, or one unit
        // more, at scale 2^124; never negative)
        const u128 sz = u128_sub(S, sa);
        if (lane == BS_WALK0 + b) { myX = sa; myY = sz; }
      }
    }
    // ---- per-arc scaling on the owning lanes (internal arcs lane, lane + 32)
#if !BS_ACC_REG
    const mx wpre = bs_prefix_mass(P, ptab, prefix);
    const mx f0 = bs_arc_factor(P, ptab, ptab_ex, prefix, lane, wpre);
    const mx f1 = lane + 32 < BS_M ? bs_arc_factor(P, ptab, ptab_ex, prefix, lane + 32, wpre) : wpre;
    facc accR, accA, accB;
    if (lane == 0) accR = acc[0];
    if (lane < BS_M) {
      accA = acc[1 + 2 * lane];
      accB = acc[2 + 2 * lane];
    }
#endif
    if (lane == 0) facc_add(accR, mx_prod(wpre, S), wpre.e);
    {
      // arc `lane`: a prefix arc goes into A when it works in this item and
      // into B when it fails (the item's mass without its factor); an
      // internal arc of a fully connected item has no pair that differs
      u128 X = u128{0ull, 0ull}, Y = u128{0ull, 0ull};
      if (lane >= BS_TOP) {
        if (lane < BS_M) {
          if ((prefix >> (lane - BS_TOP)) & 1ull) X = S; else Y = S;
        }
      } else if (pr != 2) {
        X = myX;
        Y = myY;
      }
      facc_add(accA, mx_prod(f0, X), f0.e);
      facc_add(accB, mx_prod(f0, Y), f0.e);
    }
#if !BS_ACC_REG
    if (lane == 0) acc[0] = accR;
    if (lane < BS_M) {
      acc[1 + 2 * lane] = accA;
      acc[2 + 2 * lane] = accB;
    }
#endif
    if (lane + 32 < BS_M) {
      // arc lane + 32 is a prefix arc (lanes own arcs below 32 and the top
      // prefix arcs): the item's total, by whether the arc works here
      const int j = lane + 32 - BS_TOP;
#if BS_ACC_REG && BS_M > 32
      if ((prefix >> j) & 1ull) facc_add(accA2, mx_prod(f1, S), f1.e);
      else facc_add(accB2, mx_prod(f1, S), f1.e);
#else
      facc* ak = acc + 1 + 2 * (lane + 32);
      facc va = ak[0], vb = ak[1];
      if ((prefix >> j) & 1ull) facc_add(va, mx_prod(f1, S), f1.e);
      else facc_add(vb, mx_prod(f1, S), f1.e);
      ak[0] = va;
      ak[1] = vb;
#endif
    }
    __syncwarp();
  }
  if constexpr (phase == 1) bs_flush_deferred(W, pend, npend, lane);
  if (lane == 0) {
    atomicAdd(&W.stats[0], n_walk); atomicAdd(&W.stats[1], n_full); atomicAdd(&W.stats[2], n_dead);
  }
#if BS_ACC_REG
  if (lane == 0) acc[0] = accR;
  if (lane < BS_M) {
    acc[1 + 2 * lane] = accA;
    acc[2 + 2 * lane] = accB;
  }
#if BS_M > 32
  if (lane + 32 < BS_M) {
    acc[1 + 2 * (lane + 32)] = accA2;
    acc[2 + 2 * (lane + 32)] = accB2;
  }
#endif
#endif
  // ---- per block: R, then A_k and B_k of every arc; the host forms the
  // gradient (A - B for prefix arcs, A / p - B / (1 - p) for walk arcs, A
  // for lane and thread arcs)
  __syncthreads();
  bs_write_out(W, g_acc, 1 + 2 * BS_M, 1 + 2 * BS_M, s_nbins);
}

#define KERNEL_G_ARGS const __grid_constant__ BsParams P, const __grid_constant__ BsGradParams Q, \
                  const u64* __restrict__ lane_tab, const u64* __restrict__ thr_tab, \
                  const u64* __restrict__ wmid128, const mx* __restrict__ ptab, \
                  const mx* __restrict__ ptab_ex, const BsWork W
#define KERNEL_G_PASS P, Q, lane_tab, thr_tab, wmid128, ptab, ptab_ex, W
extern "C" __global__ void KERNEL_BOUNDS bs_kernel_grad(KERNEL_G_ARGS) { bs_kernel_grad_body<0>(KERNEL_G_PASS); }
extern "C" __global__ void KERNEL_BOUNDS_P1 bs_kernel_grad_p1(KERNEL_G_ARGS) { bs_kernel_grad_body<1>(KERNEL_G_PASS); }
extern "C" __global__ void KERNEL_BOUNDS bs_kernel_grad_p2(KERNEL_G_ARGS) { bs_kernel_grad_body<2>(KERNEL_G_PASS); }
#endif
)PBAT";


// Batched: every network's connectivity program is a struct of static
// functions (inv, var) with its sizes as constants; one persistent kernel
// takes (network, prefix) items from one ticket -- networks with the most
// items first -- and switches to that network's connectivity function
// (bsb_conn), which only stages the item's 2^L connectivity words in shared
// memory.  The accumulate (bsb_finish) is written once in the kernel body,
// so the module's compile time barely grows with the number of networks: it
// weights each word by every p-vector, 16 at a time in registers (byte
// tables interleaved by p-vector, read through L1), and adds each item's
// mass per p-vector exactly into a 256-bit fixed-point number (eight 32-bit
// chunks in 64-bit limbs) with integer atomics.  N_k counts collect per warp
// in shared memory.
static const char* kBsBatchTemplate = R"PBAT(
#define BSB_LIMBS 8
#define BSB_KC 16
struct BGraph {
  u64 task_begin, n_tasks;
  int gidx, m, nlev, prune;
  int lev_bits[8], lev_off[8];
  int lt_off, nt_off, wm_off, pt_off, pt_size, thw_off, nk_off, tb;
  int L, top;
  u32 lane_mask;
  int pad0;
  // gradient module only: offsets of the 128-bit walk masses, the thread
  // byte tables, the excluded-arc masses of lane, thread and prefix arcs,
  // and of this network's results; lane arcs, prefix arcs, thread mask
  int wm2_off, tt_off, lwex_off, thwex_off, ptex_off, out_off, ell, d;
  u32 thr_mask;
  int pad1;
  u64 full_counts;
  u64 pex_mask;   // gradient module: prefix arcs using the excluded-arc tables
  u64 binom[64];
};

// add P * 2^(-123 - e) (P < 2^124, e >= 0) to the 256-bit limbs (scale 2^250)
__device__ __forceinline__ void bsb_limb_add(u64* limbs, u128 P, int e) { bs_limb_add(limbs, P, 127 - e); }

// prefix mass of one p-vector: product over the levels of its table t
__device__ __forceinline__ mx bsb_prefix_mass(const mx* __restrict__ t, int nlev, const int (&lev_bits)[8],
                                              const int (&lev_off)[8], u64 prefix) {
  mx w = mx{1ull << 63, 0, 0};
  int sh = 0;
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    if (l >= nlev) break;
    const u64 v = (prefix >> sh) & ((1ull << lev_bits[l]) - 1ull);
    const ulonglong2 q = __ldg((const ulonglong2*)(t + lev_off[l] + v));
    const mx f = mx{q.x, (int)(u32)q.y, 0};
    w = l ? mx_mul(w, f) : f;
    sh += lev_bits[l];
  }
  return w;
}

template <class G>
__device__ __forceinline__ u32 bsb_uniform(const u32* a) {
  u32 e[G::NCORE > 0 ? G::NCORE : 1];
  G::inv(a, e);
  u32 w[G::L > 0 ? G::L : 1];
#pragma unroll
  for (int b = 0; b < G::L; ++b) w[b] = a[G::WALK0 + b];
  return G::var(e, w);
}

// The per-network part of one item: its state words, the monotone prune,
// and the connectivity word of every walk state into cw (stride BSB_NTHR).
// Returns 0 when every state of the item is cut, 1 when every state is
// connected, 2 when cw holds the item's words.
template <class G>
__device__ __forceinline__ int bsb_conn(u64 prefix, int lane, int prune, u32* cw) {
  u32 a[G::M];
#pragma unroll
  for (int i = 0; i < G::ELL; ++i)
    a[i] = i == 0 ? 0xAAAAAAAAu : i == 1 ? 0xCCCCCCCCu : i == 2 ? 0xF0F0F0F0u : i == 3 ? 0xFF00FF00u : 0xFFFF0000u;
#pragma unroll
  for (int i = 0; i < G::TB; ++i) a[G::ELL + i] = 0u - (u32)((lane >> i) & 1);
#pragma unroll
  for (int b = 0; b < G::L; ++b) a[G::WALK0 + b] = 0u;
#pragma unroll
  for (int j = 0; j < G::D; ++j) a[G::TOP + j] = 0u - (u32)((prefix >> j) & 1ull);
  if (prune) {
    // one evaluation for both extremes: bit 0 has every arc below the prefix
    // up, the other bits have them all down (the prefix arcs are the same in
    // every bit)
    u32 u[G::M];
#pragma unroll
    for (int k = 0; k < G::M; ++k) u[k] = k < G::TOP ? 1u : a[k];
    const u32 ext = bsb_uniform<G>(u);
    if (!(ext & 1u)) return 0;
    if (ext & 2u) return 1;
  }
  u32 e[G::NCORE > 0 ? G::NCORE : 1];
  G::inv(a, e);
#pragma unroll 1
  for (u32 g = 0; g < (1u << G::L); ++g) {
    u32 w[G::L > 0 ? G::L : 1];
#pragma unroll
    for (int b = 0; b < G::L; ++b) w[b] = 0u - ((g >> b) & 1u);
    cw[g * BSB_NTHR] = G::var(e, w) & G::LANE_MASK;
  }
  return 2;
}
// Everything of an item past connectivity, shared by every network (inlined
// once, in the kernel body): counts N_k, then sums the exact fixed-point
// mass of every p-vector, BSB_KC of them at a time (Eq. 1 restricted to the
// item) -- per thread in registers, then over the warp by a reduce-scatter
// that leaves p-vector kk's item total on lanes 2 idx(kk) and 2 idx(kk) + 1,
// so that the prefix scaling and the limb additions run on 16 lanes at once.
// The network's constants are read once into registers.
// add the warp's counts of network B (k = 0..m) to the global N_k, then clear
__device__ __forceinline__ void bsb_flush_counts(const BGraph* __restrict__ B, u64* nkw, u64* nk, int lane) {
  const int m = B->m, off = B->nk_off;
  for (int i = lane; i <= m; i += 32) {
    const u64 v = nkw[i];
    if (v) atomicAdd(&nk[off + i], v);
    nkw[i] = 0ull;
  }
  __syncwarp();
}

// N_k counts go to the warp's own array nkw (indexed by k within the
// network), which the kernel flushes to global memory when the warp moves
// to another network and at the end.
__device__ __forceinline__ void bsb_finish(const BGraph* __restrict__ Bp, int st, u64 prefix, int lane, int K,
                                           int Kp, const u64* __restrict__ lt, const u64* __restrict__ nt,
                                           const u64* __restrict__ wm, const mx* __restrict__ pt,
                                           const u64* __restrict__ thw, u64* limbs, u64* nkw, u64* bins,
                                           const u32* cw) {
  constexpr int nsh[6] = BS_NK_SHIFTS, nwd[6] = BS_NK_WIDTHS;
  const int gidx = Bp->gidx, L = Bp->L, tb = Bp->tb, nlev = Bp->nlev, top = Bp->top;
  const int lt_off = Bp->lt_off, nt_off = Bp->nt_off, wm_off = Bp->wm_off, pt_off = Bp->pt_off;
  const int pt_size = Bp->pt_size, thw_off = Bp->thw_off;
  const u32 lane_mask = Bp->lane_mask;
  const u64 full_counts = Bp->full_counts;
  int lev_bits[8], lev_off[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    lev_bits[l] = Bp->lev_bits[l];
    lev_off[l] = Bp->lev_off[l];
  }
  const int pc_pre = __popcll((long long)prefix);
  u64* glimbs = limbs + (size_t)gidx * K * BSB_LIMBS;
  const mx* gpt = pt + pt_off;
  if (st == 1) {
    // every state connected: binomial counts, and per p-vector the prefix mass
    for (int j = lane; j <= top; j += 32) nkw[pc_pre + j] += __ldg(&Bp->binom[j]);
    for (int k = lane; k < K; k += 32) {
      const mx w = bsb_prefix_mass(gpt + (size_t)k * pt_size, nlev, lev_bits, lev_off, prefix);
      bsb_limb_add(glimbs + (size_t)k * BSB_LIMBS, mx_prod(w, u128{0ull, 1ull << 60}), w.e);
    }
    return;
  }
  const int nw = 1 << L;
  for (int r = 0; r <= L; ++r) bins[r * BSB_NTHR] = 0ull;
  const u64* ntg = nt + nt_off;
  for (int g = 0; g < nw; ++g) {
    const u32 c = cw[g * BSB_NTHR];
    if (!c) continue;
    bins[__popc(g) * BSB_NTHR] += c == lane_mask ? full_counts
        : __ldg(ntg + (c & 0xffu)) + __ldg(ntg + 256 + ((c >> 8) & 0xffu)) +
          __ldg(ntg + 512 + ((c >> 16) & 0xffu)) + __ldg(ntg + 768 + (c >> 24));
  }
  const bool thr_on = lane < (1 << tb);
  {
    // this thread's counts by r + cl (walk popcount + lane class), then
    // shared atomics at k = prefix + thread + r + cl
    u64 c11[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) c11[i] = 0ull;
#pragma unroll
    for (int r = 0; r <= 5; ++r) {
      if (r > L) break;
      const u64 n = bins[r * BSB_NTHR];
#pragma unroll
      for (int cl = 0; cl < 6; ++cl) c11[r + cl] += (n >> nsh[cl]) & ((1ull << nwd[cl]) - 1ull);
    }
    if (thr_on) {
      const int base = pc_pre + __popc(lane);
#pragma unroll
      for (int i = 0; i < 11; ++i)
        if (c11[i]) atomicAdd(&nkw[base + i], c11[i]);
    }
  }
  const u64* ltg = lt + lt_off;
  const u64* wmg = wm + wm_off;
  const u64* thg = thw + thw_off + (size_t)lane * Kp;
  // p-vector whose total this lane holds after the reduce-scatter
  const int idx = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
  for (int k0 = 0; k0 < K; k0 += BSB_KC) {
    const int kc = min(BSB_KC, K - k0);
    u128 T[BSB_KC];
#pragma unroll
    for (int kk = 0; kk < BSB_KC; ++kk) T[kk] = u128{0ull, 0ull};
    for (int g = 0; g < nw; ++g) {
      const u32 c = cw[g * BSB_NTHR];
      if (!c) continue;
      // table rows hold whole chunks of 16 p-vectors (zero past K), so all
      // loads of a word are unconditional and in flight together
      const ulonglong2* wv = (const ulonglong2*)(wmg + (size_t)g * Kp + k0);
      if (c == lane_mask) {
        // every lane state connected: lane mass exactly 1, the walk mass at
        // scale 2^125
#pragma unroll
        for (int h = 0; h < BSB_KC / 2; ++h) {
          const ulonglong2 ww = __ldg(wv + h);
          u128_add(T[2 * h], ww.x << 62, ww.x >> 2);
          u128_add(T[2 * h + 1], ww.y << 62, ww.y >> 2);
        }
        continue;
      }
      const ulonglong2* l0 = (const ulonglong2*)(ltg + (size_t)(0 * 256 + (c & 0xffu)) * Kp + k0);
      const ulonglong2* l1 = (const ulonglong2*)(ltg + (size_t)(1 * 256 + ((c >> 8) & 0xffu)) * Kp + k0);
      const ulonglong2* l2 = (const ulonglong2*)(ltg + (size_t)(2 * 256 + ((c >> 16) & 0xffu)) * Kp + k0);
      const ulonglong2* l3 = (const ulonglong2*)(ltg + (size_t)(3 * 256 + (c >> 24)) * Kp + k0);
#pragma unroll
      for (int h = 0; h < BSB_KC / 2; ++h) {
        const ulonglong2 a0 = __ldg(l0 + h), a1 = __ldg(l1 + h), a2 = __ldg(l2 + h), a3 = __ldg(l3 + h);
        const ulonglong2 ww = __ldg(wv + h);
        const u64 sx = a0.x + a1.x + a2.x + a3.x, sy = a0.y + a1.y + a2.y + a3.y;
        u128_add(T[2 * h], sx * ww.x, __umul64hi(sx, ww.x));
        u128_add(T[2 * h + 1], sy * ww.y, __umul64hi(sy, ww.y));
      }
    }
    // thread-pattern masses (scale 2^124 after this), then the reduce-scatter
#pragma unroll
    for (int kk = 0; kk < BSB_KC; ++kk) {
      const u64 tw = (thr_on && kk < kc) ? __ldg(thg + k0 + kk) : 0ull;
      T[kk] = mul64x128_shr64(tw, T[kk].lo, T[kk].hi);
    }
#pragma unroll
    for (int st2 = 0; st2 < 4; ++st2) {
      const int o = 16 >> st2, n = 8 >> st2;
      const bool up = lane & o;
#pragma unroll
      for (int i = 0; i < n; ++i) {
        const u128 send = up ? T[i] : T[i + n];
        const u128 keep = up ? T[i + n] : T[i];
        const u128 got = shfl_xor_u128(send, o);
        T[i] = keep;
        u128_add(T[i], got.lo, got.hi);
      }
    }
    {
      const u128 got = shfl_xor_u128(T[0], 1);
      u128_add(T[0], got.lo, got.hi);
    }
    if (!(lane & 1) && idx < kc) {
      const mx w = bsb_prefix_mass(gpt + (size_t)(k0 + idx) * pt_size, nlev, lev_bits, lev_off, prefix);
      bsb_limb_add(glimbs + (size_t)(k0 + idx) * BSB_LIMBS, mx_prod(w, T[0]), w.e);
    }
  }
}
// ---------------------------------------------------------------------------
// Batched fused R + N_k + dR/dp (the gradient module): the item's
// connectivity words (cw, one per walk state) and their 32x32 lane
// transposes (ctw) are formed once; then for each p-vector in turn the
// per-arc sums of the single-network fused kernel are built from them --
// exact integer pair differences for lane and thread arcs, the parts A and
// T - A of the walk arcs (128-bit walk masses), item totals times the
// prefix mass without the arc for prefix arcs -- and added to that
// (network, p-vector)'s 256-bit results: R, then A_k and B_k of every
// internal arc k.  Prefix arcs take the item's whole prefix mass (the host
// divides their sums by p and 1 - p) unless some p-vector puts their p
// outside [2^-20, 1 - 2^-20] (bit set in pex_mask).
// ---------------------------------------------------------------------------
__device__ __forceinline__ mx bsb_ex_factor(const mx* __restrict__ tk, const mx* __restrict__ exk,
                                            int nlev, const int (&lev_bits)[8], const int (&lev_off)[8],
                                            u64 prefix, int j) {
  // prefix mass without prefix arc j: its level's entry from the excluded
  // table (rows of 128), the other levels from the plain table
  mx f = mx{1ull << 63, 0, 0};
  int sh = 0;
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    if (l >= nlev) break;
    const u64 v = (prefix >> sh) & ((1ull << lev_bits[l]) - 1ull);
    const bool mine = j >= sh && j < sh + lev_bits[l];
    const ulonglong2 q = __ldg((const ulonglong2*)(mine ? exk + ((size_t)j << 7) + v : tk + lev_off[l] + v));
    const mx t = mx{q.x, (int)(u32)q.y, 0};
    f = l ? mx_mul(f, t) : t;
    sh += lev_bits[l];
  }
  return f;
}

__device__ __forceinline__ void bsb_finish_grad(
    const BGraph* __restrict__ Bp, int st, u64 prefix, int lane, int K, int Kp,
    const u64* __restrict__ lt, const u64* __restrict__ nt, const u64* __restrict__ wm2,
    const mx* __restrict__ pt, const u64* __restrict__ thw, const u64* __restrict__ tt,
    const u64* __restrict__ lwex, const u64* __restrict__ thwex, const mx* __restrict__ ptex,
    u64* limbs, u64* nkw, u64* bins, const u32* cw, u32* ctw, const BsTr& tr) {
  constexpr int nsh[6] = BS_NK_SHIFTS, nwd[6] = BS_NK_WIDTHS;
  const int L = Bp->L, tb = Bp->tb, ell = Bp->ell, top = Bp->top, m = Bp->m, nlev = Bp->nlev;
  const int pt_size = Bp->pt_size, d = Bp->d;
  const u32 lane_mask = Bp->lane_mask, thr_mask = Bp->thr_mask;
  int lev_bits[8], lev_off[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    lev_bits[l] = Bp->lev_bits[l];
    lev_off[l] = Bp->lev_off[l];
  }
  const int pc_pre = __popcll((long long)prefix);
  const bool thr_on = lane < (1 << tb);
  const int nw = 1 << L;
  // ---- N_k, as in the R module
  if (st == 1) {
    for (int j = lane; j <= top; j += 32) nkw[pc_pre + j] += __ldg(&Bp->binom[j]);
  } else {
    for (int r = 0; r <= L; ++r) bins[r * BSB_NTHR] = 0ull;
    const u64* ntg = nt + Bp->nt_off;
    for (int g = 0; g < nw; ++g) {
      const u32 c = cw[g * BSB_NTHR];
      if (!c) continue;
      bins[__popc(g) * BSB_NTHR] += c == lane_mask ? Bp->full_counts
          : __ldg(ntg + (c & 0xffu)) + __ldg(ntg + 256 + ((c >> 8) & 0xffu)) +
            __ldg(ntg + 512 + ((c >> 16) & 0xffu)) + __ldg(ntg + 768 + (c >> 24));
    }
    u64 c11[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) c11[i] = 0ull;
#pragma unroll
    for (int r = 0; r <= 5; ++r) {
      if (r > L) break;
      const u64 n = bins[r * BSB_NTHR];
#pragma unroll
      for (int cl = 0; cl < 6; ++cl) c11[r + cl] += (n >> nsh[cl]) & ((1ull << nwd[cl]) - 1ull);
    }
    if (thr_on) {
      const int base = pc_pre + __popc(lane);
#pragma unroll
      for (int i = 0; i < 11; ++i)
        if (c11[i]) atomicAdd(&nkw[base + i], c11[i]);
    }
    // ---- the lane transposes, once per word: lane j then holds the
    // threads' bits of lane pattern j (lanes past the thread patterns hold
    // no thread's states); zero when no lane's word is partly connected
    for (int g = 0; g < nw; ++g) {
      const u32 c = thr_on ? cw[g * BSB_NTHR] : 0u;
      const bool mixed = __any_sync(0xffffffffu, c != 0u && c != lane_mask);
      const u32 ct = mixed ? bs_transpose32(c, tr) : 0u;
      ctw[g * BSB_NTHR] = lane < (1 << ell) ? ct : 0u;
    }
  }
  const int stride = 1 + 2 * m;
  u64* gl = limbs + Bp->out_off;
  const u64* ltg = lt + Bp->lt_off;
  const u64* ttg = tt + Bp->tt_off;
  const ulonglong2* wmg = (const ulonglong2*)(wm2 + Bp->wm2_off);
  for (int k = 0; k < K; ++k) {
    u128 S = u128{0ull, 1ull << 60};   // a fully connected item: mass 1 at scale 2^124
    u128 myX = u128{0ull, 0ull}, myY = u128{0ull, 0ull};
    if (st == 2) {
      u128 T = u128{0ull, 0ull}, T2 = u128{0ull, 0ull};
      u128 Aw[5];
#pragma unroll
      for (int b = 0; b < 5; ++b) Aw[b] = u128{0ull, 0ull};
      for (int g = 0; g < nw; ++g) {
        const u32 c = cw[g * BSB_NTHR], ct = ctw[g * BSB_NTHR];
        if (!(c | ct)) continue;
        const ulonglong2 wv = __ldg(wmg + (size_t)g * Kp + k);
        const u128 full = u128{(wv.x >> 2) | (wv.y << 62), wv.y >> 2};   // scale 2^125
        if (c) {
          u128 x = full;
          if (c != lane_mask) {
            const u64 sR = __ldg(ltg + (size_t)(c & 0xffu) * Kp + k) +
                           __ldg(ltg + (size_t)(256 + ((c >> 8) & 0xffu)) * Kp + k) +
                           __ldg(ltg + (size_t)(512 + ((c >> 16) & 0xffu)) * Kp + k) +
                           __ldg(ltg + (size_t)(768 + (c >> 24)) * Kp + k);
            x = mul64x128_shr64(sR, wv.x, wv.y);
          }
          u128_add(T, x.lo, x.hi);
#pragma unroll
          for (int b = 0; b < 5; ++b)
            if (b < L && ((g >> b) & 1)) u128_add(Aw[b], x.lo, x.hi);
        }
        if (ct) {
          u128 y = full;
          if (ct != thr_mask) {
            const u64 s2 = __ldg(ttg + (size_t)(ct & 0xffu) * Kp + k) +
                           __ldg(ttg + (size_t)(256 + ((ct >> 8) & 0xffu)) * Kp + k) +
                           __ldg(ttg + (size_t)(512 + ((ct >> 16) & 0xffu)) * Kp + k) +
                           __ldg(ttg + (size_t)(768 + (ct >> 24)) * Kp + k);
            y = mul64x128_shr64(s2, wv.x, wv.y);
          }
          u128_add(T2, y.lo, y.hi);
        }
      }
      // exact warp sums (scale 2^124); lane k ends with internal arc k's
      const u64 thwk = thr_on ? __ldg(thw + Bp->thw_off + (size_t)lane * Kp + k) : 0ull;
      S = warp_sum_u128(mul64x128_shr64(thwk, T.lo, T.hi));
      for (int i = 0; i < ell; ++i) {
        const u128 o = shfl_xor_u128(T2, 1 << i);
        const u128 d2 = u128_sub(T2, o);
        const u64 w = ((lane >> i) & 1) && lane < (1 << ell)
                          ? __ldg(lwex + Bp->lwex_off + ((size_t)(i * 32 + lane)) * Kp + k) : 0ull;
        const u128 sv = warp_sum_u128(mul64x128_shr64(w, d2.lo, d2.hi));
        if (lane == i) myX = sv;
      }
      for (int i = 0; i < tb; ++i) {
        const u128 o = shfl_xor_u128(T, 1 << i);
        const u128 d1 = u128_sub(T, o);
        const u64 w = ((lane >> i) & 1) && thr_on
                          ? __ldg(thwex + Bp->thwex_off + ((size_t)(i * 32 + lane)) * Kp + k) : 0ull;
        const u128 sv = warp_sum_u128(mul64x128_shr64(w, d1.lo, d1.hi));
        if (lane == ell + i) myX = sv;
      }
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        if (b >= L) break;
        const u128 sa = warp_sum_u128(mul64x128_shr64(thwk, Aw[b].lo, Aw[b].hi));
        const u128 sz = u128_sub(S, sa);   // the failed half, as in the fused kernel
        if (lane == ell + tb + b) { myX = sa; myY = sz; }
      }
    }
    // ---- prefix factors of p-vector k and the additions to its results
    const mx* tk = pt + Bp->pt_off + (size_t)k * pt_size;
    const mx* exk = ptex + Bp->ptex_off + ((size_t)k * d << 7);
    const mx wpre = bsb_prefix_mass(tk, nlev, lev_bits, lev_off, prefix);
    u64* out = gl + (size_t)k * stride * BSB_LIMBS;
    if (lane == 0) bsb_limb_add(out, mx_prod(wpre, S), wpre.e);
    if (lane < m) {
      u128 X = u128{0ull, 0ull}, Y = u128{0ull, 0ull};
      mx f = wpre;
      if (lane >= top) {
        // a prefix arc: the item's total, into A when the arc works in this
        // item and into B when it fails -- with the whole prefix mass (the
        // host divides by p and 1 - p), or for an arc whose p is outside
        // [2^-20, 1 - 2^-20] under some p-vector, without its own factor
        if ((Bp->pex_mask >> lane) & 1ull)
          f = bsb_ex_factor(tk, exk, nlev, lev_bits, lev_off, prefix, lane - top);
        if ((prefix >> (lane - top)) & 1ull) X = S; else Y = S;
      } else if (st == 2) {
        X = myX;
        Y = myY;
      }
      bsb_limb_add(out + (1 + 2 * lane) * BSB_LIMBS, mx_prod(f, X), f.e);
      bsb_limb_add(out + (2 + 2 * lane) * BSB_LIMBS, mx_prod(f, Y), f.e);
    }
    if (lane + 32 < m) {
      const int j = lane + 32 - top;
      const mx f = ((Bp->pex_mask >> (lane + 32)) & 1ull)
                       ? bsb_ex_factor(tk, exk, nlev, lev_bits, lev_off, prefix, j) : wpre;
      const bool on = (prefix >> j) & 1ull;
      bsb_limb_add(out + ((on ? 1 : 2) + 2 * (lane + 32)) * BSB_LIMBS, mx_prod(f, S), f.e);
    }
  }
}
//@@BATCH_KERNEL@@
)PBAT";
}  // namespace pbat
