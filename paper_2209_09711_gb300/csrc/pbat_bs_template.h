// pbat_bs_template.h -- CUDA source of the bit-sliced enumeration kernel.
//
// The engine prepends a block of #defines and the graph-specific
// connectivity functions (bs_inv / bs_var, written by the planner in
// pbat_bitslice.cu) and compiles the result with NVRTC for sm_103a.
//
// State layout of one thread's 32-bit word: bit j of the word is the state
// whose BS_ELL lane arcs follow the bits of j.  The BS_TB thread arcs follow
// the bits of the warp lane id, the BS_L walk arcs are walked in reflected
// Gray order, and the BS_D prefix arcs are fixed per work item (one item per
// warp, from an atomic ticket: the equal division of Sec. 4.3).
//
// Per word the connectivity of all 32 states is one evaluation of the
// straight-line program: c = bs_var(inv, walk words), bit j of c set iff the
// sink is reachable from the source in state j (PLSA reachability, Sec.
// 3.2).  R (Eq. 1) accumulates exactly: the lane mass of the connected bits
// comes from four byte tables (u64, scale 2^62), times the walk mass of g
// (u64, scale 2^63), into a 128-bit integer per thread; the prefix and
// thread-arc masses are applied once per item in double-double.
#pragma once

namespace pbat {

static const char* kBsTemplate = R"PBAT(
typedef unsigned int u32;
typedef unsigned long long u64;

struct dd { double hi, lo; };
__device__ __forceinline__ dd two_sum(double a, double b) {
  double s = a + b; double bb = s - a; double e = (a - (s - bb)) + (b - bb); return dd{s, e};
}
__device__ __forceinline__ dd fast_two_sum(double a, double b) {
  double s = a + b; double e = b - (s - a); return dd{s, e};
}
__device__ __forceinline__ dd two_prod(double a, double b) {
  double p = a * b; double e = fma(a, b, -p); return dd{p, e};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi); dd t = two_sum(a.lo, b.lo);
  s.lo += t.hi; s = fast_two_sum(s.hi, s.lo); s.lo += t.lo; return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi); p.lo += a.hi * b.lo + a.lo * b.hi; return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b); p.lo += a.lo * b; return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_ldexp(dd a, int e) { return dd{ldexp(a.hi, e), ldexp(a.lo, e)}; }

struct u128 { u64 lo, hi; };
__device__ __forceinline__ void u128_add(u128& a, u64 blo, u64 bhi) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(a.lo), "+l"(a.hi) : "l"(blo), "l"(bhi));
}
__device__ __forceinline__ dd u128_to_dd(u128 v) {
  double h = __ull2double_rd(v.hi);
  u64 hr = v.hi - (u64)h;
  dd r = two_sum(ldexp(h, 64), ldexp((double)hr, 64));
  return dd_add(r, two_sum(ldexp((double)(v.lo >> 32), 32), (double)(v.lo & 0xffffffffull)));
}

struct BsParams {
  u64 task_lo, n_tasks, budget_ns;
  int prune, pad;
  double p[64];
  dd q[64];
  dd thr_w[32];
  u64 binom[64];
};
struct BsWork {
  u64* counter; u32* status; u64* stats;
  dd* part_acc; u64* part_n; dd* out_acc; u64* out_n;
};

__device__ __forceinline__ u64 bs_timer() {
  u64 t; asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t)); return t;
}

__device__ __forceinline__ dd bs_warp_sum(dd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd w; w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o); w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = dd_add(v, w);
  }
  return v;
}

__device__ __forceinline__ dd bs_prefix_mass(const BsParams& P, u64 prefix) {
  dd w = dd{1.0, 0.0};
#pragma unroll 1
  for (int j = 0; j < BS_D; ++j) {
    const int k = BS_TOP + j;
    w = ((prefix >> j) & 1ull) ? dd_mul_d(w, P.p[k]) : dd_mul(w, P.q[k]);
  }
  return w;
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

extern "C" __global__ void __launch_bounds__(BS_NTHR)
bs_kernel(const __grid_constant__ BsParams P, const u64* __restrict__ lane_tab,
          const u64* __restrict__ wmid_tab, BsWork W) {
  extern __shared__ __align__(16) unsigned char smem[];
  // lane tables: [4 bytes][256 values][3]: R (scale 2^62), N classes 0-2, N classes 3-5
  u64* s_lt = (u64*)smem;
  u64* s_wmid = s_lt + 4 * 256 * 3;
  u64* s_bins = s_wmid + (1 << BS_L);             // [(BS_L + 1) * 2][BS_NTHR]
  dd* s_wacc = (dd*)(s_bins + (BS_L + 1) * 2 * BS_NTHR);  // [warps][1 + BS_M]
  u64* s_nbins = (u64*)(s_wacc + (BS_NTHR / 32) * (1 + BS_M));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 4 * 256 * 3; i += BS_NTHR) s_lt[i] = lane_tab[i];
  for (int i = tid; i < (1 << BS_L); i += BS_NTHR) s_wmid[i] = wmid_tab[i];
  for (int i = tid; i < (BS_NTHR / 32) * (1 + BS_M); i += BS_NTHR) s_wacc[i] = dd{0.0, 0.0};
  for (int i = tid; i <= BS_M; i += BS_NTHR) s_nbins[i] = 0ull;
  __syncthreads();
  dd* wacc = s_wacc + warp * (1 + BS_M);
  u64* bins = s_bins + tid;
  const bool thr_on = lane < (1 << BS_TB);
  const int pc_thr = __popc(lane & ((1 << BS_TB) - 1));
  const dd thr_w = thr_on ? P.thr_w[lane] : dd{0.0, 0.0};
  const u64 t_start = bs_timer();
  u64 n_walk = 0, n_full = 0, n_dead = 0;
  u32 a[BS_M];
  // lane arcs: fixed patterns over the 32 bits of the word
#pragma unroll
  for (int i = 0; i < BS_ELL; ++i)
    a[i] = i == 0 ? 0xAAAAAAAAu : i == 1 ? 0xCCCCCCCCu : i == 2 ? 0xF0F0F0F0u : i == 3 ? 0xFF00FF00u : 0xFFFF0000u;
  // thread arcs: all-ones or all-zeros from the lane id
#pragma unroll
  for (int i = 0; i < BS_TB; ++i) a[BS_ELL + i] = 0u - (u32)((lane >> i) & 1);
#pragma unroll
  for (int b = 0; b < BS_L; ++b) a[BS_WALK0 + b] = 0u;

  for (;;) {
    u64 task = 0;
    if (lane == 0) {
      task = atomicAdd(W.counter, 1ull);
      if (P.budget_ns && bs_timer() - t_start > P.budget_ns) { atomicOr(W.status, 1u); task = ~0ull; }
    }
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= P.n_tasks) break;
    const u64 prefix = P.task_lo + task;
#pragma unroll
    for (int j = 0; j < BS_D; ++j) a[BS_TOP + j] = 0u - (u32)((prefix >> j) & 1ull);
    const dd wpre = bs_prefix_mass(P, prefix);
    const int pc_pre = __popcll((long long)prefix);
    if (P.prune) {
      u32 u[BS_M];
#pragma unroll
      for (int k = 0; k < BS_M; ++k) u[k] = k < BS_TOP ? ~0u : a[k];
      if (bs_uniform(u) == 0u) { ++n_dead; continue; }
#pragma unroll
      for (int k = 0; k < BS_M; ++k) u[k] = k < BS_TOP ? 0u : a[k];
      if (bs_uniform(u) != 0u) {
        ++n_full;
        for (int j = lane; j <= BS_TOP; j += 32) atomicAdd(&s_nbins[pc_pre + j], P.binom[j]);
        if (lane == 0) wacc[0] = dd_add(wacc[0], wpre);
        continue;
      }
    }
    ++n_walk;
    u32 e[BS_NCORE > 0 ? BS_NCORE : 1];
    bs_inv(a, e);
#pragma unroll
    for (int r = 0; r < (BS_L + 1) * 2; ++r) bins[r * BS_NTHR] = 0ull;
    u128 T = u128{0ull, 0ull};
    u32 g = 0;
    int pc = 0;
#pragma unroll 1
    for (u32 s = 0; s < (1u << BS_L); ++s) {
      if (s) {
        const int b = __ffs(s) - 1;
        g ^= 1u << b;
        pc += ((g >> b) & 1u) ? 1 : -1;
      }
      u32 w[BS_L > 0 ? BS_L : 1];
#pragma unroll
      for (int b = 0; b < BS_L; ++b) w[b] = 0u - ((g >> b) & 1u);
      u32 c = bs_var(e, w) & BS_LANE_MASK;
      if (c) {
        const u64* t0 = s_lt + (0 * 256 + (c & 0xffu)) * 3;
        const u64* t1 = s_lt + (1 * 256 + ((c >> 8) & 0xffu)) * 3;
        const u64* t2 = s_lt + (2 * 256 + ((c >> 16) & 0xffu)) * 3;
        const u64* t3 = s_lt + (3 * 256 + (c >> 24)) * 3;
        const u64 sR = t0[0] + t1[0] + t2[0] + t3[0];
        const u64 n0 = t0[1] + t1[1] + t2[1] + t3[1];
        const u64 n1 = t0[2] + t1[2] + t2[2] + t3[2];
        const u64 wm = s_wmid[g];
        u128_add(T, sR * wm, __umul64hi(sR, wm));
        bins[(2 * pc) * BS_NTHR] += n0;
        bins[(2 * pc + 1) * BS_NTHR] += n1;
      }
    }
    if (thr_on) {
      const int base = pc_pre + pc_thr;
#pragma unroll 1
      for (int r = 0; r <= BS_L; ++r) {
        const u64 n0 = bins[(2 * r) * BS_NTHR], n1 = bins[(2 * r + 1) * BS_NTHR];
#pragma unroll
        for (int cl = 0; cl < 3; ++cl) {
          const u64 c0 = (n0 >> (21 * cl)) & 0x1fffffull, c1 = (n1 >> (21 * cl)) & 0x1fffffull;
          if (c0) atomicAdd(&s_nbins[base + r + cl], c0);
          if (c1) atomicAdd(&s_nbins[base + r + 3 + cl], c1);
        }
      }
    }
    const dd t = dd_ldexp(u128_to_dd(T), -125);
    const dd ws = bs_warp_sum(dd_mul(thr_w, t));
    if (lane == 0) wacc[0] = dd_add(wacc[0], dd_mul(wpre, ws));
  }
  if (lane == 0) {
    atomicAdd(&W.stats[0], n_walk); atomicAdd(&W.stats[1], n_full); atomicAdd(&W.stats[2], n_dead);
  }
  __syncthreads();
  for (int i = tid; i <= BS_M; i += BS_NTHR) {
    dd s = dd{0.0, 0.0};
    for (int w = 0; w < BS_NTHR / 32; ++w) s = dd_add(s, s_wacc[w * (1 + BS_M) + i]);
    W.part_acc[(size_t)blockIdx.x * (1 + BS_M) + i] = s;
    W.part_n[(size_t)blockIdx.x * (BS_M + 1) + i] = s_nbins[i];
  }
}

#if BS_GRAD
// ---------------------------------------------------------------------------
// Fused R + N_k + dR/dp.  Every gradient term is a difference of two exact
// integer sums over the two halves of a pair of states (X, X + e_i) that
// carry identical weights, so it is exact and non-negative:
//   thread arcs: per-thread totals T of warp lanes t and t ^ 2^i;
//   lane arcs: the 32x32 bit matrix (threads x lanes) of a word is
//     transposed across the warp, so lane j holds the states of lane pattern
//     j; its total T' (thread-arc masses from byte tables) pairs lanes j and
//     j ^ 2^i in the same way;
//   walk arcs: A_b, the part of T collected while walk arc b works (T
//     subtracted when it turns on, added when it turns off), against
//     T - A_b, divided by p_b and 1 - p_b in double-double;
//   prefix arcs: item totals in double-double, added with sign.
// Walk masses are 128-bit here (scale 2^127), so the division by p_b or
// 1 - p_b leaves an error far below 2^-100.
struct BsGradParams {
  dd thr_w_ex[5][32];
  dd lane_w_ex[5][32];
  dd inv_p[64], inv_q[64];
};

__device__ __forceinline__ u32 bs_transpose32(u32 x, int lane) {
  const u32 masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const int sh = 16 >> r;
    const u32 mk = masks[r];
    const u32 y = __shfl_xor_sync(0xffffffffu, x, sh);
    x = (lane & sh) ? ((x & ~mk) | ((y & ~mk) >> sh)) : ((x & mk) | ((y & mk) << sh));
  }
  return x;
}

// (a * b) >> 64 for a 64-bit a and a 128-bit b, as 128 bits
__device__ __forceinline__ void mul64x128_shr64(u64 a, u64 blo, u64 bhi, u64& rlo, u64& rhi) {
  const u64 h0 = __umul64hi(a, blo);
  const u64 l1 = a * bhi;
  const u64 h1 = __umul64hi(a, bhi);
  asm("add.cc.u64 %0, %2, %3;\n\taddc.u64 %1, %4, 0;" : "=l"(rlo), "=l"(rhi) : "l"(l1), "l"(h0), "l"(h1));
}

__device__ __forceinline__ double u128_to_double(u128 v) {
  return fma((double)v.hi, 18446744073709551616.0, (double)v.lo);
}

__device__ __forceinline__ double bs_warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ u128 shfl_u128(u128 v, int src_lane_xor) {
  u128 r;
  r.lo = __shfl_xor_sync(0xffffffffu, v.lo, src_lane_xor);
  r.hi = __shfl_xor_sync(0xffffffffu, v.hi, src_lane_xor);
  return r;
}

__device__ __forceinline__ u128 u128_sub(u128 a, u128 b) {
  u128 r;
  asm("sub.cc.u64 %0, %2, %4;\n\tsubc.u64 %1, %3, %5;" : "=l"(r.lo), "=l"(r.hi) : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
  return r;
}

__device__ __forceinline__ dd bs_prefix_mass_ex(const BsParams& P, u64 prefix, int skip) {
  dd w = dd{1.0, 0.0};
#pragma unroll 1
  for (int j = 0; j < BS_D; ++j) {
    if (j == skip) continue;
    const int k = BS_TOP + j;
    w = ((prefix >> j) & 1ull) ? dd_mul_d(w, P.p[k]) : dd_mul(w, P.q[k]);
  }
  return w;
}

extern "C" __global__ void __launch_bounds__(BS_NTHR)
bs_kernel_grad(const __grid_constant__ BsParams P, const __grid_constant__ BsGradParams Q,
               const u64* __restrict__ lane_tab, const u64* __restrict__ thr_tab,
               const u64* __restrict__ wmid128, BsWork W) {
  extern __shared__ __align__(16) unsigned char smem[];
  u64* s_lt = (u64*)smem;                          // [4][256][3]
  u64* s_tt = s_lt + 4 * 256 * 3;                  // [4][256] thread-pattern masses (2^62)
  u64* s_wm = s_tt + 4 * 256;                      // [2^L][2] walk masses (2^127)
  u64* s_bins = s_wm + 2 * (1 << BS_L);            // [(L + 1) * 2][NTHR]
  u128* s_A = (u128*)(s_bins + (BS_L + 1) * 2 * BS_NTHR);  // [L][NTHR]
  dd* s_wacc = (dd*)(s_A + (BS_L > 0 ? BS_L : 1) * BS_NTHR);
  u64* s_nbins = (u64*)(s_wacc + (BS_NTHR / 32) * (1 + BS_M));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 4 * 256 * 3; i += BS_NTHR) s_lt[i] = lane_tab[i];
  for (int i = tid; i < 4 * 256; i += BS_NTHR) s_tt[i] = thr_tab[i];
  for (int i = tid; i < 2 * (1 << BS_L); i += BS_NTHR) s_wm[i] = wmid128[i];
  for (int i = tid; i < (BS_NTHR / 32) * (1 + BS_M); i += BS_NTHR) s_wacc[i] = dd{0.0, 0.0};
  for (int i = tid; i <= BS_M; i += BS_NTHR) s_nbins[i] = 0ull;
  __syncthreads();
  dd* wacc = s_wacc + warp * (1 + BS_M);
  u64* bins = s_bins + tid;
  u128* A = s_A + tid;
  const bool thr_on = lane < (1 << BS_TB);
  const int pc_thr = __popc(lane & ((1 << BS_TB) - 1));
  const dd thr_w = thr_on ? P.thr_w[lane] : dd{0.0, 0.0};
  const u64 t_start = bs_timer();
  u64 n_walk = 0, n_full = 0, n_dead = 0;
  u32 a[BS_M];
#pragma unroll
  for (int i = 0; i < BS_ELL; ++i)
    a[i] = i == 0 ? 0xAAAAAAAAu : i == 1 ? 0xCCCCCCCCu : i == 2 ? 0xF0F0F0F0u : i == 3 ? 0xFF00FF00u : 0xFFFF0000u;
#pragma unroll
  for (int i = 0; i < BS_TB; ++i) a[BS_ELL + i] = 0u - (u32)((lane >> i) & 1);
#pragma unroll
  for (int b = 0; b < BS_L; ++b) a[BS_WALK0 + b] = 0u;

  for (;;) {
    u64 task = 0;
    if (lane == 0) {
      task = atomicAdd(W.counter, 1ull);
      if (P.budget_ns && bs_timer() - t_start > P.budget_ns) { atomicOr(W.status, 1u); task = ~0ull; }
    }
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= P.n_tasks) break;
    const u64 prefix = P.task_lo + task;
#pragma unroll
    for (int j = 0; j < BS_D; ++j) a[BS_TOP + j] = 0u - (u32)((prefix >> j) & 1ull);
    const dd wpre = bs_prefix_mass(P, prefix);
    const int pc_pre = __popcll((long long)prefix);
    if (P.prune) {
      u32 u[BS_M];
#pragma unroll
      for (int k = 0; k < BS_M; ++k) u[k] = k < BS_TOP ? ~0u : a[k];
      if (bs_uniform(u) == 0u) { ++n_dead; continue; }
#pragma unroll
      for (int k = 0; k < BS_M; ++k) u[k] = k < BS_TOP ? 0u : a[k];
      if (bs_uniform(u) != 0u) {
        ++n_full;
        for (int j = lane; j <= BS_TOP; j += 32) atomicAdd(&s_nbins[pc_pre + j], P.binom[j]);
        if (lane == 0) wacc[0] = dd_add(wacc[0], wpre);
        for (int j = lane; j < BS_D; j += 32) {
          const dd ex = bs_prefix_mass_ex(P, prefix, j);
          wacc[1 + BS_TOP + j] = ((prefix >> j) & 1ull) ? dd_add(wacc[1 + BS_TOP + j], ex)
                                                         : dd_add(wacc[1 + BS_TOP + j], dd{-ex.hi, -ex.lo});
        }
        continue;
      }
    }
    ++n_walk;
    u32 e[BS_NCORE > 0 ? BS_NCORE : 1];
    bs_inv(a, e);
#pragma unroll
    for (int r = 0; r < (BS_L + 1) * 2; ++r) bins[r * BS_NTHR] = 0ull;
#pragma unroll
    for (int b = 0; b < BS_L; ++b) A[b * BS_NTHR] = u128{0ull, 0ull};
    u128 T = u128{0ull, 0ull}, T2 = u128{0ull, 0ull};
    u32 g = 0;
    int pc = 0;
#pragma unroll 1
    for (u32 s = 0; s < (1u << BS_L); ++s) {
      if (s) {
        const int b = __ffs(s) - 1;
        g ^= 1u << b;
        const bool on = (g >> b) & 1u;
        pc += on ? 1 : -1;
        // walk arc b: A_b collects the growth of T while arc b works
        u128 ab = A[b * BS_NTHR];
        if (on) ab = u128_sub(ab, T); else u128_add(ab, T.lo, T.hi);
        A[b * BS_NTHR] = ab;
      }
      u32 w[BS_L > 0 ? BS_L : 1];
#pragma unroll
      for (int b = 0; b < BS_L; ++b) w[b] = 0u - ((g >> b) & 1u);
      const u32 c = bs_var(e, w) & BS_LANE_MASK;
      const u32 ct = bs_transpose32(c, lane);
      const u64 wlo = s_wm[2 * g], whi = s_wm[2 * g + 1];
      if (c) {
        const u64* t0 = s_lt + (0 * 256 + (c & 0xffu)) * 3;
        const u64* t1 = s_lt + (1 * 256 + ((c >> 8) & 0xffu)) * 3;
        const u64* t2 = s_lt + (2 * 256 + ((c >> 16) & 0xffu)) * 3;
        const u64* t3 = s_lt + (3 * 256 + (c >> 24)) * 3;
        const u64 sR = t0[0] + t1[0] + t2[0] + t3[0];
        u64 plo, phi;
        mul64x128_shr64(sR, wlo, whi, plo, phi);
        u128_add(T, plo, phi);
        bins[(2 * pc) * BS_NTHR] += t0[1] + t1[1] + t2[1] + t3[1];
        bins[(2 * pc + 1) * BS_NTHR] += t0[2] + t1[2] + t2[2] + t3[2];
      }
      if (ct) {
        const u64 s2 = s_tt[ct & 0xffu] + s_tt[256 + ((ct >> 8) & 0xffu)] +
                       s_tt[512 + ((ct >> 16) & 0xffu)] + s_tt[768 + (ct >> 24)];
        u64 plo, phi;
        mul64x128_shr64(s2, wlo, whi, plo, phi);
        u128_add(T2, plo, phi);
      }
    }
    // walk arcs still working at the end of the walk close their segment
#pragma unroll
    for (int b = 0; b < BS_L; ++b)
      if ((g >> b) & 1u) { u128 ab = A[b * BS_NTHR]; u128_add(ab, T.lo, T.hi); A[b * BS_NTHR] = ab; }
    if (thr_on) {
      const int base = pc_pre + pc_thr;
#pragma unroll 1
      for (int r = 0; r <= BS_L; ++r) {
        const u64 n0 = bins[(2 * r) * BS_NTHR], n1 = bins[(2 * r + 1) * BS_NTHR];
#pragma unroll
        for (int cl = 0; cl < 3; ++cl) {
          const u64 c0 = (n0 >> (21 * cl)) & 0x1fffffull, c1 = (n1 >> (21 * cl)) & 0x1fffffull;
          if (c0) atomicAdd(&s_nbins[base + r + cl], c0);
          if (c1) atomicAdd(&s_nbins[base + r + 3 + cl], c1);
        }
      }
    }
    // ---- item epilogue
    const dd t = dd_ldexp(u128_to_dd(T), -125);
    const dd S = bs_warp_sum(dd_mul(thr_w, t));      // sum over threads of thread mass * T
    if (lane == 0) wacc[0] = dd_add(wacc[0], dd_mul(wpre, S));
    for (int j = lane; j < BS_D; j += 32) {
      const dd ex = dd_mul(bs_prefix_mass_ex(P, prefix, j), S);
      wacc[1 + BS_TOP + j] = ((prefix >> j) & 1ull) ? dd_add(wacc[1 + BS_TOP + j], ex)
                                                     : dd_add(wacc[1 + BS_TOP + j], dd{-ex.hi, -ex.lo});
    }
    const double sc = 2.3509887016445750e-38;  // 2^-125
#pragma unroll
    for (int i = 0; i < BS_TB; ++i) {
      const u128 o = shfl_u128(T, 1 << i);
      double y = 0.0;
      if (((lane >> i) & 1) && thr_on) y = u128_to_double(u128_sub(T, o)) * sc * Q.thr_w_ex[i][lane].hi;
      y = bs_warp_sum_d(y);
      if (lane == i) wacc[1 + BS_ELL + i] = dd_add(wacc[1 + BS_ELL + i], dd_mul_d(wpre, y));
    }
#pragma unroll
    for (int i = 0; i < BS_ELL; ++i) {
      const u128 o = shfl_u128(T2, 1 << i);
      double y = 0.0;
      if ((lane >> i) & 1) y = u128_to_double(u128_sub(T2, o)) * sc * Q.lane_w_ex[i][lane].hi;
      y = bs_warp_sum_d(y);
      if (lane == i) wacc[1 + i] = dd_add(wacc[1 + i], dd_mul_d(wpre, y));
    }
#pragma unroll 1
    for (int b = 0; b < BS_L; ++b) {
      const int k = BS_WALK0 + b;
      const u128 Ab = A[b * BS_NTHR];
      const dd av = u128_to_dd(Ab), zv = u128_to_dd(u128_sub(T, Ab));
      const dd yv = dd_add(dd_mul(av, Q.inv_p[k]), dd{-(dd_mul(zv, Q.inv_q[k])).hi, -(dd_mul(zv, Q.inv_q[k])).lo});
      double y = thr_on ? dd_mul(dd_ldexp(yv, -125), thr_w).hi : 0.0;
      y = bs_warp_sum_d(y);
      if (lane == (k & 31)) wacc[1 + k] = dd_add(wacc[1 + k], dd_mul_d(wpre, y));
    }
  }
  if (lane == 0) {
    atomicAdd(&W.stats[0], n_walk); atomicAdd(&W.stats[1], n_full); atomicAdd(&W.stats[2], n_dead);
  }
  __syncthreads();
  for (int i = tid; i <= BS_M; i += BS_NTHR) {
    dd sacc = dd{0.0, 0.0};
    for (int w2 = 0; w2 < BS_NTHR / 32; ++w2) sacc = dd_add(sacc, s_wacc[w2 * (1 + BS_M) + i]);
    W.part_acc[(size_t)blockIdx.x * (1 + BS_M) + i] = sacc;
    W.part_n[(size_t)blockIdx.x * (BS_M + 1) + i] = s_nbins[i];
  }
}
#endif
)PBAT";

}  // namespace pbat
