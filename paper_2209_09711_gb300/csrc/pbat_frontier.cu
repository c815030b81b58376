// pbat_frontier.cu -- the per-state PBAT kernel and the final reduction.
//
// Work decomposition (equal division, arXiv 2209.09711 Sec. 4.3, Eq. 6-7):
// the top `prefix_bits` arcs of the state word form a prefix; each prefix
// value is one work item, taken by one warp from an atomic ticket.  Inside
// an item, lane j fixes the `lane_bits` lowest arcs to the pattern j and
// walks the `walk_bits` middle arcs in reflected Gray-code order, so every
// step changes exactly one arc (the BAT of Sec. 3.1 visits the same set of
// vectors in binary order; only the set matters for Eq. 1).
//
// Per state, connectivity is the PLSA of Sec. 3.2 done as frontier
// expansion on node bitmasks: adj[u] (one word per node, per thread, in
// shared memory) holds u's working out-neighbours; the frontier pops its
// lowest node with ffs, adds adj[u] minus the visited set, and stops when the
// sink appears or the frontier empties.  Monotonicity skips the search when
// the flipped arc cannot change the answer (an arc added to a connected
// state, or removed from a disconnected one).
//
// Accumulation is exact: the walk-arc mass of every walk pattern g is a
// 128-bit fixed-point table entry W[g] ~ 2^127 * prod_{walk arcs} w(g), and a
// thread adds W[g] for each connected state into a 128-bit integer T.  The
// prefix and lane factors are applied once per item in double-double.  N_k
// is a per-thread histogram by the popcount of g.  The gradient of Eq. 1
// (PBAT differentiated term by term) needs, for every walk arc b, the mass
// A_b of connected states with that arc working; Gray order makes this one
// update per step: when arc b turns on, remember T; when it turns off, add
// the growth of T since then.  Being integer, these differences are exact.
//
// Exact monotone prune per item: with every free (lane + walk) arc working
// the sink is unreachable -> the whole item contributes nothing; with every
// free arc failed it is reachable -> the item adds its closed-form mass
// Pr(prefix), C(f, j) states with |prefix| + j working arcs, and gradient
// terms for the prefix arcs only (free arcs have zero derivative there).
#include <cuda_runtime.h>

#include "pbat_internal.h"

namespace pbat {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename M>
__device__ __forceinline__ int lowest_node(M x);
template <>
__device__ __forceinline__ int lowest_node<uint32_t>(uint32_t x) {
  return __ffs(x) - 1;
}
template <>
__device__ __forceinline__ int lowest_node<unsigned long long>(unsigned long long x) {
  return __ffsll((long long)x) - 1;
}

// Frontier expansion (PLSA, Sec. 3.2) on this thread's adjacency rows.
template <typename M>
__device__ __forceinline__ bool sink_reached(const M* adj, int stride, M sbit, M tbit) {
  M vis = sbit, fr = sbit;
  while (fr) {
    const int u = lowest_node<M>(fr);
    fr &= fr - 1;
    const M nb = adj[u * stride] & ~vis;
    if (nb & tbit) return true;
    vis |= nb;
    fr |= nb;
  }
  return false;
}

// Reachability of one arbitrary state, computed identically by every lane
// (used twice per work item by the prune).  Repeated passes over the arc
// list until nothing changes.
__device__ __noinline__ bool state_connected(const FrontierParams& P, unsigned long long x) {
  unsigned long long reach = 1ull << P.source;
  const unsigned long long tb = 1ull << P.sink;
  for (int pass = 0; pass < P.n; ++pass) {
    const unsigned long long before = reach;
    for (int k = 0; k < P.m; ++k) {
      if (!((x >> k) & 1ull)) continue;
      const unsigned long long bu = 1ull << P.au[k], bv = 1ull << P.av[k];
      if (reach & bu) reach |= bv;
      if (!P.directed && (reach & bv)) reach |= bu;
    }
    if (reach & tb) return true;
    if (reach == before) return false;
  }
  return (reach & tb) != 0;
}

__device__ __forceinline__ dd warp_sum(dd v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = dd_add(v, w);
  }
  return v;
}

// Mass of the prefix arcs of `prefix`, optionally without prefix arc `skip`.
__device__ __forceinline__ dd prefix_mass(const FrontierParams& P, unsigned long long prefix,
                                          int skip) {
  const int base = P.lane_bits + P.walk_bits;
  dd w = dd{1.0, 0.0};
  for (int j = 0; j < P.prefix_bits; ++j) {
    if (j == skip) continue;
    const int k = base + j;
    w = ((prefix >> j) & 1ull) ? dd_mul_d(w, P.p[k]) : dd_mul(w, P.q[k]);
  }
  return w;
}

__device__ __forceinline__ void acc_signed(dd& slot, dd v, bool plus) {
  slot = plus ? dd_add(slot, v) : dd_sub(slot, v);
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename M, bool GRAD>
__global__ void __launch_bounds__(256) frontier_kernel(const __grid_constant__ FrontierParams P,
                                                       const u128* __restrict__ wmid_g,
                                                       DevWork W) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = P.walk_bits, ell = P.lane_bits, n = P.n, m = P.m;
  const int nthr = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  const int nW = 1 << L;

  size_t off = 0;
  u128* s_wmid = reinterpret_cast<u128*>(smem + off);
  off = align16(off + (size_t)nW * sizeof(u128));
  M* s_adj = reinterpret_cast<M*>(smem + off);
  off = align16(off + (size_t)n * nthr * sizeof(M));
  uint32_t* s_ncnt = reinterpret_cast<uint32_t*>(smem + off);
  off = align16(off + (size_t)(L + 1) * nthr * sizeof(uint32_t));
  u128* s_seg = reinterpret_cast<u128*>(smem + off);
  if (GRAD) off = align16(off + (size_t)2 * L * nthr * sizeof(u128));
  dd* s_wacc = reinterpret_cast<dd*>(smem + off);
  off = align16(off + (size_t)nwarps * (1 + m) * sizeof(dd));
  unsigned long long* s_nbins = reinterpret_cast<unsigned long long*>(smem + off);

  for (int i = tid; i < nW; i += nthr) s_wmid[i] = wmid_g[i];
  for (int i = tid; i < nwarps * (1 + m); i += nthr) s_wacc[i] = dd{0.0, 0.0};
  for (int i = tid; i <= m; i += nthr) s_nbins[i] = 0ull;
  __syncthreads();

  M* adj = s_adj + tid;
  uint32_t* ncnt = s_ncnt + tid;
  u128* seg_start = s_seg + tid;
  u128* seg_acc = s_seg + (size_t)L * nthr + tid;
  dd* wacc = s_wacc + (size_t)warp * (1 + m);
  const M sbit = (M)1 << P.source, tbit = (M)1 << P.sink;
  const bool lane_on = lane < (1 << ell);
  const int top = ell + L;  // first prefix arc
  const unsigned long long t_start = globaltimer_ns();
  unsigned long long n_walk = 0, n_full = 0, n_dead = 0;

  for (;;) {
    unsigned long long task = 0;
    if (lane == 0) {
      task = atomicAdd(W.counter, 1ull);
      if (P.budget_ns && globaltimer_ns() - t_start > P.budget_ns) {
        atomicOr(W.status, 1u);
        task = ~0ull;
      }
    }
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= P.n_tasks) break;
    const unsigned long long prefix = P.task_lo + task;
    const unsigned long long xpre = top < 64 ? (prefix << top) : 0ull;
    const dd wpre = prefix_mass(P, prefix, -1);
    const int pc_pre = __popcll((long long)prefix);

    if (P.prune) {
      if (!state_connected(P, xpre | P.free_mask)) {
        ++n_dead;
        continue;
      }
      if (state_connected(P, xpre)) {
        ++n_full;
        for (int j = lane; j <= top; j += 32) atomicAdd(&s_nbins[pc_pre + j], P.binom[j]);
        if (lane == 0) wacc[0] = dd_add(wacc[0], wpre);
        if (GRAD) {
          for (int j = lane; j < P.prefix_bits; j += 32)
            acc_signed(wacc[1 + top + j], prefix_mass(P, prefix, j), (prefix >> j) & 1ull);
        }
        continue;
      }
    }
    ++n_walk;

    // ---- Gray walk of the middle arcs, one state per step
    unsigned long long x = xpre | (unsigned long long)(lane_on ? lane : 0);
    for (int u = 0; u < n; ++u) adj[u * nthr] = (M)0;
    for (int k = 0; k < m; ++k) {
      if ((x >> k) & 1ull) {
        adj[P.au[k] * nthr] |= (M)1 << P.av[k];
        if (!P.directed) adj[P.av[k] * nthr] |= (M)1 << P.au[k];
      }
    }
    bool conn = sink_reached<M>(adj, nthr, sbit, tbit);
    u128 T = u128_zero();
    for (int c = 0; c <= L; ++c) ncnt[c * nthr] = 0u;
    if (GRAD) {
      for (int b = 0; b < L; ++b) {
        seg_start[b * nthr] = u128_zero();
        seg_acc[b * nthr] = u128_zero();
      }
    }
    if (conn) {
      u128_add_to(T, s_wmid[0]);
      ncnt[0] += 1u;
    }
    uint32_t g = 0;
    int pc = 0;
    for (uint32_t s = 1; s < (uint32_t)nW; ++s) {
      const int b = __ffs(s) - 1;
      const int k = ell + b;
      const unsigned long long bit = 1ull << k;
      x ^= bit;
      g ^= 1u << b;
      const bool added = (x & bit) != 0ull;
      const int u = P.au[k], v = P.av[k];
      const bool present = (x & P.grp[k]) != 0ull;
      M* ru = adj + u * nthr;
      *ru = present ? (*ru | ((M)1 << v)) : (*ru & ~((M)1 << v));
      if (!P.directed) {
        M* rv = adj + v * nthr;
        *rv = present ? (*rv | ((M)1 << u)) : (*rv & ~((M)1 << u));
      }
      pc += added ? 1 : -1;
      if (added != conn) conn = sink_reached<M>(adj, nthr, sbit, tbit);
      if (GRAD) {
        if (added)
          seg_start[b * nthr] = T;
        else
          u128_add_to(seg_acc[b * nthr], u128_sub(T, seg_start[b * nthr]));
      }
      if (conn) {
        u128_add_to(T, s_wmid[g]);
        ncnt[pc * nthr] += 1u;
      }
    }
    // the walk ends on g = 2^(L-1): only the top walk arc is still working
    if (GRAD && L > 0) u128_add_to(seg_acc[(L - 1) * nthr], u128_sub(T, seg_start[(L - 1) * nthr]));

    // ---- item epilogue: histogram, then masses in double-double
    if (lane_on) {
      const int base = pc_pre + __popc(lane);
      for (int c = 0; c <= L; ++c) {
        const uint32_t cnt = ncnt[c * nthr];
        if (cnt) atomicAdd(&s_nbins[base + c], (unsigned long long)cnt);
      }
    }
    const dd t = dd_ldexp(u128_to_dd(T), -127);
    const dd lw = lane_on ? P.lane_w[lane] : dd{0.0, 0.0};
    const dd wsum = warp_sum(dd_mul(lw, t));
    if (lane == 0) wacc[0] = dd_add(wacc[0], dd_mul(wpre, wsum));
    if (GRAD) {
      for (int b = 0; b < L; ++b) {
        const int k = ell + b;
        const u128 A = seg_acc[b * nthr];
        const dd a = dd_ldexp(u128_to_dd(A), -127);
        const dd z = dd_ldexp(u128_to_dd(u128_sub(T, A)), -127);
        dd y = dd_sub(dd_mul(a, P.inv_p[k]), dd_mul(z, P.inv_q[k]));
        y = warp_sum(dd_mul(lw, y));
        if (lane == (k & 31)) wacc[1 + k] = dd_add(wacc[1 + k], dd_mul(wpre, y));
      }
      for (int i = 0; i < ell; ++i) {
        dd y = lane_on ? dd_mul(P.lane_w_ex[i][lane], t) : dd{0.0, 0.0};
        if (!((lane >> i) & 1)) y = dd_neg(y);
        y = warp_sum(y);
        if (lane == i) wacc[1 + i] = dd_add(wacc[1 + i], dd_mul(wpre, y));
      }
      for (int j = lane; j < P.prefix_bits; j += 32)
        acc_signed(wacc[1 + top + j], dd_mul(prefix_mass(P, prefix, j), wsum), (prefix >> j) & 1ull);
    }
  }

  if (lane == 0) {
    atomicAdd(&W.stats[0], n_walk);
    atomicAdd(&W.stats[1], n_full);
    atomicAdd(&W.stats[2], n_dead);
  }
  __syncthreads();
  for (int i = tid; i <= m; i += nthr) {
    dd s = dd{0.0, 0.0};
    for (int w = 0; w < nwarps; ++w) s = dd_add(s, s_wacc[(size_t)w * (1 + m) + i]);
    W.part_acc[(size_t)blockIdx.x * (1 + m) + i] = s;
    W.part_n[(size_t)blockIdx.x * (m + 1) + i] = s_nbins[i];
  }
}

// Fixed-order sum of the per-block partials (PBAT STEP 3).  One CTA per
// output value; thread t sums blocks t, t + 256, ... in order, then a fixed
// shared-memory tree combines the 256 partial sums, so the result does not
// depend on scheduling.
constexpr int kReduceThreads = 256;

// Output i sums entry i of every block's partials (n_acc double-double
// sums and n_cnt counts per block) in a fixed order.
__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(DevWork W, int nblocks, int n_acc, int n_cnt) {
  __shared__ dd s_acc[kReduceThreads];
  __shared__ unsigned long long s_n[kReduceThreads];
  const int i = blockIdx.x, t = threadIdx.x;
  dd s = dd{0.0, 0.0};
  unsigned long long c = 0ull;
  for (int b = t; b < nblocks; b += kReduceThreads) {
    if (i < n_acc) s = dd_add(s, W.part_acc[(size_t)b * n_acc + i]);
    if (i < n_cnt) c += W.part_n[(size_t)b * n_cnt + i];
  }
  s_acc[t] = s;
  s_n[t] = c;
  __syncthreads();
  for (int h = kReduceThreads / 2; h > 0; h >>= 1) {
    if (t < h) {
      s_acc[t] = dd_add(s_acc[t], s_acc[t + h]);
      s_n[t] += s_n[t + h];
    }
    __syncthreads();
  }
  if (t == 0) {
    if (i < n_acc) W.out_acc[i] = s_acc[0];
    if (i < n_cnt) W.out_n[i] = s_n[0];
  }
}

size_t frontier_smem_bytes(int n, int m, int L, int nthr, bool grad, bool wide) {
  size_t off = 0;
  off = align16(off + ((size_t)1 << L) * sizeof(u128));
  off = align16(off + (size_t)n * nthr * (wide ? 8 : 4));
  off = align16(off + (size_t)(L + 1) * nthr * sizeof(uint32_t));
  if (grad) off = align16(off + (size_t)2 * L * nthr * sizeof(u128));
  off = align16(off + (size_t)(nthr / 32) * (1 + m) * sizeof(dd));
  off += (size_t)(m + 1) * sizeof(unsigned long long);
  return off;
}

const void* frontier_kernel_ptr(bool grad, bool wide) {
  if (wide)
    return grad ? (const void*)frontier_kernel<unsigned long long, true>
                : (const void*)frontier_kernel<unsigned long long, false>;
  return grad ? (const void*)frontier_kernel<uint32_t, true>
              : (const void*)frontier_kernel<uint32_t, false>;
}

cudaError_t launch_frontier(bool grad, bool wide, int grid, int nthr, size_t smem,
                            cudaStream_t st, const FrontierParams& P, const u128* wmid,
                            const DevWork& W) {
  if (wide) {
    if (grad)
      frontier_kernel<unsigned long long, true><<<grid, nthr, smem, st>>>(P, wmid, W);
    else
      frontier_kernel<unsigned long long, false><<<grid, nthr, smem, st>>>(P, wmid, W);
  } else {
    if (grad)
      frontier_kernel<uint32_t, true><<<grid, nthr, smem, st>>>(P, wmid, W);
    else
      frontier_kernel<uint32_t, false><<<grid, nthr, smem, st>>>(P, wmid, W);
  }
  return cudaGetLastError();
}

cudaError_t launch_reduce(cudaStream_t st, const DevWork& W, int nblocks, int n_acc, int n_cnt) {
  reduce_kernel<<<n_acc > n_cnt ? n_acc : n_cnt, kReduceThreads, 0, st>>>(W, nblocks, n_acc, n_cnt);
  return cudaGetLastError();
}

}  // namespace pbat
