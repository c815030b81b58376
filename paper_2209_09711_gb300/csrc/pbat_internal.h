// pbat_internal.h -- structures shared by the host engine and the kernels.
#pragma once
#include <stdint.h>
#include <string>
#include <vector>

#include "pbat_num.cuh"

namespace pbat {

constexpr int kMaxNodes = 64;
constexpr int kMaxArcs = 63;
constexpr int kMaxLaneBits = 5;       // one warp lane per low-arc pattern
constexpr int kMaxWalkBitsR = 12;     // Gray-walk arcs per thread, R only
constexpr int kMaxWalkBitsGrad = 10;  // with the gradient segment sums

// Everything a frontier-kernel launch needs that is not a table, passed by
// value (it lives in the kernel parameter bank, read with uniform indices).
// Arc index k below is the INTERNAL arc position: bit k of a state word.
// Internal layout of a state word, low to high bits:
//   [lane arcs: lane_bits][walk arcs: walk_bits][prefix arcs: prefix_bits]
struct FrontierParams {
  int n, m, directed, source, sink;
  int lane_bits, walk_bits, prefix_bits;
  int prune;
  int pad0;
  unsigned long long task_lo;   // first prefix value
  unsigned long long n_tasks;   // number of prefix values (work items)
  unsigned long long budget_ns; // 0 = no deadline
  unsigned long long free_mask; // bits of lane + walk arcs
  unsigned char au[64], av[64]; // arc endpoints (tail, head)
  unsigned long long grp[64];   // arcs joining the same node pair (same direction if directed)
  double p[64];                 // p_k
  dd q[64];                     // 1 - p_k, exact
  dd inv_p[64], inv_q[64];      // 1/p_k, 1/(1-p_k) for walk arcs (gradient)
  dd lane_w[32];                // mass of each lane pattern: prod over lane arcs
  dd lane_w_ex[kMaxLaneBits][32];  // the same without lane arc i's factor
  unsigned long long binom[64];    // C(lane_bits + walk_bits, j)
};

// Device scratch of one launch.
struct DevWork {
  unsigned long long* counter;  // work-item ticket
  unsigned int* status;         // bit 0: deadline hit
  unsigned long long* stats;    // [0] walked items, [1] full items, [2] dead items
  dd* part_acc;                 // [grid][n_acc]: R, then per internal arc dR/dp (frontier)
                                //   or the two sums A, B (fused bit-sliced kernel)
  unsigned long long* part_n;   // [grid][m + 1]
  dd* out_acc;                  // [n_acc]
  unsigned long long* out_n;    // [m + 1]
  void* wacc;                   // fused bit-sliced kernel: per-warp accumulators (24 B each)
  unsigned long long* out_limbs;  // bit-sliced kernels: [n_acc][8] 256-bit fixed point, scale 2^250
  // two-phase bit-sliced launches: the first defers the items its prune
  // leaves to walk to `list` (capacity list_cap, count list_n), the second
  // walks them, taking them by the ticket counter2
  unsigned long long* list;
  unsigned long long list_cap;
  unsigned long long* list_n;
  unsigned long long* counter2;
};

}  // namespace pbat
