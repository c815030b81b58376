// pbat_bs_plan.h -- role assignment and generated connectivity program of
// the bit-sliced kernels (pbat_bs_plan.cu), shared with their launcher.
#pragma once
#include <string>
#include <vector>

#include "pbat_engine.h"

namespace pbat {

// Which arcs are lane / thread / walk / prefix arcs, and the generated
// bs_inv / bs_var connectivity program for that assignment.
struct BsPlan {
  bool grad = false;
  int ell = 0, tb = 0, L = 0, d = 0, r = 0;
  int minb = 0;           // __launch_bounds__ minimum blocks per SM (0: none)
  // fused kernel: internal prefix arcs whose p is outside [2^-20, 1 - 2^-20]
  // (their sums use the excluded-arc tables instead of dividing by p, 1 - p)
  unsigned long long pex = 0;
  std::vector<int> perm;  // internal position -> input arc
  std::string gen;        // generated bs_inv / bs_var
  int ncore = 0, ops_inv = 0, ops_var = 0;
};

// The fused kernel divides walk masses by p and 1 - p: an arc may be a walk
// arc of the gradient only with p in [2^-20, 1 - 2^-20].
bool bs_walk_ok(const double* p, int a);

// Plan one network for the bit-sliced kernels (Sec. 4.3 equal division:
// lane, thread, walk and prefix arcs, range arcs on top) and generate its
// connectivity program.  p_for_grad: the reliabilities when planning the
// fused kernel (walk arcs must pass bs_walk_ok), else null.
int bs_make_plan(const GraphIn& g, const pbat_options& o, int nthr, BsPlan& bp,
                 const double* p_for_grad);

}  // namespace pbat
