// pbat_bs_plan.cu -- planner and code generator of the bit-sliced
// enumeration kernels (their launcher is pbat_bitslice.cu).
//
// Connectivity as Boolean elimination.  For a fixed assignment of the
// non-lane arcs, each node pair (u, v) carries a 32-bit word E[u][v]: bit j
// set iff the pair is joined by a working arc in lane state j.  Eliminating
// a node k (neither source nor sink) replaces every path i -> k -> j by the
// shortcut E[i][j] |= E[i][k] & E[k][j] -- Gaussian elimination over the
// Boolean semiring, i.e. Floyd-Warshall restricted to the graph's sparsity.
// After every other node is gone, E[s][t] holds, for all 32 lane states at
// once, whether the sink is reachable from the source: the PLSA answer of
// Sec. 3.2, thirty-two states per 32-bit operation.  Loops the paper
// excludes never arise (i != j), and for directed graphs edges into the
// source or out of the sink are dropped (no s-t path uses them).
//
// The elimination program is specialised per graph and compiled with NVRTC,
// so every word lives in a register.  Nodes that touch no walk arc are
// eliminated first: those operations do not depend on the Gray walk and run
// once per work item (bs_inv); only the small "core" left around the source,
// the sink and the walk arcs is eliminated per word (bs_var).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <queue>
#include <string>
#include <vector>

#include "pbat.h"
#include "pbat_bs_plan.h"
#include "pbat_engine.h"
#include "pbat_internal.h"

namespace pbat {

// ---------------------------------------------------------------------------
// elimination program builder
// ---------------------------------------------------------------------------
class Elim {
 public:
  Elim(int n, bool directed, int s, int t) : n_(n), dir_(directed), s_(s), t_(t), E_(n * n) {}

  bool has(int i, int j) const { return !at(i, j).empty(); }
  const std::string& at(int i, int j) const {
    if (!dir_ && i > j) std::swap(i, j);
    return E_[i * n_ + j];
  }
  // E[i][j] |= expr
  void or_in(int i, int j, const std::string& expr) {
    if (i == j) return;
    if (dir_ && (j == s_ || i == t_)) return;  // no s-t path enters s or leaves t
    std::string& e = ref(i, j);
    const std::string v = "v" + std::to_string(nvar_++);
    if (e.empty())
      code_ += "  const u32 " + v + " = " + expr + ";\n";
    else
      code_ += "  const u32 " + v + " = " + e + " | " + expr + ";\n";
    e = v;
  }
  void set(int i, int j, const std::string& v) { ref(i, j) = v; }
  int degree(int k) const {
    int d = 0;
    for (int i = 0; i < n_; ++i)
      if (i != k && (has(i, k) || (dir_ && has(k, i)))) ++d;
    return d;
  }
  // cost of eliminating k now (number of shortcut operations)
  int cost(int k) const {
    int in = 0, out = 0;
    for (int i = 0; i < n_; ++i) {
      if (i == k) continue;
      if (has(i, k)) ++in;
      if (dir_ && has(k, i)) ++out;
    }
    return dir_ ? in * out : in * (in - 1) / 2;
  }
  void eliminate(int k) {
    std::vector<int> in, out;
    for (int i = 0; i < n_; ++i) {
      if (i == k) continue;
      if (has(i, k)) in.push_back(i);
      if (dir_ && has(k, i)) out.push_back(i);
    }
    if (!dir_) out = in;
    for (int i : in)
      for (int j : out) {
        if (i == j || (!dir_ && i > j)) continue;
        or_in(i, j, "(" + at(i, k) + " & " + at(k, j) + ")");
        ++ops_;
      }
    for (int i = 0; i < n_; ++i) {
      if (i == k) continue;
      ref(i, k).clear();
      ref(k, i).clear();
    }
  }
  // min-cost elimination of the given nodes (greedy, recomputed each step)
  void eliminate_all(std::vector<int> nodes) {
    while (!nodes.empty()) {
      size_t best = 0;
      int bc = cost(nodes[0]);
      for (size_t x = 1; x < nodes.size(); ++x) {
        const int c = cost(nodes[x]);
        if (c < bc) bc = c, best = x;
      }
      eliminate(nodes[best]);
      nodes.erase(nodes.begin() + best);
    }
  }
  std::vector<std::pair<int, int>> edges() const {
    std::vector<std::pair<int, int>> r;
    for (int i = 0; i < n_; ++i)
      for (int j = 0; j < n_; ++j) {
        if (!dir_ && j <= i) continue;
        if (i != j && has(i, j)) r.emplace_back(i, j);
      }
    return r;
  }
  std::string& code() { return code_; }
  int ops() const { return ops_; }

 private:
  std::string& ref(int i, int j) {
    if (!dir_ && i > j) std::swap(i, j);
    return E_[i * n_ + j];
  }
  int n_;
  bool dir_;
  int s_, t_;
  std::vector<std::string> E_;
  std::string code_;
  int nvar_ = 0, ops_ = 0;
};

// ---------------------------------------------------------------------------
// plan: which arcs are lane / thread / walk / prefix arcs
// ---------------------------------------------------------------------------

static std::vector<int> bfs_dist(const GraphIn& g, int src) {
  std::vector<std::vector<int>> adj(g.n);
  for (int k = 0; k < g.m; ++k) {
    adj[g.tail[k]].push_back(g.head[k]);
    adj[g.head[k]].push_back(g.tail[k]);
  }
  std::vector<int> d(g.n, 1 << 20);
  std::queue<int> q;
  d[src] = 0;
  q.push(src);
  while (!q.empty()) {
    const int u = q.front();
    q.pop();
    for (int v : adj[u])
      if (d[v] > d[u] + 1) {
        d[v] = d[u] + 1;
        q.push(v);
      }
  }
  return d;
}

// ---------------------------------------------------------------------------
// prune-aware prefix arcs (opt-in, pbat_options.prune == 2)
// ---------------------------------------------------------------------------
// The monotone prune resolves a work item when the sink is cut off with every
// non-prefix arc working, or reached with every non-prefix arc failed.  Which
// arcs form the prefix therefore decides how many items are walked: an s-t
// cut lying wholly in the prefix resolves every item in which its arcs all
// fail.  This picks the prefix arcs first -- the arcs nearest to the source
// or the sink, then a deterministic swap search that maximises the number of
// resolved items over a fixed sample of prefix values -- and leaves the walk
// cluster to the remaining arcs.  Work items are counted uniformly (each is
// 2^(m-d) states of work whatever its probability).
class PruneScorer {
 public:
  // kWords words of 64 prefix values each are scored at once, bit-sliced:
  // every arc's state across 64 values is one word
  static constexpr int kWords = 16;
  explicit PruneScorer(const GraphIn& g) : g_(g) {
    uint64_t x = 0x2209097110ull;   // fixed: plans must be reproducible
    uint64_t v[64];
    for (int w = 0; w < kWords; ++w) {
      for (int i = 0; i < 64; ++i) {
        x += 0x9e3779b97f4a7c15ull;  // splitmix64
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        v[i] = z ^ (z >> 31);
      }
      for (int j = 0; j < 64; ++j) {   // sample word: bit i = bit j of value i
        uint64_t t = 0;
        for (int i = 0; i < 64; ++i) t |= ((v[i] >> j) & 1ull) << i;
        sample_[w][j] = t;
      }
    }
  }
  // items resolved by the prune -- cut with every other arc working, or
  // connected with every other arc failed -- over every value of a prefix
  // of at most 10 arcs, else over the fixed sample of kWords * 64 values
  int score(const std::vector<int>& pre) const {
    const int d = (int)pre.size();
    const bool exact = d <= 10;
    const int nw = exact ? std::max(1, (1 << d) / 64) : kWords;
    const uint64_t valid = exact && d < 6 ? ((1ull << (1 << d)) - 1) : ~0ull;
    uint64_t up[64], dn[64];
    int res = 0;
    for (int w = 0; w < nw; ++w) {
      for (int k = 0; k < g_.m; ++k) up[k] = ~0ull, dn[k] = 0ull;
      for (int j = 0; j < d; ++j) {
        const uint64_t b = exact ? exact_word(w, j) : sample_[w][j];
        up[pre[j]] = dn[pre[j]] = b;
      }
      const uint64_t reach_up = reach(up), reach_dn = reach(dn);
      res += __builtin_popcountll((~reach_up | reach_dn) & valid);
    }
    return res;
  }

 private:
  // bit i of value 64 w + i, bit j
  static uint64_t exact_word(int w, int j) {
    static const uint64_t pat[6] = {0xAAAAAAAAAAAAAAAAull, 0xCCCCCCCCCCCCCCCCull,
                                    0xF0F0F0F0F0F0F0F0ull, 0xFF00FF00FF00FF00ull,
                                    0xFFFF0000FFFF0000ull, 0xFFFFFFFF00000000ull};
    return j < 6 ? pat[j] : (((w >> (j - 6)) & 1) ? ~0ull : 0ull);
  }
  // s-t reachability of 64 states at once (arc words `on`): a fixed point
  uint64_t reach(const uint64_t* on) const {
    uint64_t R[64] = {};
    R[g_.source] = ~0ull;
    for (bool grew = true; grew;) {
      grew = false;
      for (int k = 0; k < g_.m; ++k) {
        const int u = g_.tail[k], v = g_.head[k];
        const uint64_t nv = R[v] | (R[u] & on[k]);
        if (nv != R[v]) R[v] = nv, grew = true;
        if (!g_.directed) {
          const uint64_t nu = R[u] | (R[v] & on[k]);
          if (nu != R[u]) R[u] = nu, grew = true;
        }
      }
    }
    return R[g_.sink];
  }
  const GraphIn& g_;
  uint64_t sample_[kWords][64];
};

static std::vector<int> bfs_dist(const GraphIn& g, int src);

// `fixed` (the range arcs) are always prefix arcs; choose `want` more among
// `cand`.  Returns the chosen arcs (not including `fixed`).
static std::vector<int> bs_prune_prefix_search(const GraphIn& g, const std::vector<int>& fixed,
                                               const std::vector<int>& cand, int want);

// The search is deterministic and depends only on the network, the range
// arcs and the number of arcs wanted: its result is kept (the autotuner
// plans every candidate shape, several with the same prefix length).
static std::mutex g_prefix_mu;
static std::map<std::string, std::vector<int>> g_prefix;

static std::vector<int> bs_prune_prefix(const GraphIn& g, const std::vector<int>& fixed,
                                        const std::vector<int>& cand, int want) {
  std::string key;
  auto put = [&](long long v) { key.append((const char*)&v, sizeof v); };
  put(g.n); put(g.m); put(g.directed); put(g.source); put(g.sink); put(want);
  put((long long)fixed.size());
  for (int a : cand) put(a);
  key.append((const char*)g.tail, sizeof(int32_t) * g.m);
  key.append((const char*)g.head, sizeof(int32_t) * g.m);
  {
    std::lock_guard<std::mutex> lk(g_prefix_mu);
    auto it = g_prefix.find(key);
    if (it != g_prefix.end()) return it->second;
  }
  std::vector<int> r = bs_prune_prefix_search(g, fixed, cand, want);
  std::lock_guard<std::mutex> lk(g_prefix_mu);
  g_prefix[key] = r;
  return r;
}

static std::vector<int> bs_prune_prefix_search(const GraphIn& g, const std::vector<int>& fixed,
                                               const std::vector<int>& cand, int want) {
  const std::vector<int> ds = bfs_dist(g, g.source), dt = bfs_dist(g, g.sink);
  auto near = [&](int a) {
    return std::min(std::min(ds[g.tail[a]], ds[g.head[a]]), std::min(dt[g.tail[a]], dt[g.head[a]]));
  };
  std::vector<int> order = cand;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return near(x) < near(y); });
  std::vector<int> chosen(order.begin(), order.begin() + want);
  std::vector<int> others(order.begin() + want, order.end());
  if (chosen.empty() || others.empty()) return chosen;
  const PruneScorer sc(g);
  auto full = [&](const std::vector<int>& ch) {
    std::vector<int> pre = fixed;
    pre.insert(pre.end(), ch.begin(), ch.end());
    return pre;
  };
  int best = sc.score(full(chosen));
  // first-improvement swaps in a fixed order, at most kMaxEvals evaluations
  constexpr int kMaxEvals = 20000;
  int evals = 0;
  for (bool improved = true; improved && evals < kMaxEvals;) {
    improved = false;
    for (size_t i = 0; i < chosen.size() && !improved && evals < kMaxEvals; ++i)
      for (size_t o = 0; o < others.size() && evals < kMaxEvals; ++o) {
        std::vector<int> trial = chosen;
        trial[i] = others[o];
        const int sc_t = sc.score(full(trial));
        ++evals;
        if (sc_t > best) {
          std::swap(chosen[i], others[o]);
          best = sc_t;
          improved = true;
          break;
        }
      }
  }
  return chosen;
}

// Generate bs_inv / bs_var for a given role assignment; returns bs_var's op count.
static void bs_generate(const GraphIn& g, BsPlan& bp) {
  const int m = g.m, top = bp.ell + bp.tb + bp.L, w0 = bp.ell + bp.tb;
  std::vector<bool> core(g.n, false);
  core[g.source] = core[g.sink] = true;
  for (int k = w0; k < top; ++k) {
    const int a = bp.perm[k];
    core[g.tail[a]] = core[g.head[a]] = true;
  }
  // phase A: every arc but the walk arcs, then every non-core node
  Elim A(g.n, g.directed != 0, g.source, g.sink);
  for (int k = 0; k < m; ++k) {
    if (k >= w0 && k < top) continue;
    const int a = bp.perm[k];
    const std::string w = "a[" + std::to_string(k) + "]";
    A.or_in(g.tail[a], g.head[a], w);
    if (!g.directed) continue;
  }
  std::vector<int> outer;
  for (int v = 0; v < g.n; ++v)
    if (!core[v]) outer.push_back(v);
  A.eliminate_all(outer);
  const auto ce = A.edges();
  std::string inv = "__device__ __forceinline__ void bs_inv(const u32* a, u32* e) {\n" + A.code();
  // phase B: the core edges plus the walk arcs, then the core nodes
  Elim B(g.n, g.directed != 0, g.source, g.sink);
  for (size_t x = 0; x < ce.size(); ++x) {
    inv += "  e[" + std::to_string(x) + "] = " + A.at(ce[x].first, ce[x].second) + ";\n";
    B.set(ce[x].first, ce[x].second, "e[" + std::to_string(x) + "]");
  }
  inv += "}\n";
  for (int k = w0; k < top; ++k) {
    const int a = bp.perm[k];
    B.or_in(g.tail[a], g.head[a], "w[" + std::to_string(k - w0) + "]");
  }
  std::vector<int> inner;
  for (int v = 0; v < g.n; ++v)
    if (core[v] && v != g.source && v != g.sink) inner.push_back(v);
  B.eliminate_all(inner);
  std::string var = "__device__ __forceinline__ u32 bs_var(const u32* e, const u32* w) {\n" + B.code();
  var += "  return " + (B.has(g.source, g.sink) ? B.at(g.source, g.sink) : std::string("0u")) + ";\n}\n";
  bp.gen = inv + var;
  bp.ncore = (int)ce.size();
  bp.ops_inv = A.ops();
  bp.ops_var = B.ops() + bp.L;
}

// The fused kernel divides walk masses by p and 1 - p (p-dependent roles).
bool bs_walk_ok(const double* p, int a) {
  return !p || (p[a] >= 0x1p-20 && p[a] <= 1.0 - 0x1p-20);
}

// Prune-aware mode: with the prefix arcs fixed, the walk cluster may sit
// anywhere among the other arcs.  Grow one from every eligible seed arc (the
// arc first, then the arcs adding the fewest new core nodes), generate each
// program and keep the one with the fewest operations per word (then per
// item).  Lane and thread arcs take what is left, in input order.
static void bs_smaller_walk(const GraphIn& g, BsPlan& bp, const double* p_for_grad) {
  const int m = g.m, w0 = bp.ell + bp.tb, top = w0 + bp.L;
  std::vector<int> pool(bp.perm.begin(), bp.perm.begin() + top);   // lane, thread, walk arcs
  std::sort(pool.begin(), pool.end());
  BsPlan best = bp;
  for (int seed : pool) {
    if (!bs_walk_ok(p_for_grad, seed)) continue;
    std::vector<bool> incore(g.n, false), used(m, false);
    incore[g.source] = incore[g.sink] = true;
    std::vector<int> walk{seed};
    used[seed] = true;
    incore[g.tail[seed]] = incore[g.head[seed]] = true;
    while ((int)walk.size() < bp.L) {
      int pick = -1, bscore = 1 << 30;
      for (int a : pool) {
        if (used[a] || !bs_walk_ok(p_for_grad, a)) continue;
        const int add = (!incore[g.tail[a]]) + (!incore[g.head[a]]);
        if (add < bscore) bscore = add, pick = a;
      }
      if (pick < 0) break;
      used[pick] = true;
      walk.push_back(pick);
      incore[g.tail[pick]] = incore[g.head[pick]] = true;
    }
    if ((int)walk.size() < bp.L) continue;
    BsPlan t = bp;
    int x = 0;
    for (int a : pool)
      if (!used[a]) t.perm[x++] = a;
    for (int b = 0; b < bp.L; ++b) t.perm[w0 + b] = walk[b];
    bs_generate(g, t);
    if (t.ops_var < best.ops_var || (t.ops_var == best.ops_var && t.ops_inv < best.ops_inv))
      best = std::move(t);
  }
  bp = std::move(best);
}

int bs_make_plan(const GraphIn& g, const pbat_options& o, int nthr, BsPlan& bp,
                 const double* p_for_grad) {
  if (fault_at("plan")) return fail(PBAT_EINVAL, "injected fault: planning");
  const int m = g.m, r = o.range_bits;
  bp.r = r;
  bp.grad = p_for_grad != nullptr;
  bp.minb = std::max(0, o.occupancy);
  bp.ell = std::min(kMaxLaneBits, m - r);
  bp.tb = std::min(5, m - r - bp.ell);
  const int free_bits = m - r - bp.ell - bp.tb;
  const int lmax = 10;
  if (o.walk_bits >= 0) {
    bp.L = std::min(std::min(o.walk_bits, lmax), free_bits);
  } else if (o.prefix_bits >= 0) {
    bp.L = std::max(0, std::min(lmax, m - bp.ell - bp.tb - std::max(o.prefix_bits, r)));
  } else {
    // about 2^11 work items: measured best on GB300 for 27..40 arcs (larger
    // items amortise the per-item epilogue, which is heavier in the fused
    // kernel, so that one walks two arcs more)
    bp.L = std::max(0, std::min(lmax, free_bits - std::max(0, 11 - r) + (p_for_grad ? 2 : 0)));
  }
  bp.L = std::max(0, std::min(bp.L, free_bits));  // never into the range arcs
  bp.d = m - bp.ell - bp.tb - bp.L;
  (void)nthr;
  // ---- roles.  range arcs are the top prefix bits in input order.
  std::vector<int> cand;
  for (int a = r; a < m; ++a) cand.push_back(a);
  // prune-aware mode: the prefix arcs first, the walk cluster from the rest
  std::vector<bool> incore(g.n, false), used(m, false);
  std::vector<int> pre_first;
  if (o.prune == 2 && bp.d - r > 0) {
    std::vector<int> fixed;
    for (int i = 0; i < r; ++i) fixed.push_back(i);
    pre_first = bs_prune_prefix(g, fixed, cand, bp.d - r);
    for (int a : pre_first) used[a] = true;
  }
  // walk arcs: a compact cluster grown from {source, sink}, so the per-word
  // core stays small
  incore[g.source] = incore[g.sink] = true;
  std::vector<int> walk;
  for (int it = 0; it < bp.L; ++it) {
    int best = -1, bscore = 1 << 30;
    for (int a : cand) {
      if (used[a] || !bs_walk_ok(p_for_grad, a)) continue;
      const int add = (!incore[g.tail[a]]) + (!incore[g.head[a]]);
      if (add < bscore) bscore = add, best = a;
    }
    if (best < 0) {  // not enough eligible walk arcs: shorter walk, deeper prefix
      bp.L = it;
      bp.d = m - bp.ell - bp.tb - bp.L;
      break;
    }
    used[best] = true;
    walk.push_back(best);
    incore[g.tail[best]] = incore[g.head[best]] = true;
  }
  // prefix arcs: the arcs nearest to the source or the sink (they decide the
  // prune), among the rest
  const std::vector<int> ds = bfs_dist(g, g.source), dt = bfs_dist(g, g.sink);
  std::vector<int> rest;   // neither walk arcs nor prefix arcs chosen above
  for (int a : cand)
    if (!used[a]) rest.push_back(a);
  std::stable_sort(rest.begin(), rest.end(), [&](int x, int y) {
    const int dx = std::min(std::min(ds[g.tail[x]], ds[g.head[x]]), std::min(dt[g.tail[x]], dt[g.head[x]]));
    const int dy = std::min(std::min(ds[g.tail[y]], ds[g.head[y]]), std::min(dt[g.tail[y]], dt[g.head[y]]));
    return dx < dy;
  });
  const int npre_free = bp.d - r;
  // a walk shortened for want of eligible arcs deepens the prefix: the
  // extra prefix arcs are the nearest of the rest
  const int extra = npre_free - (int)pre_first.size();
  if (npre_free < 0 || extra < 0 || extra + bp.ell + bp.tb != (int)rest.size())
    return fail(PBAT_EINVAL, "internal: bit-sliced plan does not fit (m=%d r=%d L=%d)", m, r, bp.L);
  bp.perm.assign(m, -1);
  // prefix positions [top, m - r): chosen or nearest arcs; range arcs at [m - r, m)
  const int top = bp.ell + bp.tb + bp.L;
  for (int j = 0; j < (int)pre_first.size(); ++j) bp.perm[top + j] = pre_first[j];
  for (int j = 0; j < extra; ++j) bp.perm[top + (int)pre_first.size() + j] = rest[j];
  for (int i = 0; i < r; ++i) bp.perm[m - 1 - i] = i;
  for (int b = 0; b < bp.L; ++b) bp.perm[bp.ell + bp.tb + b] = walk[b];
  int x = extra;
  for (int k = 0; k < bp.ell + bp.tb; ++k) bp.perm[k] = rest[x++];
  // invariants the kernel relies on: a permutation, range arcs on top, and
  // every role within its limits
  std::vector<int> seen(m, 0);
  bool ok = bp.L >= 0 && bp.L <= 10 && bp.ell <= 5 && bp.tb <= 5 && bp.d >= r &&
            bp.ell + bp.tb + bp.L + bp.d == m && npre_free >= 0 && x == (int)rest.size();
  for (int k = 0; ok && k < m; ++k) {
    ok = bp.perm[k] >= 0 && bp.perm[k] < m && !seen[bp.perm[k]];
    if (ok) seen[bp.perm[k]] = 1;
  }
  for (int i = 0; ok && i < r; ++i) ok = bp.perm[m - 1 - i] == i;
  if (!ok)
    return fail(PBAT_EINVAL, "internal: inconsistent bit-sliced plan (m=%d r=%d L=%d d=%d)", m, r,
                bp.L, bp.d);
  bs_generate(g, bp);
  if (o.prune == 2 && bp.L > 0 && extra == 0) bs_smaller_walk(g, bp, p_for_grad);
  bp.pex = 0;
  if (p_for_grad)
    for (int k = bp.ell + bp.tb + bp.L; k < m; ++k)
      if (!bs_walk_ok(p_for_grad, bp.perm[k])) bp.pex |= 1ull << k;
  return PBAT_OK;
}

}  // namespace pbat
