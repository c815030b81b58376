"""Seeded synthetic inputs for the PBAT engine and its oracle.

This module holds no reliability arithmetic: it only draws graphs and arc
reliabilities from a counter-based generator (splitmix64), so that the CUDA
path, the CPU oracle, the tests and the benchmark all see bit-identical
inputs.  The paper's 20 benchmark networks (Sec. 5.3, Figure 3) are not
recoverable from the text, so every workload here is synthetic; the recipe
is stated next to each builder.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

MASK64 = (1 << 64) - 1
BASE_SEED = 220909711  # arXiv id 2209.09711 as an integer


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014): state += golden gamma, then mix."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform01(self) -> float:
        """53-bit uniform in [0, 1): (x >> 11) * 2^-53."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def below(self, k: int) -> int:
        """Uniform integer in [0, k) by rejection (no modulo bias)."""
        if k <= 0:
            raise ValueError("k must be positive")
        limit = (1 << 64) - ((1 << 64) % k)
        while True:
            x = self.next_u64()
            if x < limit:
                return x % k


@dataclass
class Network:
    """A binary-state network G(V, E, D_b) with a source and a sink.

    Nodes are 0-based ids in [0, n).  Arc k joins tail[k] and head[k]; when
    ``directed`` is false each arc is usable in both directions.  ``p[k]`` is
    the probability that arc k works.
    """

    n: int
    tail: List[int]
    head: List[int]
    p: List[float]
    source: int
    sink: int
    directed: bool = False
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return len(self.tail)


def uniform_p(rng: SplitMix64, m: int, lo: float, hi: float) -> List[float]:
    return [lo + (hi - lo) * rng.uniform01() for _ in range(m)]


def random_connected_undirected(n: int, m: int, seed: int) -> tuple:
    """Random spanning tree (node i >= 1 attaches to a uniform j < i), then
    uniform non-edges until there are m arcs.  No loops, no parallel arcs."""
    if m < n - 1 or m > n * (n - 1) // 2:
        raise ValueError(f"m={m} impossible for a simple connected graph on n={n}")
    rng = SplitMix64(seed)
    tail, head, seen = [], [], set()
    for i in range(1, n):
        j = rng.below(i)
        tail.append(j)
        head.append(i)
        seen.add((j, i))
    while len(tail) < m:
        u, v = rng.below(n), rng.below(n)
        if u == v:
            continue
        a, b = min(u, v), max(u, v)
        if (a, b) in seen:
            continue
        seen.add((a, b))
        tail.append(a)
        head.append(b)
    return tail, head, rng


def random_directed_reachable(n: int, m: int, seed: int, source: int) -> tuple:
    """Directed arcs: first a random arborescence out of ``source`` (every
    other node gets one incoming arc from a node already placed), so every
    node -- the sink included -- is reachable from the source; then uniform
    distinct ordered pairs (u != v) until there are m arcs."""
    if m < n - 1 or m > n * (n - 1):
        raise ValueError("bad m for directed graph")
    rng = SplitMix64(seed)
    order = [source] + [v for v in range(n) if v != source]
    # shuffle the non-source nodes (Fisher-Yates) so placement is random
    rest = order[1:]
    for i in range(len(rest) - 1, 0, -1):
        j = rng.below(i + 1)
        rest[i], rest[j] = rest[j], rest[i]
    order = [source] + rest
    tail, head, seen = [], [], set()
    for i in range(1, n):
        u = order[rng.below(i)]
        v = order[i]
        tail.append(u)
        head.append(v)
        seen.add((u, v))
    while len(tail) < m:
        u, v = rng.below(n), rng.below(n)
        if u == v or (u, v) in seen:
            continue
        seen.add((u, v))
        tail.append(u)
        head.append(v)
    return tail, head, rng


def grid(rows: int, cols: int) -> tuple:
    """Undirected rows x cols grid, row-major node ids; for each node in id
    order, the arc to its right neighbour, then the arc to the one below."""
    tail, head = [], []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if c + 1 < cols:
                tail.append(v)
                head.append(v + 1)
            if r + 1 < rows:
                tail.append(v)
                head.append(v + cols)
    return tail, head


# ---------------------------------------------------------------------------
# The five workloads.  Seeds are BASE_SEED + workload index (batched graphs
# add 1000 * g).
# ---------------------------------------------------------------------------

def workload_small_random() -> Network:
    """Random connected undirected graph, n=8, m=16, p ~ U[0.80, 0.99];
    source 0, sink 7; 2^16 states."""
    seed = BASE_SEED + 1
    tail, head, rng = random_connected_undirected(8, 16, seed)
    p = uniform_p(rng, 16, 0.80, 0.99)
    return Network(8, tail, head, p, 0, 7, False, "random-undirected-n8-m16")


def workload_grid_3x6() -> Network:
    """Undirected 3x6 grid (18 nodes, 27 arcs), corners 0 and 17, p = 0.9;
    2^27 states."""
    tail, head = grid(3, 6)
    return Network(18, tail, head, [0.9] * len(tail), 0, 17, False, "grid-3x6")


def workload_directed_20_34() -> Network:
    """Random directed graph, n=20, m=34, source 0 reaches sink 19,
    p ~ U[0.70, 0.99]; 2^34 states."""
    seed = BASE_SEED + 3
    tail, head, rng = random_directed_reachable(20, 34, seed, 0)
    p = uniform_p(rng, 34, 0.70, 0.99)
    return Network(20, tail, head, p, 0, 19, True, "random-directed-n20-m34")


def workload_batched(n_graphs: int = 64, n_pvec: int = 16):
    """n_graphs random connected undirected graphs, n ~ U{8..20},
    m ~ U{20..min(32, C(n,2))}, source 0, sink n-1, and n_pvec p-vectors per
    graph with p ~ U[0.6, 0.999].  Returns (networks, pvecs) where pvecs[g]
    is a list of n_pvec lists of length m_g."""
    nets, pvecs = [], []
    for g in range(n_graphs):
        seed = BASE_SEED + 4 + 1000 * g
        rng = SplitMix64(seed)
        n = 8 + rng.below(13)
        mmax = min(32, n * (n - 1) // 2)
        m = 20 + rng.below(mmax - 20 + 1)
        tail, head, rng2 = random_connected_undirected(n, m, seed ^ 0x5DEECE66D)
        pv = [uniform_p(rng2, m, 0.6, 0.999) for _ in range(n_pvec)]
        nets.append(Network(n, tail, head, pv[0], 0, n - 1, False, f"batched-g{g}-n{n}-m{m}"))
        pvecs.append(pv)
    return nets, pvecs


def workload_random_24_40() -> Network:
    """Random connected undirected graph, n=24, m=40, p ~ U[0.90, 0.999];
    source 0, sink 23; 2^40 states."""
    seed = BASE_SEED + 5
    tail, head, rng = random_connected_undirected(24, 40, seed)
    p = uniform_p(rng, 40, 0.90, 0.999)
    return Network(24, tail, head, p, 0, 23, False, "random-undirected-n24-m40")


def random_small(seed: int, n: Optional[int] = None, m: Optional[int] = None,
                 directed: bool = False, p_lo: float = 0.05, p_hi: float = 0.95) -> Network:
    """Small random network for property tests (not necessarily connected,
    parallel arcs allowed): n in [3, 9], m in [1, 14]."""
    rng = SplitMix64(seed)
    if n is None:
        n = 3 + rng.below(7)
    if m is None:
        m = 1 + rng.below(14)
    tail, head = [], []
    for _ in range(m):
        u = rng.below(n)
        v = rng.below(n - 1)
        if v >= u:
            v += 1
        tail.append(u)
        head.append(v)
    s = rng.below(n)
    t = rng.below(n - 1)
    if t >= s:
        t += 1
    p = uniform_p(rng, m, p_lo, p_hi)
    return Network(n, tail, head, p, s, t, directed, f"random-small-{seed}")


def series(m: int, p: List[float]) -> Network:
    """m arcs in series 0 -> 1 -> ... -> m."""
    return Network(m + 1, list(range(m)), list(range(1, m + 1)), list(p), 0, m, False, "series")


def parallel(m: int, p: List[float]) -> Network:
    """m parallel arcs between nodes 0 and 1."""
    return Network(2, [0] * m, [1] * m, list(p), 0, 1, False, "parallel")


def bridge(p: List[float], directed: bool = False) -> Network:
    """The 5-arc bridge: 0-1, 0-2, 1-2, 1-3, 2-3; source 0, sink 3."""
    return Network(4, [0, 0, 1, 1, 2], [1, 2, 2, 3, 3], list(p), 0, 3, directed, "bridge")


def figure1(directed: bool = True) -> Network:
    """Sec. 2.2, Figure 1 and Table 1, rebuilt (the figure itself is not in
    the text): nodes 1..5 become 0..4, source node 1 -> 0, sink node 4 -> 3;
    a1: 1-2, a2: 1-3, a3: 2-3, a4: 3-5, a5: 3-4, a6: 5-4."""
    return Network(5, [0, 0, 1, 2, 2, 4], [1, 2, 2, 4, 3, 3],
                   [0.99, 0.89, 0.88, 0.95, 0.85, 0.87], 0, 3, directed, "figure1")
