"""Pins for the CPU oracle: every check here comes from something other
than the oracle itself -- values printed in the paper, closed forms,
invariants of the reliability polynomial, and brute force with an
independent (union-find / DFS, exact rational) implementation."""
import math
import os
from fractions import Fraction
from itertools import product

import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------
# Independent brute force: exact rationals, union-find (undirected) or
# iterative DFS (directed).  Bit convention of Sec. 4.2: arc k <-> bit m-1-k.
# ---------------------------------------------------------------------------

def _reach_uf(net, x):
    parent = list(range(net.n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    m = net.m
    for k in range(m):
        if (x >> (m - 1 - k)) & 1:
            a, b = find(net.tail[k]), find(net.head[k])
            if a != b:
                parent[a] = b
    return find(net.source) == find(net.sink)


def _reach_dfs(net, x):
    m = net.m
    adj = [[] for _ in range(net.n)]
    for k in range(m):
        if (x >> (m - 1 - k)) & 1:
            adj[net.tail[k]].append(net.head[k])
            if not net.directed:
                adj[net.head[k]].append(net.tail[k])
    seen = {net.source}
    stack = [net.source]
    while stack:
        u = stack.pop()
        for v in adj[u]:
            if v not in seen:
                seen.add(v)
                stack.append(v)
    return net.sink in seen


def _exact(net, p=None):
    """Exact rational R, N_k and dR/dp (as R(p_i=1) - R(p_i=0))."""
    m = net.m
    p = [Fraction(v) for v in (net.p if p is None else p)]
    reach = _reach_dfs if net.directed else _reach_uf
    conn = [reach(net, x) for x in range(1 << m)]
    R = Fraction(0)
    Nk = [0] * (m + 1)
    grad = [Fraction(0)] * m
    for x in range(1 << m):
        if not conn[x]:
            continue
        w = Fraction(1)
        bits = [(x >> (m - 1 - k)) & 1 for k in range(m)]
        for k in range(m):
            w *= p[k] if bits[k] else 1 - p[k]
        R += w
        Nk[sum(bits)] += 1
        for i in range(m):
            wi = Fraction(1)
            for k in range(m):
                if k != i:
                    wi *= p[k] if bits[k] else 1 - p[k]
            grad[i] += wi if bits[i] else -wi
    return R, Nk, grad


def _close(a, b, rel=1e-15, abs_=1e-300):
    return abs(a - b) <= max(rel * abs(b), abs_)


# ---------------------------------------------------------------------------
# The paper's worked example and printed values
# ---------------------------------------------------------------------------

def test_figure1_reliability_matches_worked_example():
    """Sec. 5.2 STEP 3 prints R(G) = 0.960175722 for Figure 1 / Table 1."""
    want = float([r for r in _golden("figure1_table4.txt") if r[0] == "R"][0][1])
    for directed in (True, False):
        r = oracle.enumerate_states(synth.figure1(directed))
        assert abs(r.R - want) < 5e-10, (directed, r.R)


def test_figure1_connected_state_probabilities_match_table4():
    """Table 4 prints Pr(X) for the 25 connected states (5 significant digits)."""
    want = sorted(float(r[1]) for r in _golden("figure1_table4.txt") if r[0] == "PR")
    net = synth.figure1(True)
    got = []
    for x in range(1 << net.m):
        if oracle.connected(net, x):
            got.append(oracle.state_probability(net.p, x))
    assert len(got) == 25
    got = sorted(float(f"{v:.4E}") for v in got)
    assert got == want


def test_figure1_counts_from_minimal_paths():
    """Figure 1's minimal path sets {a2,a5}, {a2,a4,a6}, {a1,a3,a5},
    {a1,a3,a4,a6}: a state is connected iff it contains one of them."""
    net = synth.figure1(True)
    mps = [{1, 4}, {1, 3, 5}, {0, 2, 4}, {0, 2, 3, 5}]
    Nk = [0] * 7
    for x in range(64):
        on = {k for k in range(6) if (x >> (5 - k)) & 1}
        conn = any(s <= on for s in mps)
        assert conn == oracle.connected(net, x)
        if conn:
            Nk[len(on)] += 1
    assert oracle.enumerate_states(net).Nk == Nk == [0, 0, 1, 6, 11, 6, 1]


def test_table2_order_and_equal_division_starts():
    """Table 2 / Sec. 4.2: Dec(X_17) = 17 for X_17 = (0,1,0,0,0,0) and
    X_31 = (0,1,1,1,1,0); Sec. 4.3: with chi = 4 the divisions start at
    X_1, X_17, X_33, X_49 and have mu = 16 states."""
    p = [0.99, 0.89, 0.88, 0.95, 0.85, 0.87]

    def pr(vec):
        w = 1.0
        for k, b in enumerate(vec):
            w *= p[k] if b else 1 - p[k]
        return w

    for idx1, vec in ((17, (0, 1, 0, 0, 0, 0)), (31, (0, 1, 1, 1, 1, 0)), (1, (0,) * 6),
                      (64, (1,) * 6)):
        assert _close(oracle.state_probability(p, idx1 - 1), pr(vec), 1e-15)
    # divisions: enumerating prefix [i, i+1) with 2 prefix bits covers states
    # (i*16, (i+1)*16]; the union is the whole space
    net = synth.figure1(True)
    parts = [oracle.enumerate_states(net, prefix_bits=2, prefix_lo=i, prefix_hi=i + 1)
             for i in range(4)]
    assert sum(sum(r.Nk) for r in parts) == sum(oracle.enumerate_states(net).Nk)
    assert _close(sum(r.R for r in parts), oracle.enumerate_states(net).R, 1e-15)
    # division i holds exactly the states with the i-th 2-bit prefix
    for i in range(4):
        n_conn = sum(1 for x in range(16 * i, 16 * (i + 1)) if _reach_dfs(net, x))
        assert sum(parts[i].Nk) == n_conn


def test_table3_plsa_layers():
    """Table 3: PLSA on Figure 1 with all arcs working: L_1 = {1},
    L_2 = {2, 3}, L_3 = {4, 5} (paper's 1-based node ids)."""
    net = synth.figure1(True)
    layers = oracle.plsa_layers(net, (1 << 6) - 1)
    assert layers == [1, 2, 2, 3, 3]


def test_table6_bridge():
    """Table 6, network (1): R = 0.97848 at p = 0.9; it equals the bridge
    polynomial 2p^2 + 2p^3 - 5p^4 + 2p^5 with N = [0, 0, 2, 8, 5, 1]."""
    g = dict((r[0], r[1]) for r in _golden("table6_bridge.txt"))
    p = float(g["p"])
    r = oracle.enumerate_states(synth.bridge([p] * 5))
    assert abs(r.R - float(g["R"])) < 5e-11
    assert r.Nk == [0, 0, 2, 8, 5, 1]
    for q in (0.1, 0.37, 0.5, 0.9, 0.999):
        r = oracle.enumerate_states(synth.bridge([q] * 5))
        poly = 2 * q**2 + 2 * q**3 - 5 * q**4 + 2 * q**5
        assert _close(r.R, poly, 1e-14)


def test_directed_bridge_by_conditioning():
    """Directed bridge 0->1, 0->2, 1->2, 1->3, 2->3: conditioning on the
    middle arc 1->2 gives R = p3*[1-(1-p1)(1-p2)... closed form below."""
    p = [0.91, 0.73, 0.55, 0.66, 0.88]
    p1, p2, p3, p4, p5 = p
    # middle arc 1->2 works: 0 reaches {1,2} region; 1->3 or 2->3
    # reach1 = p1; reach2 = 1-(1-p2)(1-p1 p3) ... enumerate exactly by cases
    R_mid_on = 0.0
    R_mid_off = 0.0
    for a, b in product((0, 1), repeat=2):  # arcs 0->1 (p1), 0->2 (p2)
        w = (p1 if a else 1 - p1) * (p2 if b else 1 - p2)
        # mid on: node 2 reached if b or a; node 1 reached if a
        r1, r2 = a, (b or a)
        R_mid_on += w * (1 - (1 - p4 * r1) * (1 - p5 * r2))
        r1, r2 = a, b
        R_mid_off += w * (1 - (1 - p4 * r1) * (1 - p5 * r2))
    want = p3 * R_mid_on + (1 - p3) * R_mid_off
    got = oracle.enumerate_states(synth.bridge(p, directed=True)).R
    assert _close(got, want, 1e-14)
    got_g = oracle.grad_critical(synth.bridge(p, directed=True))
    assert _close(got_g[2], R_mid_on - R_mid_off, 1e-13)


# ---------------------------------------------------------------------------
# Closed forms: series, parallel, random series-parallel networks
# ---------------------------------------------------------------------------

def test_series_parallel_closed_forms():
    rng = synth.SplitMix64(7)
    for m in (1, 2, 5, 9):
        p = [0.05 + 0.9 * rng.uniform01() for _ in range(m)]
        s = oracle.enumerate_states(synth.series(m, p), grad=True)
        assert _close(s.R, math.prod(p), 1e-14)
        assert s.Nk == [0] * m + [1]
        gs = oracle.grad_critical(synth.series(m, p))
        for i in range(m):
            want = math.prod(p[:i] + p[i + 1:])
            assert _close(gs[i], want, 1e-14) and _close(s.grad_t1t0[i], want, 1e-13)
        q = oracle.enumerate_states(synth.parallel(m, p), grad=True)
        assert _close(q.R, 1 - math.prod(1 - v for v in p), 1e-14)
        assert q.Nk == [0] + [math.comb(m, k) for k in range(1, m + 1)]
        gq = oracle.grad_critical(synth.parallel(m, p))
        for i in range(m):
            want = math.prod(1 - v for j, v in enumerate(p) if j != i)
            assert _close(gq[i], want, 1e-13)


def _random_sp(rng, depth, directed):
    """Random series-parallel network with exact R and gradient computed by
    the composition rules (series: product; parallel: 1 - prod(1 - R))."""
    # represent as (n, tail, head, p, src, dst, R, dR list)
    if depth == 0 or rng.below(3) == 0:
        pv = 0.05 + 0.9 * rng.uniform01()
        return dict(n=2, tail=[0], head=[1], p=[pv], s=0, t=1, R=pv, dR=[1.0])
    a = _random_sp(rng, depth - 1, directed)
    b = _random_sp(rng, depth - 1, directed)
    off = a["n"]
    if rng.below(2) == 0:  # series: a.t == b.s
        remap = {v: v + off for v in range(b["n"])}
        remap[b["s"]] = a["t"]
        tail = a["tail"] + [remap[v] for v in b["tail"]]
        head = a["head"] + [remap[v] for v in b["head"]]
        n = off + b["n"]
        R = a["R"] * b["R"]
        dR = [d * b["R"] for d in a["dR"]] + [d * a["R"] for d in b["dR"]]
        s, t = a["s"], remap[b["t"]]
    else:  # parallel: share both terminals
        remap = {v: v + off for v in range(b["n"])}
        remap[b["s"]] = a["s"]
        remap[b["t"]] = a["t"]
        tail = a["tail"] + [remap[v] for v in b["tail"]]
        head = a["head"] + [remap[v] for v in b["head"]]
        n = off + b["n"]
        R = 1 - (1 - a["R"]) * (1 - b["R"])
        dR = [d * (1 - b["R"]) for d in a["dR"]] + [d * (1 - a["R"]) for d in b["dR"]]
        s, t = a["s"], a["t"]
    # compact node ids
    used = sorted(set(tail) | set(head) | {s, t})
    ren = {v: i for i, v in enumerate(used)}
    return dict(n=len(used), tail=[ren[v] for v in tail], head=[ren[v] for v in head],
                p=a["p"] + b["p"], s=ren[s], t=ren[t], R=R, dR=dR)


@pytest.mark.parametrize("directed", [False, True])
def test_random_series_parallel(directed):
    rng = synth.SplitMix64(1234 + directed)
    done = 0
    while done < 25:
        sp = _random_sp(rng, 4, directed)
        if not (2 <= len(sp["tail"]) <= 14):
            continue
        net = synth.Network(sp["n"], sp["tail"], sp["head"], sp["p"], sp["s"], sp["t"], directed)
        r = oracle.enumerate_states(net, grad=True)
        assert _close(r.R, sp["R"], 1e-13)
        g = oracle.grad_critical(net)
        for i in range(net.m):
            assert abs(g[i] - sp["dR"][i]) <= 1e-13 * max(1.0, abs(sp["dR"][i]))
            assert abs(r.grad_t1t0[i] - sp["dR"][i]) <= 1e-13
        done += 1


# ---------------------------------------------------------------------------
# Brute force with independent connectivity and exact rationals
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("directed", [False, True])
def test_exact_rational_brute_force(directed):
    for seed in range(60):
        net = synth.random_small(seed * 7919 + directed, directed=directed)
        if net.m > 10:
            net = synth.Network(net.n, net.tail[:10], net.head[:10], net.p[:10], net.source,
                                net.sink, directed)
        R, Nk, grad = _exact(net)
        r = oracle.enumerate_states(net, grad=True)
        assert r.Nk == Nk, seed
        assert abs(Fraction(r.R_hilo[0]) + Fraction(r.R_hilo[1]) - R) <= Fraction(1, 10**17)
        g = oracle.grad_critical(net)
        for i in range(net.m):
            assert abs(Fraction(g[i]) - grad[i]) <= Fraction(1, 10**15), (seed, i)
            assert abs(Fraction(r.grad_t1t0[i]) - grad[i]) <= Fraction(1, 10**15), (seed, i)


def test_connectivity_against_union_find_many_graphs():
    """Thousands of tiny undirected graphs: PLSA == union-find, state by state."""
    checked = 0
    for seed in range(400):
        net = synth.random_small(10_000 + seed, directed=False)
        m = min(net.m, 7)
        net = synth.Network(net.n, net.tail[:m], net.head[:m], net.p[:m], net.source, net.sink)
        for x in range(1 << m):
            assert oracle.connected(net, x) == _reach_uf(net, x)
            checked += 1
    assert checked > 10_000


# ---------------------------------------------------------------------------
# Invariants of N_k and of R
# ---------------------------------------------------------------------------

def _shortest_paths(net):
    """BFS distance d(s,t) and number of shortest s-t paths (counted by BFS)."""
    adj = [[] for _ in range(net.n)]
    for u, v in zip(net.tail, net.head):
        adj[u].append(v)
        if not net.directed:
            adj[v].append(u)
    dist = [-1] * net.n
    cnt = [0] * net.n
    dist[net.source], cnt[net.source] = 0, 1
    q = [net.source]
    for u in q:
        for v in adj[u]:
            if dist[v] < 0:
                dist[v] = dist[u] + 1
                q.append(v)
            if dist[v] == dist[u] + 1:
                cnt[v] += cnt[u]
    return dist[net.sink], cnt[net.sink]


@pytest.mark.parametrize("rows,cols", [(2, 4), (3, 4), (3, 5)])
def test_grid_polynomial_invariants(rows, cols):
    tail, head = synth.grid(rows, cols)
    n = rows * cols
    m = len(tail)
    net = synth.Network(n, tail, head, [0.5] * m, 0, n - 1)
    r = oracle.enumerate_states(net)
    d, npaths = _shortest_paths(net)
    assert all(v == 0 for v in r.Nk[:d])
    assert r.Nk[d] == npaths == math.comb(rows + cols - 2, rows - 1)
    assert r.Nk[m] == 1
    # N_{m-c} = C(m, c) - (number of c-arc sets whose removal cuts s from t),
    # the cut sets counted here with union-find on the full graph
    full = (1 << m) - 1
    cuts1 = sum(1 for i in range(m) if not _reach_uf(net, full & ~(1 << (m - 1 - i))))
    cuts2 = sum(1 for i in range(m) for j in range(i + 1, m)
                if not _reach_uf(net, full & ~(1 << (m - 1 - i)) & ~(1 << (m - 1 - j))))
    assert cuts1 == 0
    assert r.Nk[m - 1] == m - cuts1
    assert r.Nk[m - 2] == math.comb(m, 2) - cuts2
    if rows >= 3:
        assert cuts2 == 2  # only the two arc pairs at the corners
    assert all(r.Nk[k] <= math.comb(m, k) for k in range(m + 1))
    # p = 1/2: R * 2^m equals the number of connected states exactly
    assert r.R * 2.0**m == sum(r.Nk)
    # uniform p: R(p) = sum_k N_k p^k (1-p)^(m-k), and sum_i dR/dp_i = dR/dp
    p = 0.83
    r2 = oracle.enumerate_states(net, p=[p] * m, grad=True)
    poly = sum(c * p**k * (1 - p) ** (m - k) for k, c in enumerate(r.Nk))
    dpoly = sum(c * (k * p ** (k - 1) * (1 - p) ** (m - k) - (m - k) * p**k * (1 - p) ** (m - k - 1))
                for k, c in enumerate(r.Nk))
    assert _close(r2.R, poly, 1e-13)
    assert abs(sum(r2.grad_t1t0) - dpoly) < 1e-12


def test_affine_identity_and_finite_difference():
    """R is affine in each p_i: R = p_i R(1_i) + (1 - p_i) R(0_i), and the
    central difference is exact up to rounding."""
    net = synth.workload_small_random()
    net = synth.Network(net.n, net.tail[:12], net.head[:12], net.p[:12], net.source, net.sink)
    base = oracle.enumerate_states(net, grad=True)
    gcrit = oracle.grad_critical(net)
    for i in range(net.m):
        p1 = list(net.p); p1[i] = 1.0
        p0 = list(net.p); p0[i] = 0.0
        R1 = oracle.enumerate_states(net, p=p1).R
        R0 = oracle.enumerate_states(net, p=p0).R
        assert _close(base.R, net.p[i] * R1 + (1 - net.p[i]) * R0, 1e-14)
        assert abs(gcrit[i] - (R1 - R0)) < 1e-14
        assert abs(base.grad_t1t0[i] - (R1 - R0)) < 1e-14
        h = 1e-4
        pp = list(net.p); pp[i] += h
        pm = list(net.p); pm[i] -= h
        fd = (oracle.enumerate_states(net, p=pp).R - oracle.enumerate_states(net, p=pm).R) / (2 * h)
        assert abs(fd - gcrit[i]) < 1e-10


def test_planted_mistakes_are_caught():
    """Mutations of the oracle's arithmetic, planted on the CPU in a copy of
    the formula, must break at least one pin above: a swapped p / 1-p, a
    dropped factor and a reversed bit order all change Figure 1's R or the
    bridge polynomial."""
    net = synth.figure1(True)
    want = 0.960175722
    p = net.p
    conn = [x for x in range(64) if oracle.connected(net, x)]

    def R_with(weight):
        return sum(weight(x) for x in conn)

    def w_ok(x):
        return math.prod(p[k] if (x >> (5 - k)) & 1 else 1 - p[k] for k in range(6))

    def w_swapped(x):
        return math.prod(1 - p[k] if (x >> (5 - k)) & 1 else p[k] for k in range(6))

    def w_dropped(x):
        return math.prod(p[k] if (x >> (5 - k)) & 1 else 1 - p[k] for k in range(5))

    def w_reversed(x):
        return math.prod(p[k] if (x >> k) & 1 else 1 - p[k] for k in range(6))

    assert abs(R_with(w_ok) - want) < 5e-10
    for bad in (w_swapped, w_dropped):
        assert abs(R_with(bad) - want) > 1e-4
    # Figure 1 is symmetric under a1..a6 -> a6..a1, so a reversed bit order
    # keeps R; the Table 2 pin (X_17 = (0,1,0,0,0,0), index 16 from 0)
    # catches it instead.
    x17 = 16
    only_a2 = (1 - p[0]) * p[1] * (1 - p[2]) * (1 - p[3]) * (1 - p[4]) * (1 - p[5])
    assert abs(w_ok(x17) - only_a2) < 1e-18
    assert abs(w_reversed(x17) - only_a2) > 0.1 * only_a2


# ---------------------------------------------------------------------------
# The 3x6 grid workload at full size (2^27 states)
# ---------------------------------------------------------------------------

# Values of the 3x6 grid, corner to corner, every p = 0.9, from a separate
# brute force written before this project's oracle (plain C, its own
# connectivity search): R to 12 decimals and the whole coefficient list.
GRID_3X6_R = 0.969984456182
GRID_3X6_NK = [0] * 7 + [21, 420, 4035, 24635, 106652, 346092, 867889, 1709032, 2659298, 3267444,
                         3155927, 2388481, 1421756, 669306, 249627, 73359, 16721, 2866, 349, 27, 1]


def _grid_division(d):
    import oracle as orc
    net = synth.workload_grid_3x6()
    r = orc.enumerate_states(net, prefix_bits=8, prefix_lo=d, prefix_hi=d + 1, grad=True)
    return r.R_hilo, r.Nk, r.T1_hilo, r.T0_hilo


def test_grid_3x6_full_space_reproduces_independent_values_and_golden_file():
    """The oracle over all 2^27 states of the grid (equal divisions on a
    process pool) gives the independent values above, and the stored
    expected values that the GPU parity tests compare with are exactly what
    the oracle computes now."""
    import multiprocessing as mp
    net = synth.workload_grid_3x6()
    m = net.m
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        parts = pool.map(_grid_division, range(256), chunksize=2)

    def exact(pairs):
        return sum((Fraction(h) + Fraction(lo) for h, lo in pairs), Fraction(0))

    R = exact([q[0] for q in parts])
    Nk = [sum(q[1][k] for q in parts) for k in range(m + 1)]
    assert Nk == GRID_3X6_NK
    assert abs(float(R) - GRID_3X6_R) <= 5e-13
    # the polynomial in p = 0.9 from the counts
    assert abs(float(R) - sum(c * 0.9**k * 0.1 ** (m - k) for k, c in enumerate(Nk))) <= 1e-14
    rows = _golden("grid-3x6_full.txt")
    gold = {}
    for r in rows:
        gold.setdefault(r[0], []).append(r[1:])
    gR = Fraction(float.fromhex(gold["R"][0][0])) + Fraction(float.fromhex(gold["R"][0][1]))
    # the oracle's long double sums of different division sizes round apart
    # by about 2^-64 of the mass
    assert abs(gR - R) <= Fraction(1, 2**60) and [int(v) for v in gold["NK"][0]] == Nk
    for key, idx in (("T1", 2), ("T0", 3)):
        for i, hi, lo in gold[key]:
            want = Fraction(float.fromhex(hi)) + Fraction(float.fromhex(lo))
            assert abs(want - exact([q[idx][int(i)] for q in parts])) <= Fraction(1, 2**59)
    # every arc's T1 + T0 is the mass of the other arcs' connected half
    # states: at most 2, and T1 - T0 = dR/dp >= 0 (R is monotone)
    for i in range(m):
        t1 = exact([q[2][i] for q in parts])
        t0 = exact([q[3][i] for q in parts])
        assert 0 <= t1 - t0 and t1 + t0 <= 2
