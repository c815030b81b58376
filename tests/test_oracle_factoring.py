"""Pins for the oracle's factoring method (oracle/pbat_factoring.c), the
exact values of full-size undirected workloads.

It is a different algorithm from the brute force (pivotal decomposition on
each arc, over frontier partitions), so agreement with the pinned brute
force on many networks, with closed forms and with the stored full-space
values of the 3x6 grid pins it.  Counts must match exactly; R and the
T1/T0 sums agree to the rounding of two long double computations.
"""
import math
import os
from fractions import Fraction

import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_matches_brute_force_on_random_networks():
    for seed in range(1500):
        rng = synth.SplitMix64(60000 + seed)
        net = synth.random_small(70000 + seed, n=2 + rng.below(9), m=1 + rng.below(14),
                                 p_lo=0.01, p_hi=0.99)
        ref = oracle.enumerate_states(net)
        f = oracle.factor(net)
        assert f.Nk == ref.Nk, seed
        assert abs(f.R - ref.R) <= 1e-16 * max(ref.R, 1e-300) + 1e-300, (seed, f.R, ref.R)


def test_t1_t0_match_brute_force():
    for seed in range(200):
        rng = synth.SplitMix64(61000 + seed)
        net = synth.random_small(71000 + seed, n=3 + rng.below(7), m=2 + rng.below(11),
                                 p_lo=0.0, p_hi=1.0)
        ref = oracle.enumerate_states(net, grad=True)
        T1, T0 = oracle.factor_t1t0(net)
        for i in range(net.m):
            assert abs(sum(T1[i]) - ref.T1[i]) <= 1e-16 * max(1.0, ref.T1[i]), (seed, i)
            assert abs(sum(T0[i]) - ref.T0[i]) <= 1e-16 * max(1.0, ref.T0[i]), (seed, i)


def test_wider_networks_against_brute_force():
    # 2^20 - 2^22 states, frontiers of 7 to 10 nodes
    for seed, (n, m) in enumerate([(12, 20), (14, 21), (10, 22)]):
        tail, head, rng = synth.random_connected_undirected(n, m, 62000 + seed)
        net = synth.Network(n, tail, head, synth.uniform_p(rng, m, 0.5, 0.99), 0, n - 1)
        ref = oracle.enumerate_states(net)
        f = oracle.factor(net)
        assert f.Nk == ref.Nk and abs(f.R - ref.R) <= 1e-15 * ref.R


def test_closed_forms():
    p = [0.9, 0.8, 0.95, 0.7, 0.85]
    f = oracle.factor(synth.series(5, p))
    assert abs(f.R - math.prod(p)) <= 1e-16 and f.Nk == [0, 0, 0, 0, 0, 1]
    f = oracle.factor(synth.parallel(5, p))
    assert abs(f.R - (1 - math.prod(1 - x for x in p))) <= 1e-16
    assert f.Nk == [0] + [math.comb(5, k) for k in range(1, 6)]
    for q in (0.1, 0.5, 0.9):
        f = oracle.factor(synth.bridge([q] * 5))
        assert abs(f.R - (2 * q**2 + 2 * q**3 - 5 * q**4 + 2 * q**5)) <= 1e-15
        assert f.Nk == [0, 0, 2, 8, 5, 1]


def test_grid_3x6_full_space_against_stored_brute_force():
    rows = {}
    with open(os.path.join(GOLDEN, "grid-3x6_full.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                w = line.split()
                rows.setdefault(w[0], []).append(w[1:])
    net = synth.workload_grid_3x6()

    def val(hi, lo):
        return Fraction(float.fromhex(hi)) + Fraction(float.fromhex(lo))

    f = oracle.factor(net)
    assert f.Nk == [int(v) for v in rows["NK"][0]]
    assert abs(Fraction(f.R_hilo[0]) + Fraction(f.R_hilo[1]) - val(*rows["R"][0])) <= Fraction(1, 2**60)
    T1, T0 = oracle.factor_t1t0(net)
    for i, hi, lo in rows["T1"]:
        assert abs(Fraction(T1[int(i)][0]) + Fraction(T1[int(i)][1]) - val(hi, lo)) <= Fraction(1, 2**58)
    for i, hi, lo in rows["T0"]:
        assert abs(Fraction(T0[int(i)][0]) + Fraction(T0[int(i)][1]) - val(hi, lo)) <= Fraction(1, 2**58)


def test_forty_arc_workload_invariants():
    """The 24-node, 40-arc workload (2^40 states): what the counts must
    satisfy whatever the network, checked on the factoring result."""
    net = synth.workload_random_24_40()
    m = net.m
    f = oracle.factor(net)
    N = f.Nk
    assert N[m] == 1 and all(0 <= N[k] <= math.comb(m, k) for k in range(m + 1))
    # shortest s-t paths (BFS layer counts) give the first nonzero count
    adj = [[] for _ in range(net.n)]
    for u, v in zip(net.tail, net.head):
        adj[u].append(v)
        adj[v].append(u)
    dist, ways = {net.source: 0}, {net.source: 1}
    frontier = [net.source]
    while frontier:
        nxt = []
        for u in frontier:
            for v in adj[u]:
                if v not in dist:
                    dist[v] = dist[u] + 1
                    ways[v] = 0
                    nxt.append(v)
                if dist[v] == dist[u] + 1:
                    ways[v] += ways[u]
        frontier = nxt
    d = dist[net.sink]
    assert all(N[k] == 0 for k in range(d)) and N[d] == ways[net.sink]
    # N_{m-1}: every single failed arc that is not a bridge of s-t keeps the
    # network connected; count s-t cut arcs by brute force over one arc
    cut1 = sum(1 for i in range(m)
               if not oracle.connected(net, ((1 << m) - 1) & ~(1 << (m - 1 - i))))
    assert N[m - 1] == m - cut1
    # p = 1/2: R is the count of connected states over 2^m
    half = oracle.factor(net, [0.5] * m)
    assert abs(half.R - sum(N) / 2.0**m) <= 1e-18


def test_directed_and_too_wide_are_refused():
    with pytest.raises(ValueError):
        oracle.factor(synth.figure1(True))
    # a 3 x 20 grid walked row by row still has a narrow frontier; a random
    # dense network on 40 nodes does not
    tail, head, rng = synth.random_connected_undirected(40, 63, 63001)
    net = synth.Network(40, tail, head, [0.9] * 63, 0, 39)
    try:
        oracle.factor(net)
    except ValueError as e:
        assert "frontier" in str(e)
