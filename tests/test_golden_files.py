"""The stored full-space values under tests/golden/ (written by
tests/golden/make_golden.py from the brute-force oracle) against what any
correct result must satisfy, checked independently of the oracle's sums:
counts bounded by binomials, the first nonzero count equal to the number of
shortest source-sink paths (BFS path counting), N_{m-1} equal to m minus the
number of single-arc cuts (one connectivity test per arc), N_m = 1, every
dR/dp = T1 - T0 non-negative (R is monotone in each p) and T1 + T0 >= R."""
import math
import os
from collections import deque
from fractions import Fraction

import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FILES = {"grid-3x6": synth.workload_grid_3x6,
         "random-directed-n20-m34": synth.workload_directed_20_34}


def _read(name):
    rows = {}
    with open(os.path.join(GOLDEN, f"{name}_full.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = line.split()
                rows.setdefault(w[0], []).append(w[1:])

    def val(hi, lo):
        return Fraction(float.fromhex(hi)) + Fraction(float.fromhex(lo))

    R = val(*rows["R"][0])
    Nk = [int(v) for v in rows["NK"][0]]
    T1 = {int(i): val(h, l) for i, h, l in rows["T1"]}
    T0 = {int(i): val(h, l) for i, h, l in rows["T0"]}
    return R, Nk, T1, T0


def _shortest_paths(net):
    adj = [[] for _ in range(net.n)]
    for u, v in zip(net.tail, net.head):
        adj[u].append(v)
        if not net.directed:
            adj[v].append(u)
    dist, ways = {net.source: 0}, {net.source: 1}
    q = deque([net.source])
    while q:
        u = q.popleft()
        for v in adj[u]:
            if v not in dist:
                dist[v], ways[v] = dist[u] + 1, 0
                q.append(v)
            if dist[v] == dist[u] + 1:
                ways[v] += ways[u]
    return dist[net.sink], ways[net.sink]


@pytest.mark.parametrize("name", sorted(FILES))
def test_stored_full_space_values_satisfy_invariants(name):
    if not os.path.exists(os.path.join(GOLDEN, f"{name}_full.txt")):
        pytest.skip("not written")
    net = FILES[name]()
    m = net.m
    R, Nk, T1, T0 = _read(name)
    assert len(Nk) == m + 1 and Nk[m] == 1
    assert all(0 <= Nk[k] <= math.comb(m, k) for k in range(m + 1))
    d, ways = _shortest_paths(net)
    assert all(Nk[k] == 0 for k in range(d)) and Nk[d] == ways
    everything = (1 << m) - 1
    cut1 = sum(1 for i in range(m) if not oracle.connected(net, everything & ~(1 << (m - 1 - i))))
    assert Nk[m - 1] == m - cut1
    assert 0 < R < 1 and sorted(T1) == sorted(T0) == list(range(m))
    for i in range(m):
        assert T1[i] - T0[i] >= 0 and T1[i] + T0[i] >= R
