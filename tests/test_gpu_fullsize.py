"""Full-size parity of the benchmark workloads, at the launch shapes the
benchmark times, against the oracle's exact values.

- 3x6 grid (2^27 states): the brute-force oracle's stored values
  (tests/golden/grid-3x6_full.txt, written by tests/golden/make_golden.py).
- 24-node, 40-arc network (2^40 states) and the 64 batched networks: the
  oracle's factoring method (exact sums by pivotal decomposition, pinned
  against the brute force in tests/test_oracle_factoring.py), computed here.
- Directed 34-arc network (2^34 states; the factoring method covers
  undirected networks only): the brute-force oracle's stored values
  (tests/golden/random-directed-n20-m34_full.txt), sampled equal divisions
  in both planning modes, and invariants of the whole run.

N_k must be bit-exact, R within 1e-12 relative, dR/dp within the reading of
the 1e-12 target for gradients: 1e-12 * |g*| where the oracle's T1/T0
condition number is small, else 1e-12 * max(|g*|, 1e-4 * R).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import bench
import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def pb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_09711_gb300 import build
    build.build()
    import paper_2209_09711_gb300 as mod
    return mod


def _grad_tol(gstar, t1, t0, R):
    kappa = (t1 + t0) / max(abs(gstar), 1e-300)
    if kappa * 2.0**-53 <= 1e-13:
        return 1e-12 * abs(gstar) + 1e-300
    return 1e-12 * max(abs(gstar), 1e-4 * abs(R)) + 1e-300


def _check(res, R, Nk, T=None, ctx=""):
    """T: (G, T1, T0) -- the exact gradient (from the oracle's hi/lo sums,
    not from T1 - T0 rounded to doubles) and the two sums for the condition
    number."""
    assert res.Nk == Nk, ctx
    assert abs(res.R - R) <= 1e-12 * abs(R) + 1e-300, (ctx, res.R, R)
    if T is not None and res.grad is not None:
        G, T1, T0 = T
        for i in range(len(Nk) - 1):
            assert abs(res.grad[i] - G[i]) <= _grad_tol(G[i], T1[i], T0[i], R), \
                (ctx, i, res.grad[i], G[i])


def _exact_grad(T1h, T0h):
    """dR/dp_i = T1_i - T0_i from (hi, lo) pairs, exactly, then rounded."""
    return [float(Fraction(a[0]) + Fraction(a[1]) - Fraction(b[0]) - Fraction(b[1]))
            for a, b in zip(T1h, T0h)]


def _bench_plan(pb, net, name, kind, **extra):
    """Run the benchmark's own launch: a prepared plan at the pinned shape."""
    grad = kind == "fused"
    plan = pb.Plan(net, grad=grad, opts=bench.shape_opts(pb, name, kind, **extra))
    plan.execute(0)
    plan.execute(0)   # a second launch re-zeroes and re-accumulates
    r = plan.read(0)
    plan.close()
    return r


def _golden(name):
    """R, N_k and (exact dR/dp, T1, T0) stored for a workload by
    tests/golden/make_golden.py (the brute-force oracle over every state)."""
    rows = {}
    with open(os.path.join(GOLDEN, f"{name}_full.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = line.split()
                rows.setdefault(w[0], []).append(w[1:])

    def val(hi, lo):
        return Fraction(float.fromhex(hi)) + Fraction(float.fromhex(lo))

    R = float(val(*rows["R"][0]))
    Nk = [int(v) for v in rows["NK"][0]]
    m = len(Nk) - 1
    T1, T0 = [Fraction(0)] * m, [Fraction(0)] * m
    for i, hi, lo in rows["T1"]:
        T1[int(i)] = val(hi, lo)
    for i, hi, lo in rows["T0"]:
        T0[int(i)] = val(hi, lo)
    G = [float(a - b) for a, b in zip(T1, T0)]
    return R, Nk, (G, [float(x) for x in T1], [float(x) for x in T0])


def test_grid_3x6_full_space_at_bench_shapes(pb):
    net = synth.workload_grid_3x6()
    R, Nk, T = _golden("grid-3x6")
    _check(_bench_plan(pb, net, "grid-3x6", "fused"), R, Nk, T, "bench fused launch")
    _check(_bench_plan(pb, net, "grid-3x6", "r_only"), R, Nk, ctx="bench R launch")
    # the public call with default options (autotuned shape)
    _check(pb.reliability_net(net, grad=True), R, Nk, T, "autotuned fused")
    _check(pb.reliability_net(net), R, Nk, ctx="autotuned R")
    # both planning modes and the plain GPU BAT
    for prune in (0, 2):
        _check(pb.reliability_net(net, grad=True, opts=pb.options(prune=prune, walk_bits=5)), R, Nk,
               T, f"prune {prune}")
    _check(pb.reliability_net(net, grad=True, opts=pb.options(algo=pb.ALGO_FRONTIER)), R, Nk, T,
           "frontier kernel")


@pytest.fixture(scope="module")
def forty():
    net = synth.workload_random_24_40()
    f = oracle.factor(net)
    T1h, T0h = oracle.factor_t1t0(net)
    return net, f.R, f.Nk, (_exact_grad(T1h, T0h), [sum(x) for x in T1h], [sum(x) for x in T0h])


def test_forty_arc_full_space_at_bench_shapes(pb, forty):
    """The benchmark's headline workload, 2^40 states, every output."""
    net, R, Nk, T = forty
    name = "random-undirected-n24-m40"
    _check(_bench_plan(pb, net, name, "fused"), R, Nk, T, "bench fused launch")
    _check(_bench_plan(pb, net, name, "r_only"), R, Nk, ctx="bench R launch")


def test_forty_arc_full_space_other_plans(pb, forty):
    """The source/sink-near planner (prune 1) and the public call with its
    autotuned choice."""
    net, R, Nk, T = forty
    _check(pb.reliability_net(net, grad=True, opts=pb.options(prune=1, walk_bits=10,
                                                                block_threads=160)),
           R, Nk, T, "prune 1 fused")
    _check(pb.reliability_net(net, opts=pb.options(prune=1, walk_bits=10, block_threads=224)), R, Nk,
           ctx="prune 1 R")
    _check(pb.reliability_net(net, grad=True), R, Nk, T, "autotuned fused")


def test_forty_arc_half_probability_and_partition(pb, forty):
    """At p = 1/2, R is the count of connected states over 2^40, exactly;
    partial results of four range blocks add up to the whole."""
    net, R, Nk, _ = forty
    m = net.m
    half = pb.reliability_net(net, p=[0.5] * m, opts=bench.shape_opts(pb, "random-undirected-n24-m40",
                                                                       "r_only"))
    assert half.Nk == Nk and half.R == sum(Nk) / 2.0**m
    parts = [pb.reliability_net(net, opts=pb.options(range_bits=2, range_lo=i, range_hi=i + 1,
                                                     prune=2, walk_bits=9, block_threads=128))
             for i in range(4)]
    assert [sum(x) for x in zip(*[q.Nk for q in parts])] == Nk
    assert abs(sum(q.R for q in parts) - R) <= 1e-12 * R


def test_batched_workload_full_against_factoring(pb):
    """All 64 networks x 16 p-vectors of the batched workload: every R and
    every network's N_k against the factoring method."""
    nets, pvecs = synth.workload_batched()
    Rb, Nkb, _ = pb.reliability_batched(nets, pvecs)
    for g, net in enumerate(nets):
        f0 = oracle.factor(net, pvecs[g][0])
        assert Nkb[g] == f0.Nk, g
        for k in range(len(pvecs[g])):
            Rk = f0.R if k == 0 else oracle.factor(net, pvecs[g][k]).R
            assert abs(Rb[g][k] - Rk) <= 1e-12 * Rk, (g, k, Rb[g][k], Rk)


def test_directed_34_full_space_at_bench_shapes(pb):
    """The directed workload, all 2^34 states, against the brute-force
    oracle's stored values: the benchmark's fused and R launches, the other
    planning mode and the autotuned call."""
    net = synth.workload_directed_20_34()
    name = "random-directed-n20-m34"
    R, Nk, T = _golden(name)
    _check(_bench_plan(pb, net, name, "fused"), R, Nk, T, "bench fused launch")
    _check(_bench_plan(pb, net, name, "r_only"), R, Nk, ctx="bench R launch")
    _check(pb.reliability_net(net, grad=True, opts=pb.options(prune=1, walk_bits=10,
                                                                block_threads=256)),
           R, Nk, T, "prune 1 fused")
    _check(pb.reliability_net(net, grad=True), R, Nk, T, "autotuned fused")


def test_directed_34_at_bench_shapes(pb):
    """The directed workload: sampled divisions in the benchmark's planning
    mode against the brute force, and invariants of the full run at the
    benchmark's shapes."""
    net = synth.workload_directed_20_34()
    name = "random-directed-n20-m34"
    fused = _bench_plan(pb, net, name, "fused")
    ronly = _bench_plan(pb, net, name, "r_only")
    m = net.m
    assert fused.Nk == ronly.Nk and abs(fused.R - ronly.R) <= 1e-13 * ronly.R
    assert fused.Nk[m] == 1 and all(fused.Nk[k] <= math.comb(m, k) for k in range(m + 1))
    for opts in (bench.shape_opts(pb, name, "fused"), pb.options(prune=1)):
        prune = opts.prune
        bits = 20
        for d in (0, 517_000, (1 << bits) - 1):
            o = bench.shape_opts(pb, name, "fused", range_bits=bits, range_lo=d, range_hi=d + 1) \
                if prune == 2 else pb.options(range_bits=bits, range_lo=d, range_hi=d + 1)
            r = pb.reliability_net(net, grad=True, opts=o)
            ref = oracle.enumerate_states(net, prefix_bits=bits, prefix_lo=d, prefix_hi=d + 1, grad=True)
            _check(r, ref.R, ref.Nk, (ref.grad_t1t0, ref.T1, ref.T0), f"division {d} prune {prune}")
    # p = 1/2 ties R to the counts
    half = pb.reliability_net(net, p=[0.5] * m, opts=bench.shape_opts(pb, name, "r_only"))
    assert half.Nk == fused.Nk and half.R == sum(fused.Nk) / 2.0**m
    # every planning mode and kernel gives identical counts
    plain = pb.reliability_net(net, opts=pb.options(algo=pb.ALGO_FRONTIER))
    assert plain.Nk == fused.Nk and abs(plain.R - fused.R) <= 1e-13 * fused.R
    g1 = pb.reliability_net(net, grad=True, opts=pb.options(prune=1))
    assert g1.Nk == fused.Nk
    assert np.max(np.abs(np.asarray(g1.grad) - np.asarray(fused.grad))) <= 1e-15


def test_small_random_full_space_at_default(pb):
    """The 8-node, 16-arc workload (2^16 states), whole space."""
    net = synth.workload_small_random()
    ref = oracle.enumerate_states(net, grad=True)
    _check(pb.reliability_net(net, grad=True), ref.R, ref.Nk, (ref.grad_t1t0, ref.T1, ref.T0),
           "default")
    f = oracle.factor(net)
    assert f.Nk == ref.Nk


def test_shard_blocks_sum_to_the_whole_at_bench_shape(pb, forty):
    """The sharded mode's blocks of equal divisions (four ranks, run here one
    after another on one GPU) at the benchmark's fused shape: their counts
    add up exactly to the whole, and R and dR/dp to the factoring values."""
    from paper_2209_09711_gb300 import shard
    net, R, Nk, (G, T1, T0) = forty
    name = "random-undirected-n24-m40"
    world = 4
    parts = []
    for rank in range(world):
        bits, lo, hi = shard.shard_range(net.m, world, rank)
        parts.append(_bench_plan(pb, net, name, "fused", range_bits=bits, range_lo=lo, range_hi=hi))
    fv = sum(shard.pack(q.R, q.Nk, list(q.grad))[0] for q in parts)
    nv = sum(shard.pack(q.R, q.Nk, list(q.grad))[1] for q in parts)
    Rs, Nks, gs = shard.unpack(fv, nv, True)
    assert Nks == Nk
    assert abs(Rs - R) <= 1e-12 * R
    for i in range(net.m):
        assert abs(gs[i] - G[i]) <= 4 * _grad_tol(G[i], T1[i], T0[i], R), (i, gs[i], G[i])
    # the library's own sharded driver on one rank (identity exchange)
    r1 = shard.reliability_sharded(net, shard.gpu_compute, 1, 0, lambda v: v, grad=True)
    assert r1[1] == Nk and abs(r1[0] - R) <= 1e-12 * R
