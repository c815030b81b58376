"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

N_k must be bit-exact.  R must agree within 1e-12 relative.  dR/dp must
agree within 1e-12 relative where the oracle's T1/T0 condition number is
small, otherwise within 1e-12 * max(|g*|, 1e-4 * R) (the reading of the
1e-12 target for gradients that are cancellations of two large sums).
Full-size workloads the oracle cannot finish in seconds are checked on
sampled equal divisions (Sec. 4.3) -- the same division on both sides --
and through invariants that hold at any size.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

R_TOL = 1e-12


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


def check(res, ref, grad=False, ctx=""):
    assert res.Nk == ref.Nk, ctx
    assert abs(res.R - ref.R) <= R_TOL * abs(ref.R) + 1e-300, (ctx, res.R, ref.R)
    if grad:
        gstar = ref.grad_t1t0
        for i, (a, b) in enumerate(zip(res.grad, gstar)):
            tol = _grad_tol(b, ref.T1[i], ref.T0[i], ref.R)
            assert abs(a - b) <= tol, (ctx, i, a, b, tol)


def run(pb, net, p=None, grad=False, **opt):
    return pb.reliability_net(net, p=p, grad=grad, opts=pb.options(**opt))


# ---------------------------------------------------------------------------
# small cases, whole space
# ---------------------------------------------------------------------------

def test_small_random_workload(pb):
    net = synth.workload_small_random()
    ref = oracle.enumerate_states(net, grad=True)
    for prune in (1, 0):
        for walk in (-1, 0, 3, 6, 11):
            for algo in (pb.ALGO_FRONTIER, pb.ALGO_BITSLICE):
                check(run(pb, net, grad=True, prune=prune, walk_bits=walk, algo=algo), ref, True,
                      f"grad algo={algo} prune={prune} walk={walk}")
                check(run(pb, net, prune=prune, walk_bits=walk, algo=algo), ref, False,
                      f"algo={algo} prune={prune} walk={walk}")
    check(run(pb, net), ref)


@pytest.mark.parametrize("directed", [False, True])
def test_bitslice_random_graphs(pb, directed):
    for seed in range(25):
        rng = synth.SplitMix64(9100 + seed)
        m = 1 + rng.below(20)
        n = 2 + rng.below(12)
        net = synth.random_small(7000 + seed, n=n, m=m, directed=directed, p_lo=0.05, p_hi=0.95)
        ref = oracle.enumerate_states(net)
        gref = oracle.enumerate_states(net, grad=True)
        for walk in (-1, 2):
            check(run(pb, net, algo=pb.ALGO_BITSLICE, walk_bits=walk), ref, False, f"seed={seed}")
            check(run(pb, net, grad=True, algo=pb.ALGO_BITSLICE, walk_bits=walk), gref, True,
                  f"seed={seed} grad")


def test_paper_worked_example_and_bridge(pb):
    for directed in (True, False):
        net = synth.figure1(directed)
        res = run(pb, net, grad=True)
        assert abs(res.R - 0.960175722) < 5e-10
        assert res.Nk == [0, 0, 1, 6, 11, 6, 1]
        check(res, oracle.enumerate_states(net, grad=True), True)
    res = run(pb, synth.bridge([0.9] * 5))
    assert abs(res.R - 0.97848) < 5e-11 and res.Nk == [0, 0, 2, 8, 5, 1]


@pytest.mark.parametrize("directed", [False, True])
def test_random_graphs(pb, directed):
    for seed in range(30):
        rng = synth.SplitMix64(777 + seed)
        m = 1 + rng.below(18)
        n = 2 + rng.below(9)
        net = synth.random_small(5000 + seed, n=n, m=m, directed=directed, p_lo=0.02, p_hi=0.98)
        ref = oracle.enumerate_states(net, grad=True)
        check(run(pb, net, grad=True), ref, True, f"seed={seed}")
        check(run(pb, net, grad=True, algo=pb.ALGO_FRONTIER), ref, True, f"seed={seed} frontier")
        check(run(pb, net, prune=0), ref, False, f"seed={seed} noprune")


def test_edge_cases(pb):
    # a single s-t arc
    net = synth.Network(2, [0], [1], [0.3], 0, 1)
    res = run(pb, net, grad=True)
    assert res.Nk == [0, 1] and abs(res.R - 0.3) < 1e-16 and abs(res.grad[0] - 1.0) < 1e-15
    # sink unreachable in every state
    net = synth.Network(4, [0, 1], [1, 0], [0.6, 0.7], 0, 3)
    res = run(pb, net, grad=True)
    assert res.R == 0.0 and res.Nk == [0, 0, 0] and all(g == 0.0 for g in res.grad)
    # deterministic arcs (p = 0 and p = 1), parallel arcs, directed
    net = synth.Network(4, [0, 0, 1, 1, 2, 0, 1], [1, 2, 2, 3, 3, 1, 3],
                        [1.0, 0.0, 0.5, 0.25, 1.0, 0.7, 0.0], 0, 3, True)
    check(run(pb, net, grad=True), oracle.enumerate_states(net, grad=True), True, "p01")
    # more than 32 nodes: 64-bit node masks
    n = 40
    tail = list(range(n - 1)) + [0, 5, 10, 20]
    head = list(range(1, n)) + [10, 15, 30, 39]
    p = [0.9 - 0.01 * (k % 7) for k in range(len(tail))]
    net = synth.Network(n, tail, head, p, 0, n - 1)
    if net.m <= 22:
        check(run(pb, net, grad=True), oracle.enumerate_states(net, grad=True), True, "wide")
    else:
        r = run(pb, net, grad=True, range_bits=net.m - 18, range_lo=3, range_hi=4)
        ref = oracle.enumerate_states(net, prefix_bits=net.m - 18, prefix_lo=3, prefix_hi=4,
                                      grad=True)
        check(r, ref, True, "wide-range")


# ---------------------------------------------------------------------------
# full-size workloads: sampled divisions + invariants
# ---------------------------------------------------------------------------

def _sampled(pb, net, bits, picks, grad):
    for d in picks:
        r = run(pb, net, grad=grad, range_bits=bits, range_lo=d, range_hi=d + 1)
        ref = oracle.enumerate_states(net, prefix_bits=bits, prefix_lo=d, prefix_hi=d + 1,
                                      grad=grad)
        check(r, ref, grad, f"{net.name} division {d}/{1 << bits}")


def test_grid_3x6_full_and_sampled(pb):
    net = synth.workload_grid_3x6()
    m = net.m
    _sampled(pb, net, 12, [0, 1370, 3000, 4095], True)
    _sampled(pb, net, 9, [300], False)
    full = run(pb, net, grad=True)
    N = full.Nk
    assert all(v == 0 for v in N[:7]) and N[7] == 21 and N[m] == 1 and N[m - 1] == m
    assert N[m - 2] == math.comb(m, 2) - 2
    assert all(N[k] <= math.comb(m, k) for k in range(m + 1))
    # uniform p: R(p) = sum N_k p^k (1-p)^(m-k), sum_i dR/dp_i = dR/dp
    p = 0.9
    poly = sum(c * p**k * (1 - p) ** (m - k) for k, c in enumerate(N))
    dpoly = sum(c * (k * p ** (k - 1) * (1 - p) ** (m - k) - (m - k) * p**k * (1 - p) ** (m - k - 1))
                for k, c in enumerate(N))
    assert abs(full.R - poly) <= 1e-13
    assert abs(sum(full.grad) - dpoly) <= 1e-12
    fr = run(pb, net, grad=True, algo=pb.ALGO_FRONTIER)
    assert fr.Nk == N and abs(fr.R - full.R) <= 1e-14
    assert np.max(np.abs(np.asarray(fr.grad) - np.asarray(full.grad))) <= 1e-15
    # p = 1/2 ties R to the integer counts exactly
    half = run(pb, net, p=[0.5] * m)
    assert half.R == sum(N) / 2.0**m and half.Nk == N
    # every split of the work and both connectivity kernels give identical counts
    for walk in (4, 8, 12):
        for prune in (0, 1):
            for algo in (pb.ALGO_FRONTIER, pb.ALGO_BITSLICE):
                r = run(pb, net, walk_bits=walk, prune=prune, algo=algo)
                assert r.Nk == N and abs(r.R - full.R) <= 1e-14, (walk, prune, algo)


def test_directed_34_sampled(pb):
    net = synth.workload_directed_20_34()
    _sampled(pb, net, 20, [0, 400000, (1 << 20) - 1], True)
    _sampled(pb, net, 16, [40000], False)
    full = run(pb, net, grad=True)
    m = net.m
    assert full.Nk[m] == 1 and all(full.Nk[k] <= math.comb(m, k) for k in range(m + 1))
    # partial results over a partition of the divisions add up to the whole
    parts = [run(pb, net, grad=True, range_bits=2, range_lo=i, range_hi=i + 1) for i in range(4)]
    assert [sum(x) for x in zip(*[q.Nk for q in parts])] == full.Nk
    assert abs(sum(q.R for q in parts) - full.R) <= 1e-13
    g = np.sum([q.grad for q in parts], axis=0)
    assert np.max(np.abs(g - full.grad)) <= 1e-13


def test_fused_accumulator_placements_against_oracle(pb):
    """The fused kernel keeps a lane's accumulators in registers for short
    walks or small connectivity programs and in global slots otherwise: both,
    with the bit-sliced kernel forced, on sampled 2^19-state divisions of a
    dense seeded network (16 nodes, 38 arcs: its program at walk 9 is over
    128 operations per word), against the oracle."""
    tail, head, rng = synth.random_connected_undirected(16, 38, 4243)
    net = synth.Network(16, tail, head, synth.uniform_p(rng, 38, 0.85, 0.99), 0, 15, False, "dense-16-38")
    bits = 19
    for walk in (4, 9):
        src = pb.kernel_source(net, pb.options(walk_bits=walk, range_bits=bits), grad=True)
        want = "1" if walk <= 6 else "0"
        assert f"#define BS_ACC_REG {want}" in src
        for d in (7, (1 << bits) - 2):
            r = run(pb, net, grad=True, algo=pb.ALGO_BITSLICE, walk_bits=walk,
                    range_bits=bits, range_lo=d, range_hi=d + 1)
            ref = oracle.enumerate_states(net, prefix_bits=bits, prefix_lo=d, prefix_hi=d + 1, grad=True)
            check(r, ref, True, f"walk {walk} division {d}")


def test_random_40_sampled(pb):
    net = synth.workload_random_24_40()
    _sampled(pb, net, 26, [0, 20_000_000, (1 << 26) - 1], True)
    _sampled(pb, net, 22, [1_234_567], False)


# ---------------------------------------------------------------------------
# batched
# ---------------------------------------------------------------------------

def test_batched_against_oracle(pb):
    nets, pvecs = [], []
    for i in range(6):
        rng = synth.SplitMix64(31 + i)
        m = 5 + rng.below(10)
        net = synth.random_small(900 + i, n=3 + rng.below(6), m=m, directed=bool(i & 1))
        nets.append(net)
        pvecs.append([synth.uniform_p(rng, m, 0.05, 0.95) for _ in range(3)])
    R, Nk, G = pb.reliability_batched(nets, pvecs, grad=True)
    for g, net in enumerate(nets):
        for k in range(3):
            ref = oracle.enumerate_states(net, p=pvecs[g][k], grad=True)
            assert Nk[g] == ref.Nk
            assert abs(R[g][k] - ref.R) <= R_TOL * ref.R + 1e-300
            for i in range(net.m):
                assert abs(G[g][k][i] - ref.grad_t1t0[i]) <= _grad_tol(
                    ref.grad_t1t0[i], ref.T1[i], ref.T0[i], ref.R)


def test_batched_bitsliced_against_oracle_odd_many_pvectors(pb):
    """The bit-sliced batched module against the oracle: 19 p-vectors (one
    full register chunk of 16 plus a ragged 3, and an odd count that leaves a
    zero padding column in the tables), networks from 12 to 18 arcs so that
    items have walk arcs and prefix arcs, with and without the prune, and
    with the module's registers capped for 8 blocks per SM."""
    nets, pvecs = [], []
    for i in range(5):
        rng = synth.SplitMix64(71 + i)
        m = 12 + rng.below(7)
        nets.append(synth.random_small(950 + i, n=5 + rng.below(5), m=m, directed=bool(i & 1)))
        pvecs.append([synth.uniform_p(rng, m, 0.05, 0.95) for _ in range(19)])
    refs = [[oracle.enumerate_states(net, p=pvecs[g][k]) for k in range(19)] for g, net in enumerate(nets)]
    for prune, occ in ((1, 0), (0, 0), (1, 8)):
        R, Nk, _ = pb.reliability_batched(nets, pvecs, opts=pb.options(algo=pb.ALGO_BITSLICE, prune=prune,
                                                                       occupancy=occ))
        for g in range(len(nets)):
            assert Nk[g] == refs[g][0].Nk
            for k in range(19):
                assert abs(R[g][k] - refs[g][k].R) <= R_TOL * refs[g][k].R + 1e-300


def test_batched_frontier_kernel_matches_bitsliced(pb):
    nets, pvecs = synth.workload_batched(12, 5)
    R1, N1, _ = pb.reliability_batched(nets, pvecs, opts=pb.options(algo=pb.ALGO_FRONTIER))
    R2, N2, _ = pb.reliability_batched(nets, pvecs, opts=pb.options(algo=pb.ALGO_BITSLICE))
    assert N1 == N2
    assert np.max(np.abs(R1 - R2) / R1) <= 1e-13
    # prune off gives the same counts
    R3, N3, _ = pb.reliability_batched(nets, pvecs, opts=pb.options(prune=0))
    assert N3 == N2 and np.max(np.abs(R3 - R2) / R2) <= 1e-13


def test_batched_workload_matches_single(pb):
    nets, pvecs = synth.workload_batched()
    R, Nk, _ = pb.reliability_batched(nets, pvecs)
    R2, Nk2, _ = pb.reliability_batched(nets, pvecs)  # replayed CUDA graph
    assert np.array_equal(R, R2) and Nk == Nk2
    small = sorted(range(len(nets)), key=lambda g: nets[g].m)[:3]
    for g in small:
        for k in (0, 7, 15):
            r = pb.reliability_net(nets[g], p=pvecs[g][k])
            assert r.Nk == Nk[g]
            assert abs(r.R - R[g][k]) <= 1e-13 * r.R


# ---------------------------------------------------------------------------
# failure path and autograd
# ---------------------------------------------------------------------------

def test_time_budget_returns_etimeout_and_context_survives(pb):
    net = synth.workload_random_24_40()
    with pytest.raises(pb.PbatError) as e:
        run(pb, net, time_budget_s=0.002, prune=0)
    assert "PBAT_ETIMEOUT" in str(e.value)
    res = run(pb, synth.bridge([0.9] * 5))
    assert abs(res.R - 0.97848) < 5e-11


def test_autograd_function(pb):
    import torch
    net = synth.workload_small_random()
    p = torch.tensor(net.p, dtype=torch.float64, device="cuda", requires_grad=True)
    R = pb.PBATReliability.apply(p, net)
    R.backward()
    ref = oracle.enumerate_states(net, grad=True)
    assert abs(R.item() - ref.R) <= R_TOL * ref.R
    gref = ref.grad_t1t0
    for i in range(net.m):
        assert abs(p.grad[i].item() - gref[i]) <= _grad_tol(gref[i], ref.T1[i], ref.T0[i], ref.R)
    # R is affine in each p_i: central differences are exact up to rounding
    q = torch.tensor(net.p[:], dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: pb.PBATReliability.apply(x, net), (q,),
                                    eps=1e-4, atol=1e-9, rtol=1e-7)


# ---------------------------------------------------------------------------
# prune-aware planning (prune = 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("directed", [False, True])
def test_prune_aware_plans_whole_space(pb, directed):
    """Prefix arcs chosen by the prune-aware search: whole small networks,
    fused and R-only, bit-sliced kernel forced, several walk lengths."""
    for seed in range(20):
        rng = synth.SplitMix64(12100 + seed)
        m = 6 + rng.below(14)
        net = synth.random_small(12200 + seed, n=3 + rng.below(10), m=m, directed=directed,
                                 p_lo=0.03, p_hi=0.97)
        ref = oracle.enumerate_states(net, grad=True)
        for walk in (-1, 1, 3):
            o = dict(algo=pb.ALGO_BITSLICE, prune=2, walk_bits=walk)
            check(run(pb, net, grad=True, **o), ref, True, f"seed={seed} walk={walk} fused")
            check(run(pb, net, **o), ref, False, f"seed={seed} walk={walk} R")


@pytest.mark.parametrize("make,bits,picks", [
    (synth.workload_directed_20_34, 19, [0, 77777, (1 << 19) - 1]),
    (synth.workload_random_24_40, 25, [0, 12_345_678, (1 << 25) - 1]),
])
def test_prune_aware_plans_sampled_divisions(pb, make, bits, picks):
    net = make()
    for d in picks:
        ref = oracle.enumerate_states(net, prefix_bits=bits, prefix_lo=d, prefix_hi=d + 1, grad=True)
        for L, nt in ((10, 256), (7, 192), (4, 128)):
            o = dict(prune=2, walk_bits=L, block_threads=nt, range_bits=bits, range_lo=d,
                     range_hi=d + 1)
            check(run(pb, net, grad=True, **o), ref, True, f"{net.name} {d} L={L} fused")
            check(run(pb, net, **o), ref, False, f"{net.name} {d} L={L} R")


# ---------------------------------------------------------------------------
# precision: small R, extreme arc reliabilities
# ---------------------------------------------------------------------------

def _small_r_network(seed, n_chain=14, extra=4, p_lo=0.15, p_hi=0.35):
    """A chain from source to sink with a few shortcuts: R between about 1e-7 and 1e-4."""
    rng = synth.SplitMix64(seed)
    tail = list(range(n_chain))
    head = list(range(1, n_chain + 1))
    for _ in range(extra):
        u = rng.below(n_chain - 2)
        tail.append(u)
        head.append(u + 2 + rng.below(2))
    p = synth.uniform_p(rng, len(tail), p_lo, p_hi)
    return synth.Network(n_chain + 1, tail, head, p, 0, n_chain, False, f"small-r-{seed}")


def test_small_reliability_gradient_meets_tolerance(pb):
    """R between 5e-7 and 6e-5: the default path must meet the 1e-12 targets
    (the engine re-runs exactly when the bit-sliced bounds cannot), and the
    bit-sliced kernel, forced, must stay within its stated absolute bounds:
    2^-58.4 of the mass for R and 2^-57 for each gradient entry."""
    seen = []
    for seed in range(6):
        net = _small_r_network(14000 + seed, n_chain=12 + seed % 4)
        ref = oracle.enumerate_states(net, grad=True)
        seen.append(ref.R)
        check(run(pb, net, grad=True), ref, True, f"seed={seed} R={ref.R:.3g}")
        check(run(pb, net), ref, False, f"seed={seed}")
        forced = run(pb, net, grad=True, algo=pb.ALGO_BITSLICE)
        assert forced.Nk == ref.Nk
        assert abs(forced.R - ref.R) <= 2.0**-58.4 + 1e-12 * ref.R
        for i, (a, b) in enumerate(zip(forced.grad, ref.grad_t1t0)):
            assert abs(a - b) <= 2.0**-57 + 1e-12 * abs(b), (seed, i, a, b)
    assert min(seen) < 1e-6


def test_extreme_interior_reliabilities_on_walk_arcs(pb):
    """Arcs with p at 2^-20, 2^-19, 1 - 2^-19 and 1 - 2^-20 -- the edge of
    what the fused kernel accepts as walk arcs (it divides their sums by p
    and 1 - p) -- against the oracle, with every arc forced into the walk
    where the network allows it."""
    tail, head, rng = synth.random_connected_undirected(9, 18, 15151)
    ext = [2.0**-20, 2.0**-19, 1 - 2.0**-19, 1 - 2.0**-20]
    p = [ext[k % 4] if k % 3 else 0.5 + 0.4 * rng.uniform01() for k in range(18)]
    for directed in (False, True):
        net = synth.Network(9, tail, head, p, 0, 8, directed, "extreme-p")
        ref = oracle.enumerate_states(net, grad=True)
        for walk in (-1, 3, 8):
            check(run(pb, net, grad=True, walk_bits=walk), ref, True, f"dir={directed} walk={walk}")
            check(run(pb, net, grad=True, walk_bits=walk, algo=pb.ALGO_BITSLICE), ref, True,
                  f"dir={directed} walk={walk} bit-sliced")


# ---------------------------------------------------------------------------
# failure detection: host-side fault injection on the GPU path
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("site,code", [("compile", "PBAT_ECUDA"), ("alloc", "PBAT_ENOMEM"),
                                       ("launch", "PBAT_ECUDA")])
def test_injected_host_faults_then_clean_call(pb, site, code, monkeypatch):
    """PBAT_FAULT fails one host step the way its real call can; the call
    returns that error code with a message naming the site, no output is
    written, and the next call without the fault succeeds."""
    # a network structure no other test has compiled, so that the compile
    # site is reached (compiled kernels are cached per structure)
    tail, head, rng = synth.random_connected_undirected(7, 13, 16000 + len(site))
    net = synth.Network(7, tail, head, synth.uniform_p(rng, 13, 0.6, 0.95), 0, 6, False, site)
    ref = oracle.enumerate_states(net, grad=True)
    monkeypatch.setenv("PBAT_FAULT", site)
    with pytest.raises(pb.PbatError) as e:
        run(pb, net, grad=True, algo=pb.ALGO_BITSLICE)
    assert code in str(e.value) and "injected fault" in str(e.value)
    monkeypatch.delenv("PBAT_FAULT")
    check(run(pb, net, grad=True, algo=pb.ALGO_BITSLICE), ref, True, f"after {site}")
    check(run(pb, net), ref, False, f"after {site}, default")


# ---------------------------------------------------------------------------
# batched gradient (one launch of the gradient module)
# ---------------------------------------------------------------------------

def test_batched_gradient_against_oracle_odd_many_pvectors(pb):
    """dR/dp of several networks x 7 p-vectors from one launch, against the
    oracle's T1 - T0: directed and undirected networks, networks too small
    for five thread arcs, and a p-vector with arcs at exactly 0 and 1 (which
    then cannot be walk arcs)."""
    nets, pvecs = [], []
    for i in range(6):
        rng = synth.SplitMix64(17100 + i)
        m = 6 + rng.below(12)
        nets.append(synth.random_small(17200 + i, n=4 + rng.below(6), m=m, directed=bool(i & 1)))
        pv = [synth.uniform_p(rng, m, 0.05, 0.95) for _ in range(7)]
        if i == 2:
            pv[3][0], pv[3][m - 1] = 0.0, 1.0
        pvecs.append(pv)
    R, Nk, G = pb.reliability_batched(nets, pvecs, grad=True)
    for g, net in enumerate(nets):
        for k in range(7):
            ref = oracle.enumerate_states(net, p=pvecs[g][k], grad=True)
            assert Nk[g] == ref.Nk, g
            assert abs(R[g][k] - ref.R) <= R_TOL * ref.R + 1e-300, (g, k)
            gstar = ref.grad_t1t0
            for i in range(net.m):
                assert abs(G[g][k][i] - gstar[i]) <= _grad_tol(gstar[i], ref.T1[i], ref.T0[i], ref.R), \
                    (g, k, i, G[g][k][i], gstar[i])
    # the same batch without the gradient gives the same R and N_k
    R2, Nk2, _ = pb.reliability_batched(nets, pvecs)
    assert Nk2 == Nk and np.all(np.abs(R2 - R) <= 1e-13 * R)
    # the gradient module with its registers capped for 6 blocks per SM
    R3, Nk3, G3 = pb.reliability_batched(nets, pvecs, grad=True, opts=pb.options(occupancy=6))
    assert Nk3 == Nk and np.all(np.abs(R3 - R) <= 1e-13 * R)
    for g, net in enumerate(nets):
        assert np.all(np.abs(np.asarray(G3[g]) - np.asarray(G[g])) <= 1e-14)


def test_batched_workload_gradient_one_launch(pb):
    """The 64-network x 16-p-vector workload with the gradient: one
    persistent launch (timed by the library), R and N_k identical to the
    R-only module, and dR/dp of sampled networks against the factoring
    method's T1 - T0."""
    nets, pvecs = synth.workload_batched()
    o = pb.options()
    R, Nk, G = pb.reliability_batched(nets, pvecs, grad=True, opts=o)
    assert o.stats[5] == 1 and o.stats[4] > 0
    R0, Nk0, _ = pb.reliability_batched(nets, pvecs)
    assert Nk == Nk0 and np.max(np.abs(R - R0) / R0) <= 1e-13
    for g in (0, 9, 31, 47, 63):
        net = nets[g]
        for k in (0, 5, 15):
            T1, T0 = oracle.factor_t1t0(net, pvecs[g][k])
            Rk = oracle.factor(net, pvecs[g][k]).R
            for i in range(net.m):
                t1, t0 = sum(T1[i]), sum(T0[i])
                gs = (T1[i][0] - T0[i][0]) + (T1[i][1] - T0[i][1])   # from the hi/lo pairs
                assert abs(G[g][k][i] - gs) <= _grad_tol(gs, t1, t0, Rk), (g, k, i, G[g][k][i], gs)


# ---------------------------------------------------------------------------
# two-launch runs (the first resolves and defers, the second walks)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("directed", [False, True])
def test_two_launch_runs_against_oracle(pb, directed):
    """launches = 2 on whole small networks (few items, many warps without
    any), both kernels, both planning modes, several walk lengths; one
    launch gives identical results."""
    for seed in range(12):
        rng = synth.SplitMix64(18100 + seed)
        m = 8 + rng.below(12)
        net = synth.random_small(18200 + seed, n=3 + rng.below(10), m=m, directed=directed,
                                 p_lo=0.03, p_hi=0.97)
        ref = oracle.enumerate_states(net, grad=True)
        for prune in (1, 2):
            for walk in (0, 2, 4):
                o = dict(algo=pb.ALGO_BITSLICE, prune=prune, walk_bits=walk, launches=2)
                check(run(pb, net, grad=True, **o), ref, True, f"seed={seed} p{prune} w{walk} fused")
                check(run(pb, net, **o), ref, False, f"seed={seed} p{prune} w{walk} R")


def test_two_launch_runs_on_sampled_divisions_and_empty_range(pb):
    net = synth.workload_random_24_40()
    bits = 24
    for d in (5, 9_999_999):
        ref = oracle.enumerate_states(net, prefix_bits=bits, prefix_lo=d, prefix_hi=d + 1, grad=True)
        for L in (4, 9):
            o = dict(prune=2, walk_bits=L, block_threads=256, range_bits=bits, range_lo=d,
                     range_hi=d + 1, launches=2)
            check(run(pb, net, grad=True, **o), ref, True, f"division {d} L={L} fused")
            check(run(pb, net, **o), ref, False, f"division {d} L={L} R")
    # an empty range: no item in either launch
    r = run(pb, net, grad=True, range_bits=bits, range_lo=7, range_hi=7, launches=2, prune=2)
    assert r.R == 0.0 and all(v == 0 for v in r.Nk) and all(g == 0.0 for g in r.grad)
