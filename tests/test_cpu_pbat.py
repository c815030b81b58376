"""The benchmark's CPU baseline (the paper's PBAT in C on POSIX threads,
cpu_pbat/) against the oracle, on the CPU.

It must compute what the oracle computes (Eq. 1 over the same states): N_k
exactly, R within 1e-12 relative, T1 - T0 within its FP64 rounding -- on
whole small networks and on sampled equal divisions (Sec. 4.3) of the
benchmark workloads, whatever the thread count.
"""
import math

import pytest

import cpu_pbat
import oracle
import synth


def _grad_tol(gstar, t1, t0):
    # the baseline sums T1 and T0 in FP64, as the paper's program would: its
    # T1 - T0 is within a few units of 2^-53 of T1 + T0 (Kahan sums), which
    # for an ill-conditioned arc is more than 1e-12 of the difference
    return 1e-12 * abs(gstar) + 16 * 2.0**-53 * (t1 + t0) + 1e-300


def _check(R, Nk, g, ref, ctx):
    assert Nk == ref.Nk, ctx
    assert abs(R - ref.R) <= 1e-12 * abs(ref.R) + 1e-300, (ctx, R, ref.R)
    if g is not None:
        for i, (a, b) in enumerate(zip(g, ref.grad_t1t0)):
            assert abs(a - b) <= _grad_tol(b, ref.T1[i], ref.T0[i]), (ctx, i, a, b)


@pytest.mark.parametrize("directed", [False, True])
def test_whole_space_random_networks(directed):
    for seed in range(40):
        rng = synth.SplitMix64(4100 + seed)
        net = synth.random_small(8800 + seed, n=2 + rng.below(8), m=1 + rng.below(14),
                                 directed=directed, p_lo=0.02, p_hi=0.98)
        ref = oracle.enumerate_states(net, grad=True)
        for threads in (1, 3):
            R, Nk, g = cpu_pbat.whole(net, threads, grad=True)
            _check(R, Nk, g, ref, f"seed={seed} threads={threads}")


def test_paper_values_and_deterministic_arcs():
    for directed in (True, False):
        R, Nk, _ = cpu_pbat.whole(synth.figure1(directed), 4)
        assert abs(R - 0.960175722) < 5e-10 and Nk == [0, 0, 1, 6, 11, 6, 1]
    R, Nk, _ = cpu_pbat.whole(synth.bridge([0.9] * 5), 2)
    assert abs(R - 0.97848) < 5e-11 and Nk == [0, 0, 2, 8, 5, 1]
    net = synth.Network(4, [0, 0, 1, 1, 2, 0, 1], [1, 2, 2, 3, 3, 1, 3],
                        [1.0, 0.0, 0.5, 0.25, 1.0, 0.7, 0.0], 0, 3, True)
    R, Nk, g = cpu_pbat.whole(net, 2, grad=True)
    _check(R, Nk, g, oracle.enumerate_states(net, grad=True), "p in {0, 1}")


@pytest.mark.parametrize("make,bits,picks", [
    (synth.workload_grid_3x6, 15, [0, 9999, (1 << 15) - 1]),
    (synth.workload_directed_20_34, 22, [0, 3_000_000, (1 << 22) - 1]),
    (synth.workload_random_24_40, 28, [0, 123_456_789, (1 << 28) - 1]),
])
def test_sampled_divisions_of_the_workloads(make, bits, picks):
    net = make()
    for d in picks:
        ref = oracle.enumerate_states(net, prefix_bits=bits, prefix_lo=d, prefix_hi=d + 1, grad=True)
        R, Nk, g = cpu_pbat.enumerate_divisions(net, bits, [d], 2, grad=True)
        _check(R, Nk, g, ref, f"{net.name} division {d}")
    # several divisions at once, over more threads than divisions
    ref = oracle.enumerate_states(net, prefix_bits=bits, prefix_lo=picks[0], prefix_hi=picks[0] + 3)
    R, Nk, _ = cpu_pbat.enumerate_divisions(net, bits, [picks[0], picks[0] + 1, picks[0] + 2], 8)
    _check(R, Nk, None, ref, "three divisions")


def test_thread_count_does_not_change_counts():
    net = synth.workload_small_random()
    base = cpu_pbat.whole(net, 1)
    for threads in (2, 5, 8, 64):
        R, Nk, _ = cpu_pbat.whole(net, threads)
        assert Nk == base[1]
        assert abs(R - base[0]) <= 1e-15
    m = net.m
    assert all(base[1][k] <= math.comb(m, k) for k in range(m + 1)) and base[1][m] == 1


def test_rate_reports_a_sample():
    r, info = cpu_pbat.rate(synth.workload_grid_3x6(), 0.2, 2, grad=False, sub_bits=14)
    assert r > 0 and info["states"] == info["divisions"] * (1 << 14)


def test_bad_input_is_rejected():
    net = synth.Network(3, [0, 1], [1, 1], [0.5, 0.5], 0, 2)   # a loop
    with pytest.raises(ValueError):
        cpu_pbat.whole(net, 1)
    net = synth.Network(3, [0, 1], [1, 2], [0.5, 1.5], 0, 2)   # p outside [0, 1]
    with pytest.raises(ValueError):
        cpu_pbat.whole(net, 1)
    net = synth.bridge([0.9] * 5)
    with pytest.raises(ValueError):
        cpu_pbat.enumerate_divisions(net, 2, [4], 1)          # division out of range


def _stored(name):
    """R, N_k and per-arc T1, T0 stored in tests/golden/ by make_golden.py
    (the oracle over every state), as exact rationals where they are sums."""
    import os
    from fractions import Fraction
    rows = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"{name}_full.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = line.split()
                rows.setdefault(w[0], []).append(w[1:])

    def val(hi, lo):
        return Fraction(float.fromhex(hi)) + Fraction(float.fromhex(lo))

    m = len(rows["NK"][0]) - 1
    T1, T0 = [Fraction(0)] * m, [Fraction(0)] * m
    for i, hi, lo in rows["T1"]:
        T1[int(i)] = val(hi, lo)
    for i, hi, lo in rows["T0"]:
        T0[int(i)] = val(hi, lo)
    return float(val(*rows["R"][0])), [int(v) for v in rows["NK"][0]], T1, T0


def _check_whole_against_stored(name, net):
    import os
    R, Nk, g = cpu_pbat.whole(net, os.cpu_count() or 1, grad=True)
    R0, N0, T1, T0 = _stored(name)
    assert Nk == N0
    assert abs(R - R0) <= 1e-12 * R0
    for i in range(net.m):
        gstar = float(T1[i] - T0[i])
        assert abs(g[i] - gstar) <= _grad_tol(gstar, float(T1[i]), float(T0[i])), (i, g[i], gstar)


def test_whole_grid_against_stored_values():
    """The baseline over all 2^27 states of the 3x6 grid reproduces the
    stored oracle values: a second, independent program (FP64 Kahan sums,
    binary-addition order, PLSA on bitmasks) against the long-double brute
    force (a few seconds on 8 cores)."""
    _check_whole_against_stored("grid-3x6", synth.workload_grid_3x6())


@pytest.mark.skipif(__import__("os").environ.get("PBAT_FULL_CPU") != "1",
                    reason="2^34 states: about 5 minutes on 8 cores; set PBAT_FULL_CPU=1")
def test_whole_directed_34_against_stored_values():
    """The same over all 2^34 states of the directed 34-arc workload."""
    _check_whole_against_stored("random-directed-n20-m34", synth.workload_directed_20_34())
