"""The allocation-free entry point, pbat_reliability_noalloc.

Callers whose device memory is owned by another allocator (or capped), or
who cannot afford an allocation on their path, get R and N_k from a static
scratch array inside the library instead of cudaMalloc.  This checks,
through the C ABI, that two calls in a row agree with pbat_reliability and
with the CPU oracle on the same inputs (N_k exactly, R within the 1e-12
relative tolerance used by the parity tests) -- on whole small networks, a
network of more than 32 nodes (64-bit node masks), a range of equal
divisions, the prune off and the largest walk table -- and that a walk
table larger than the static scratch is refused.  The file name sorts last
so a run that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_09711_gb300 import build
    build.build()
    import paper_2209_09711_gb300 as mod
    return mod


def _noalloc(pb, net, opts=None):
    lib = pb.load()
    t = np.ascontiguousarray(net.tail, dtype=np.int32)
    h = np.ascontiguousarray(net.head, dtype=np.int32)
    p = np.ascontiguousarray(net.p, dtype=np.float64)
    R = ctypes.c_double()
    Nk = (ctypes.c_uint64 * (net.m + 1))()
    rc = lib.pbat_reliability_noalloc(
        net.n, net.m, t.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        h.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(net.directed),
        p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), net.source, net.sink,
        ctypes.byref(opts) if opts is not None else None, None, ctypes.byref(R), Nk)
    return rc, R.value, list(Nk)


def _wide_network():
    """40 nodes (64-bit node masks), 44 arcs: a path with chords."""
    n = 40
    tail = list(range(n - 1)) + [0, 5, 10, 20, 3]
    head = list(range(1, n)) + [10, 15, 30, 39, 25]
    p = [0.9 - 0.01 * (k % 7) for k in range(len(tail))]
    return synth.Network(n, tail, head, p, 0, n - 1, False, "wide-40")


CASES = {
    "small-random": (synth.workload_small_random, {}),
    "grid-3x6": (synth.workload_grid_3x6, {}),
    "figure1-directed": (lambda: synth.figure1(True), {}),
    "grid-walk-12": (synth.workload_grid_3x6, dict(walk_bits=12)),
    "grid-prune-off": (synth.workload_grid_3x6, dict(prune=0)),
    "grid-range": (synth.workload_grid_3x6, dict(range_bits=9, range_lo=100, range_hi=133)),
    "wide-40-range": (_wide_network,
                      dict(range_bits=26, range_lo=(1 << 26) - 7, range_hi=(1 << 26) - 5)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_reliability_and_oracle_twice(pb, case):
    make, kw = CASES[case]
    net = make()
    ref = pb.reliability_net(net, opts=pb.options(**kw))
    rb = kw.get("range_bits", 0)
    orc = oracle.enumerate_states(net, prefix_bits=rb, prefix_lo=kw.get("range_lo", 0),
                                  prefix_hi=kw.get("range_hi", 1 << rb))
    assert ref.Nk == orc.Nk
    for _ in range(2):
        rc, R, Nk = _noalloc(pb, net, pb.options(**kw) if kw else None)
        assert rc == pb.PBAT_OK, pb.load().pbat_last_error()
        assert Nk == ref.Nk == orc.Nk
        assert abs(R - ref.R) <= 1e-12 * abs(ref.R)
        assert abs(R - orc.R) <= 1e-12 * abs(orc.R)


def test_noalloc_refuses_oversized_walk_table(pb):
    net = synth.workload_grid_3x6()
    rc, _, _ = _noalloc(pb, net, pb.options(walk_bits=13))
    assert rc == pb.PBAT_ERANGE
    assert b"static scratch" in pb.load().pbat_last_error()
