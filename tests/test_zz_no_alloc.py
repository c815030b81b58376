"""The allocation-free entry point, pbat_reliability_noalloc.

Callers whose device memory is owned by another allocator (or capped), or
who cannot afford an allocation on their path, get R and N_k from a static
scratch array inside the library instead of cudaMalloc.  This checks,
through the C ABI, that two calls in a row agree with pbat_reliability on
the same inputs (N_k exactly, R within the 1e-12 relative tolerance used by
the parity tests), and that a walk table larger than the static scratch is
refused.  The file name sorts last so a run that stops at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

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


@pytest.mark.parametrize("make", [synth.workload_small_random, synth.workload_grid_3x6,
                                  lambda: synth.figure1(True)])
def test_noalloc_matches_reliability_twice(pb, make):
    net = make()
    ref = pb.reliability_net(net)
    for _ in range(2):
        rc, R, Nk = _noalloc(pb, net)
        assert rc == pb.PBAT_OK, pb.load().pbat_last_error()
        assert Nk == ref.Nk
        assert abs(R - ref.R) <= 1e-12 * abs(ref.R)


def test_noalloc_refuses_oversized_walk_table(pb):
    net = synth.workload_grid_3x6()
    rc, _, _ = _noalloc(pb, net, pb.options(walk_bits=13))
    assert rc == pb.PBAT_ERANGE
    assert b"static scratch" in pb.load().pbat_last_error()
