"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every function include/pbat.h declares, and rejects malformed input
before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2209_09711_gb300 import build
    build.build()
    import paper_2209_09711_gb300 as pb
    return pb


def _declared():
    text = open(os.path.join(ROOT, "include", "pbat.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pbat_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "pbat_reliability" in names and "pbat_reliability_batched" in names
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in names:
        assert hasattr(so, name), name
    assert set(names) <= set(lib.EXPORTED)


def test_options_init_and_version(lib):
    o = lib.options()
    assert o.struct_size == ctypes.sizeof(lib.Options)
    assert o.prune == 1 and o.prefix_bits == -1 and o.walk_bits == -1 and o.algo == 0
    assert lib.version() >= 10000


@pytest.mark.parametrize("case,code", [
    (dict(source=0, sink=0), "PBAT_EINVAL"),             # source == sink
    (dict(tail=[0, 1, 2], head=[1, 2, 2]), "PBAT_EINVAL"),  # loop
    (dict(tail=[0, 1, 5], head=[1, 2, 3]), "PBAT_EINVAL"),  # node id out of range
    (dict(p=[0.5, 1.5, 0.5]), "PBAT_EINVAL"),            # p outside [0, 1]
    (dict(p=[0.5, float("nan"), 0.5]), "PBAT_EINVAL"),   # NaN
    (dict(n=65), "PBAT_ERANGE"),                         # too many nodes
])
def test_validation_errors(lib, case, code):
    args = dict(n=4, tail=[0, 1, 2], head=[1, 2, 3], p=[0.9, 0.9, 0.9], source=0, sink=3)
    args.update(case)
    with pytest.raises(lib.PbatError) as e:
        lib.reliability(args["n"], args["tail"], args["head"], args["p"], args["source"],
                        args["sink"])
    assert code in str(e.value)


def test_too_many_arcs(lib):
    with pytest.raises(lib.PbatError) as e:
        lib.reliability(3, [0] * 64, [1] * 64, [0.5] * 64, 0, 2)
    assert "PBAT_ERANGE" in str(e.value)


def test_bad_options(lib):
    o = lib.options(range_bits=4, range_lo=3, range_hi=2)
    with pytest.raises(lib.PbatError) as e:
        lib.reliability(4, [0, 1, 2, 0, 1], [1, 2, 3, 2, 3], [0.9] * 5, 0, 3, opts=o)
    assert "PBAT_EINVAL" in str(e.value)
    o = lib.options()
    o.struct_size = 7
    with pytest.raises(lib.PbatError):
        lib.reliability(4, [0, 1, 2], [1, 2, 3], [0.9] * 3, 0, 3, opts=o)


def test_batched_validation(lib):
    import synth
    net = synth.bridge([0.9] * 5)
    bad = synth.Network(4, [0, 1], [1, 1], [0.5, 0.5], 0, 3)
    with pytest.raises(lib.PbatError) as e:
        lib.reliability_batched([net, bad], [[net.p], [bad.p]])
    assert "network 1" in str(e.value)


def test_no_gpu_gives_ecuda_not_a_crash(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lib.PbatError) as e:
        lib.reliability(4, [0, 0, 1, 1, 2], [1, 2, 2, 3, 3], [0.9] * 5, 0, 3)
    assert "PBAT_ECUDA" in str(e.value)


def test_host_fault_injection_at_planning(lib, monkeypatch):
    """PBAT_FAULT injects failures on the host only.  The planning site is
    reachable without a GPU (the kernel-source diagnostics plan the network):
    it fails with its error code and message while listed, exact site names
    only, and the next call without it succeeds."""
    import synth
    net = synth.workload_grid_3x6()
    nets, _ = synth.workload_batched(3, 2)
    good = lib.kernel_source(net)
    monkeypatch.setenv("PBAT_FAULT", "launch,plan")
    with pytest.raises(lib.PbatError) as e:
        lib.kernel_source(net)
    assert e.value.code == lib.PBAT_EINVAL and "injected fault: planning" in str(e.value)
    with pytest.raises(lib.PbatError):
        lib.batch_kernel_source(nets, 2)
    for other in ("planning", "xplan", "compile,alloc,launch", ""):
        monkeypatch.setenv("PBAT_FAULT", other)
        assert lib.kernel_source(net) == good
    monkeypatch.delenv("PBAT_FAULT")
    assert lib.kernel_source(net) == good
