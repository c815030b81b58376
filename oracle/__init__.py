"""CPU oracle for the PBAT engine -- TEST INFRASTRUCTURE ONLY.

Plain brute force over all arc states (arXiv 2209.09711 Eq. 1 with the PLSA
connectivity test of Sec. 3.2), long double with compensated sums, written
in C (``pbat_oracle.c``) and loaded with ctypes.  For undirected networks
too large for the brute force, ``factor`` gives the same exact sums by a
second, independent method (``pbat_factoring.c``: factoring on each arc as a
dynamic program over frontier partitions), pinned against the brute force.
Only the tests, the package's smoke check and the benchmark's CPU-baseline
leg may import this module; the product path never does.  It shares no code
with the CUDA engine.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pbat_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# the factoring method (pbat_factoring.c), a separate library: independent of
# the brute force, and left out of the planted-mistake copies of it
_FSRC = os.path.join(_HERE, "pbat_factoring.c")
_FLIB = os.path.join(_HERE, "liboracle_factoring.so")
_lock = threading.Lock()
_lib = None
_flib = None


def _compile(src: str, lib: str, force: bool) -> str:
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        cc = os.environ.get("CC", "gcc")
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call([cc, "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no vendor libraries)."""
    _compile(_FSRC, _FLIB, force)
    return _compile(_SRC, _LIB, force)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # A test may point this at a copy of the oracle with a planted
            # mistake, to check that the pins catch it.
            path = os.environ.get("PBAT_ORACLE_LIB") or build()
            lib = ctypes.CDLL(path)
            I, U64, D = ctypes.c_int, ctypes.c_uint64, ctypes.c_double
            PI = ctypes.POINTER(ctypes.c_int)
            PD = ctypes.POINTER(ctypes.c_double)
            PU = ctypes.POINTER(ctypes.c_uint64)
            lib.orc_connected.argtypes = [I, I, PI, PI, I, I, I, U64]
            lib.orc_connected.restype = I
            lib.orc_plsa_layers.argtypes = [I, I, PI, PI, I, I, I, U64, PI]
            lib.orc_plsa_layers.restype = I
            lib.orc_state_probability.argtypes = [I, PD, U64, PD, PD]
            lib.orc_state_probability.restype = None
            lib.orc_enumerate.argtypes = [I, I, PI, PI, I, PD, I, I, I, U64, U64,
                                          PD, PD, PU, PD, PD, PD, PD]
            lib.orc_enumerate.restype = I
            lib.orc_grad_critical.argtypes = [I, I, PI, PI, I, PD, I, I, PD, PD]
            lib.orc_grad_critical.restype = I
            lib.orc_long_double_mant_bits.argtypes = []
            lib.orc_long_double_mant_bits.restype = I
            _lib = lib
    return _lib


def _ints(xs: Sequence[int]):
    return (ctypes.c_int * max(1, len(xs)))(*xs)


def _dbls(xs: Sequence[float]):
    return (ctypes.c_double * max(1, len(xs)))(*xs)


@dataclass
class OracleResult:
    R: float                 # hi + lo rounded to double
    R_hilo: tuple            # (hi, lo) of the long double sum
    Nk: List[int]
    T1: Optional[List[float]] = None
    T0: Optional[List[float]] = None
    T1_hilo: Optional[List[tuple]] = None
    T0_hilo: Optional[List[tuple]] = None

    @property
    def grad_t1t0(self) -> Optional[List[float]]:
        if self.T1_hilo is None:
            return None
        return [(a[0] - b[0]) + (a[1] - b[1]) for a, b in zip(self.T1_hilo, self.T0_hilo)]


def connected(net, x: int) -> bool:
    lib = _load()
    r = lib.orc_connected(net.n, net.m, _ints(net.tail), _ints(net.head), int(net.directed),
                          net.source, net.sink, x)
    if r < 0:
        raise ValueError("bad network")
    return bool(r)


def plsa_layers(net, x: int) -> List[int]:
    """1-based PLSA layer of every node for state x (0 = never placed)."""
    lib = _load()
    out = (ctypes.c_int * net.n)()
    r = lib.orc_plsa_layers(net.n, net.m, _ints(net.tail), _ints(net.head), int(net.directed),
                            net.source, net.sink, x, out)
    if r < 0:
        raise ValueError("bad network")
    return list(out)


def state_probability(p: Sequence[float], x: int) -> float:
    lib = _load()
    hi, lo = ctypes.c_double(), ctypes.c_double()
    lib.orc_state_probability(len(p), _dbls(p), x, ctypes.byref(hi), ctypes.byref(lo))
    return hi.value + lo.value


def enumerate_states(net, p: Optional[Sequence[float]] = None, prefix_bits: int = 0,
                     prefix_lo: int = 0, prefix_hi: Optional[int] = None,
                     grad: bool = False) -> OracleResult:
    """R, N_k and (optionally) T1/T0 over the states whose top prefix_bits
    coordinates lie in [prefix_lo, prefix_hi) (Sec. 4.3 equal divisions)."""
    lib = _load()
    m = net.m
    p = list(net.p if p is None else p)
    if prefix_hi is None:
        prefix_hi = 1 << prefix_bits
    Rh, Rl = ctypes.c_double(), ctypes.c_double()
    Nk = (ctypes.c_uint64 * (m + 1))()
    if grad:
        t1h, t1l = (ctypes.c_double * max(1, m))(), (ctypes.c_double * max(1, m))()
        t0h, t0l = (ctypes.c_double * max(1, m))(), (ctypes.c_double * max(1, m))()
    else:
        t1h = t1l = t0h = t0l = None
    r = lib.orc_enumerate(net.n, m, _ints(net.tail), _ints(net.head), int(net.directed),
                          _dbls(p), net.source, net.sink, prefix_bits, prefix_lo, prefix_hi,
                          ctypes.byref(Rh), ctypes.byref(Rl), Nk, t1h, t1l, t0h, t0l)
    if r < 0:
        raise ValueError("bad network or prefix range")
    res = OracleResult(R=Rh.value + Rl.value, R_hilo=(Rh.value, Rl.value), Nk=list(Nk))
    if grad:
        res.T1_hilo = [(t1h[i], t1l[i]) for i in range(m)]
        res.T0_hilo = [(t0h[i], t0l[i]) for i in range(m)]
        res.T1 = [a + b for a, b in res.T1_hilo]
        res.T0 = [a + b for a, b in res.T0_hilo]
    return res


def grad_critical(net, p: Optional[Sequence[float]] = None) -> List[float]:
    """dR/dp_i by the cancellation-free critical-state sum (whole space)."""
    lib = _load()
    m = net.m
    p = list(net.p if p is None else p)
    gh, gl = (ctypes.c_double * max(1, m))(), (ctypes.c_double * max(1, m))()
    r = lib.orc_grad_critical(net.n, m, _ints(net.tail), _ints(net.head), int(net.directed),
                              _dbls(p), net.source, net.sink, gh, gl)
    if r < 0:
        raise ValueError("bad network")
    return [gh[i] + gl[i] for i in range(m)]


def long_double_mantissa_bits() -> int:
    return _load().orc_long_double_mant_bits()


# ---------------------------------------------------------------------------
# The factoring method (undirected networks): exact values at full size
# ---------------------------------------------------------------------------

def _load_factoring():
    global _flib
    with _lock:
        if _flib is None:
            lib = ctypes.CDLL(_compile(_FSRC, _FLIB, False))
            I = ctypes.c_int
            PI = ctypes.POINTER(ctypes.c_int)
            PD = ctypes.POINTER(ctypes.c_double)
            PU = ctypes.POINTER(ctypes.c_uint64)
            lib.orc_factor.argtypes = [I, I, PI, PI, PD, I, I, PD, PD, PU, PI]
            lib.orc_factor.restype = I
            _flib = lib
    return _flib


@dataclass
class FactorResult:
    R: float
    R_hilo: tuple
    Nk: List[int]
    max_records: int


def factor(net, p: Optional[Sequence[float]] = None) -> FactorResult:
    """R and N_k of an undirected network by factoring (pbat_factoring.c)."""
    if net.directed:
        raise ValueError("the factoring method covers undirected networks only")
    lib = _load_factoring()
    m = net.m
    p = list(net.p if p is None else p)
    Rh, Rl = ctypes.c_double(), ctypes.c_double()
    Nk = (ctypes.c_uint64 * (m + 1))()
    mx = ctypes.c_int()
    r = lib.orc_factor(net.n, m, _ints(net.tail), _ints(net.head), _dbls(p), net.source, net.sink,
                       ctypes.byref(Rh), ctypes.byref(Rl), Nk, ctypes.byref(mx))
    if r < 0:
        raise ValueError({-1: "bad network", -2: "frontier wider than 16 nodes",
                          -3: "out of memory"}.get(r, str(r)))
    return FactorResult(Rh.value + Rl.value, (Rh.value, Rl.value), list(Nk), mx.value)


def factor_t1t0(net, p: Optional[Sequence[float]] = None):
    """T1_i = R with p_i = 1 and T0_i = R with p_i = 0, for every arc i (the
    sums of prod_{j != i} over connected states with x_i = 1 and x_i = 0),
    by factoring; returned as two lists of (hi, lo) pairs."""
    p = list(net.p if p is None else p)
    T1, T0 = [], []
    for i in range(net.m):
        q = p[:]
        q[i] = 1.0
        T1.append(factor(net, q).R_hilo)
        q[i] = 0.0
        T0.append(factor(net, q).R_hilo)
    return T1, T0
