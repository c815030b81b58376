"""The paper's PBAT on the host cores: the benchmark's timed CPU baseline.

``pbat_cpu.c`` runs PBAT as arXiv 2209.09711 Sec. 5.1 describes it -- equal
divisions of the state space (Sec. 4.3) on POSIX threads, binary-addition
order inside each division, the PLSA connectivity test (Sec. 3.2), FP64 sums
with Kahan compensation -- and is loaded here with ctypes.  It is a CPU
program for timing comparison, separate from the CUDA engine and from the
long-double oracle the tests use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
import time
from typing import List, Optional, Sequence, Tuple

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pbat_cpu.c")
_LIB = os.path.join(_HERE, "libpbat_cpu.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile with the host C compiler: -O3, POSIX threads, no vendor code."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cc = os.environ.get("CC", "gcc")
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([cc, "-O3", "-std=gnu99", "-pthread", "-shared", "-fPIC", "-o", tmp,
                               _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            I = ctypes.c_int
            PI = ctypes.POINTER(ctypes.c_int)
            PD = ctypes.POINTER(ctypes.c_double)
            PU = ctypes.POINTER(ctypes.c_uint64)
            lib.pcpu_enumerate.argtypes = [I, I, PI, PI, I, PD, I, I, I, PU, I, I, I, PD, PU, PD]
            lib.pcpu_enumerate.restype = I
            _lib = lib
    return _lib


def enumerate_divisions(net, prefix_bits: int, divisions: Sequence[int], threads: int,
                        grad: bool = False, p: Optional[Sequence[float]] = None
                        ) -> Tuple[float, List[int], Optional[List[float]]]:
    """R, N_k (and T1 - T0 per arc) over the listed equal divisions."""
    lib = _load()
    m = net.m
    pv = list(net.p if p is None else p)
    tail = (ctypes.c_int * m)(*net.tail)
    head = (ctypes.c_int * m)(*net.head)
    pp = (ctypes.c_double * m)(*pv)
    divs = (ctypes.c_uint64 * max(1, len(divisions)))(*divisions)
    R = ctypes.c_double()
    Nk = (ctypes.c_uint64 * (m + 1))()
    g = (ctypes.c_double * m)() if grad else None
    rc = lib.pcpu_enumerate(net.n, m, tail, head, int(net.directed), pp, net.source, net.sink,
                            prefix_bits, divs, len(divisions), threads, int(grad),
                            ctypes.byref(R), Nk, g)
    if rc != 0:
        raise ValueError(f"pcpu_enumerate failed ({rc})")
    return R.value, list(Nk), (list(g) if grad else None)


def whole(net, threads: int, grad: bool = False, p=None):
    """The whole space, chi = 2^d equal divisions with 2^d >= threads."""
    d = 0
    while (1 << d) < threads and d < net.m:
        d += 1
    return enumerate_divisions(net, d, list(range(1 << d)), threads, grad, p)


def rate(net, target_s: float, threads: int, grad: bool = True, sub_bits: int = 20):
    """States/s of PBAT on `threads` host threads: evenly spread divisions of
    2^sub_bits states each (seeded stride), as many as fill about target_s
    seconds, timed on the wall clock and extrapolated."""
    m = net.m
    sub = min(m, sub_bits)
    bits = m - sub
    total = 1 << bits

    def spread(k):
        step = max(1, total // k)
        return [(i * step + (step // 2)) % total for i in range(k)]

    # calibrate on one division per thread
    k = min(total, threads)
    t0 = time.perf_counter()
    enumerate_divisions(net, bits, spread(k), threads, grad)
    per = max(time.perf_counter() - t0, 1e-4)
    k = min(total, max(threads, int(target_s / per * k)))
    divs = spread(k)
    t0 = time.perf_counter()
    enumerate_divisions(net, bits, divs, threads, grad)
    wall = time.perf_counter() - t0
    states = len(divs) << sub
    return states / wall, dict(states=states, divisions=len(divs), division_states=1 << sub,
                               wall_s=wall, threads=threads)
