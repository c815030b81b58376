"""GB300 PBAT engine: exact two-terminal reliability of binary-state networks.

Thin Python binding over the C ABI in ``include/pbat.h`` (``libpbat.so``,
built in-tree by :mod:`paper_2209_09711_gb300.build`).  This module only
marshals arguments; every step of the enumeration runs in the CUDA kernels.
If the library is missing the calls raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpbat.so")

PBAT_OK = 0
PBAT_EINVAL = -1
PBAT_ERANGE = -2
PBAT_ECUDA = -3
PBAT_ETIMEOUT = -4
PBAT_ENOMEM = -5
PBAT_ENOTSUP = -6

ALGO_AUTO = 0
ALGO_FRONTIER = 1
ALGO_BITSLICE = 2

_ERR_NAMES = {
    PBAT_EINVAL: "PBAT_EINVAL", PBAT_ERANGE: "PBAT_ERANGE", PBAT_ECUDA: "PBAT_ECUDA",
    PBAT_ETIMEOUT: "PBAT_ETIMEOUT", PBAT_ENOMEM: "PBAT_ENOMEM", PBAT_ENOTSUP: "PBAT_ENOTSUP",
}


class PbatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    """Mirror of ``pbat_options``."""
    _fields_ = [
        ("struct_size", ctypes.c_int),
        ("algo", ctypes.c_int),
        ("prefix_bits", ctypes.c_int),
        ("walk_bits", ctypes.c_int),
        ("block_threads", ctypes.c_int),
        ("prune", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("occupancy", ctypes.c_int),
        ("launches", ctypes.c_int),
        ("range_bits", ctypes.c_int),
        ("range_lo", ctypes.c_uint64),
        ("range_hi", ctypes.c_uint64),
        ("time_budget_s", ctypes.c_double),
        ("stats", ctypes.c_uint64 * 8),
    ]


class Graph(ctypes.Structure):
    """Mirror of ``pbat_graph``."""
    _fields_ = [
        ("n_nodes", ctypes.c_int),
        ("n_arcs", ctypes.c_int),
        ("tail", ctypes.POINTER(ctypes.c_int32)),
        ("head", ctypes.POINTER(ctypes.c_int32)),
        ("directed", ctypes.c_int),
        ("source", ctypes.c_int),
        ("sink", ctypes.c_int),
    ]


_lock = threading.Lock()
_lib = None

# every symbol include/pbat.h declares
EXPORTED = [
    "pbat_options_init", "pbat_reliability", "pbat_reliability_grad",
    "pbat_reliability_batched", "pbat_plan_create", "pbat_plan_execute", "pbat_plan_read",
    "pbat_plan_destroy", "pbat_plan_stats", "pbat_plan_describe", "pbat_reliability_noalloc",
    "pbat_kernel_source", "pbat_batch_kernel_source", "pbat_batch_grad_kernel_source",
    "pbat_last_error", "pbat_version",
]


def load(path: Optional[str] = None):
    """Load libpbat.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_2209_09711_gb300.build.build()")
        lib = ctypes.CDLL(p)
        I, D, V = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        PI32 = ctypes.POINTER(ctypes.c_int32)
        PD = ctypes.POINTER(ctypes.c_double)
        PU = ctypes.POINTER(ctypes.c_uint64)
        PO = ctypes.POINTER(Options)
        lib.pbat_options_init.argtypes = [PO]
        lib.pbat_options_init.restype = None
        lib.pbat_reliability.argtypes = [I, I, PI32, PI32, I, PD, I, I, PO, V, PD, PU]
        lib.pbat_reliability.restype = I
        lib.pbat_reliability_grad.argtypes = [I, I, PI32, PI32, I, PD, I, I, PO, V, PD, PU, PD]
        lib.pbat_reliability_grad.restype = I
        lib.pbat_reliability_batched.argtypes = [I, ctypes.POINTER(Graph), I, PD, PO, V, PD, PU, PD]
        lib.pbat_reliability_batched.restype = I
        lib.pbat_plan_create.argtypes = [I, I, PI32, PI32, I, PD, I, I, I, PO, V,
                                         ctypes.POINTER(ctypes.c_void_p)]
        lib.pbat_plan_create.restype = I
        lib.pbat_plan_execute.argtypes = [V, V]
        lib.pbat_plan_execute.restype = I
        lib.pbat_plan_read.argtypes = [V, V, PD, PU, PD]
        lib.pbat_plan_read.restype = I
        lib.pbat_plan_stats.argtypes = [V, PU]
        lib.pbat_plan_stats.restype = I
        lib.pbat_plan_describe.argtypes = [V, ctypes.POINTER(ctypes.c_int)]
        lib.pbat_plan_describe.restype = I
        lib.pbat_plan_destroy.argtypes = [V]
        lib.pbat_plan_destroy.restype = None
        lib.pbat_reliability_noalloc.argtypes = [I, I, PI32, PI32, I, PD, I, I, PO, V, PD, PU]
        lib.pbat_reliability_noalloc.restype = I
        lib.pbat_kernel_source.argtypes = [I, I, PI32, PI32, I, PD, I, I, I, PO, ctypes.c_char_p,
                                           ctypes.c_size_t]
        lib.pbat_kernel_source.restype = I
        lib.pbat_batch_kernel_source.argtypes = [I, ctypes.POINTER(Graph), I, PO, ctypes.c_char_p,
                                                 ctypes.c_size_t]
        lib.pbat_batch_kernel_source.restype = I
        lib.pbat_batch_grad_kernel_source.argtypes = [I, ctypes.POINTER(Graph), I, PD, PO,
                                                      ctypes.c_char_p, ctypes.c_size_t]
        lib.pbat_batch_grad_kernel_source.restype = I
        lib.pbat_last_error.argtypes = []
        lib.pbat_last_error.restype = ctypes.c_char_p
        lib.pbat_version.argtypes = []
        lib.pbat_version.restype = I
        if path is None:
            _lib = lib
        return lib


def options(**kw) -> Options:
    o = Options()
    load().pbat_options_init(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _check(rc: int):
    if rc != PBAT_OK:
        msg = load().pbat_last_error().decode(errors="replace")
        raise PbatError(rc, msg)


def _i32(xs):
    a = np.ascontiguousarray(np.asarray(xs, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(xs):
    a = np.ascontiguousarray(np.asarray(xs, dtype=np.float64))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Result:
    R: float
    Nk: List[int]
    grad: Optional[np.ndarray] = None
    stats: Optional[List[int]] = None


def reliability(n: int, tail: Sequence[int], head: Sequence[int], p: Sequence[float],
                source: int, sink: int, directed: bool = False, grad: bool = False,
                opts: Optional[Options] = None, stream: int = 0) -> Result:
    """R, N_k (and dR/dp if grad) of one network through the C ABI."""
    lib = load()
    t, tp = _i32(tail)
    h, hp = _i32(head)
    pv, pp = _f64(p)
    m = len(t)
    R = ctypes.c_double()
    Nk = (ctypes.c_uint64 * (m + 1))()
    o = opts if opts is not None else options()
    if grad:
        g = np.zeros(m, dtype=np.float64)
        rc = lib.pbat_reliability_grad(n, m, tp, hp, int(directed), pp, source, sink,
                                       ctypes.byref(o), ctypes.c_void_p(stream), ctypes.byref(R),
                                       Nk, g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    else:
        g = None
        rc = lib.pbat_reliability(n, m, tp, hp, int(directed), pp, source, sink, ctypes.byref(o),
                                  ctypes.c_void_p(stream), ctypes.byref(R), Nk)
    _check(rc)
    return Result(R.value, list(Nk), g, list(o.stats))


def reliability_net(net, p=None, grad: bool = False, opts: Optional[Options] = None,
                    stream: int = 0) -> Result:
    """Convenience wrapper for an object with n, tail, head, p, source, sink, directed."""
    return reliability(net.n, net.tail, net.head, net.p if p is None else p, net.source, net.sink,
                       net.directed, grad, opts, stream)


def reliability_batched(nets, pvecs, grad: bool = False, want_nk: bool = True,
                        opts: Optional[Options] = None, stream: int = 0):
    """Batched call: nets is a list of networks, pvecs[g] a list of n_pvec
    p-vectors for network g.  Returns (R[g][k], Nk[g], grad[g][k] or None)."""
    lib = load()
    G = len(nets)
    K = len(pvecs[0])
    keep = []
    graphs = (Graph * G)()
    for i, net in enumerate(nets):
        t, tp = _i32(net.tail)
        h, hp = _i32(net.head)
        keep += [t, h]
        graphs[i] = Graph(net.n, len(t), tp, hp, int(net.directed), net.source, net.sink)
    flat = np.concatenate([np.asarray(pv, dtype=np.float64).reshape(K, -1).ravel() for pv in pvecs])
    pv, pp = _f64(flat)
    R = np.zeros(G * K, dtype=np.float64)
    ms = [len(net.tail) for net in nets]
    Nk = np.zeros(sum(m + 1 for m in ms), dtype=np.uint64) if want_nk else None
    gr = np.zeros(flat.shape[0], dtype=np.float64) if grad else None
    o = opts if opts is not None else options()
    rc = lib.pbat_reliability_batched(
        G, graphs, K, pp, ctypes.byref(o), ctypes.c_void_p(stream),
        R.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        Nk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if want_nk else None,
        gr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if grad else None)
    _check(rc)
    Rs = R.reshape(G, K)
    Nks, grads = [], []
    off = 0
    goff = 0
    for m in ms:
        if want_nk:
            Nks.append([int(v) for v in Nk[off:off + m + 1]])
        off += m + 1
        if grad:
            grads.append(gr[goff:goff + K * m].reshape(K, m))
        goff += K * m
    return Rs, (Nks if want_nk else None), (grads if grad else None)


class Plan:
    """A prepared enumeration (pbat_plan_*): tables live on the device, and
    execute() launches the kernels on a stream without any host work."""

    def __init__(self, net, p=None, grad: bool = False, opts: Optional[Options] = None,
                 stream: int = 0):
        lib = load()
        self._t, tp = _i32(net.tail)
        self._h, hp = _i32(net.head)
        self._p, pp = _f64(net.p if p is None else p)
        self.m = len(self._t)
        self.grad = grad
        self.opts = opts if opts is not None else options()
        h = ctypes.c_void_p()
        _check(lib.pbat_plan_create(net.n, self.m, tp, hp, int(net.directed), pp, net.source,
                                    net.sink, int(grad), ctypes.byref(self.opts),
                                    ctypes.c_void_p(stream), ctypes.byref(h)))
        self._handle = h

    def execute(self, stream: int = 0):
        _check(load().pbat_plan_execute(self._handle, ctypes.c_void_p(stream)))

    def read(self, stream: int = 0) -> Result:
        R = ctypes.c_double()
        Nk = (ctypes.c_uint64 * (self.m + 1))()
        g = np.zeros(self.m, dtype=np.float64) if self.grad else None
        _check(load().pbat_plan_read(
            self._handle, ctypes.c_void_p(stream), ctypes.byref(R), Nk,
            g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if self.grad else None))
        st = (ctypes.c_uint64 * 8)()
        _check(load().pbat_plan_stats(self._handle, st))
        return Result(R.value, list(Nk), g, list(st))

    def describe(self) -> dict:
        """Kernel and split the plan uses (pbat_plan_describe)."""
        out = (ctypes.c_int * 8)()
        _check(load().pbat_plan_describe(self._handle, out))
        return dict(kernel="bitslice" if out[0] == ALGO_BITSLICE else "frontier", lane_bits=out[1],
                    thread_bits=out[2], walk_bits=out[3], prefix_bits=out[4], block_threads=out[5],
                    blocks=out[6], grad=bool(out[7]))

    def close(self):
        if self._handle:
            load().pbat_plan_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_source(net, opts: Optional[Options] = None, grad: bool = False, p=None) -> str:
    """The generated CUDA source of the bit-sliced kernel for a network."""
    lib = load()
    t, tp = _i32(net.tail)
    h, hp = _i32(net.head)
    pv, pp = _f64(net.p if p is None else p)
    o = opts if opts is not None else options()
    n = lib.pbat_kernel_source(net.n, len(t), tp, hp, int(net.directed), pp, net.source, net.sink,
                               int(grad), ctypes.byref(o), None, 0)
    if n < 0:
        _check(n)
    buf = ctypes.create_string_buffer(n + 1)
    lib.pbat_kernel_source(net.n, len(t), tp, hp, int(net.directed), pp, net.source, net.sink,
                           int(grad), ctypes.byref(o), buf, n + 1)
    return buf.value.decode()


def batch_kernel_source(nets, n_pvec: int, opts: Optional[Options] = None) -> str:
    """The generated CUDA source of the batched bit-sliced module."""
    lib = load()
    keep = []
    graphs = (Graph * len(nets))()
    for i, net in enumerate(nets):
        t, tp = _i32(net.tail)
        h, hp = _i32(net.head)
        keep += [t, h]
        graphs[i] = Graph(net.n, len(t), tp, hp, int(net.directed), net.source, net.sink)
    o = opts if opts is not None else options()
    n = lib.pbat_batch_kernel_source(len(nets), graphs, n_pvec, ctypes.byref(o), None, 0)
    if n < 0:
        _check(n)
    buf = ctypes.create_string_buffer(n + 1)
    lib.pbat_batch_kernel_source(len(nets), graphs, n_pvec, ctypes.byref(o), buf, n + 1)
    return buf.value.decode()


def batch_grad_kernel_source(nets, pvecs, opts: Optional[Options] = None) -> str:
    """The generated CUDA source of the batched gradient module."""
    lib = load()
    keep = []
    graphs = (Graph * len(nets))()
    for i, net in enumerate(nets):
        t, tp = _i32(net.tail)
        h, hp = _i32(net.head)
        keep += [t, h]
        graphs[i] = Graph(net.n, len(t), tp, hp, int(net.directed), net.source, net.sink)
    K = len(pvecs[0])
    flat = np.concatenate([np.asarray(pv, dtype=np.float64).reshape(K, -1).ravel() for pv in pvecs])
    pv, pp = _f64(flat)
    o = opts if opts is not None else options()
    n = lib.pbat_batch_grad_kernel_source(len(nets), graphs, K, pp, ctypes.byref(o), None, 0)
    if n < 0:
        _check(n)
    buf = ctypes.create_string_buffer(n + 1)
    lib.pbat_batch_grad_kernel_source(len(nets), graphs, K, pp, ctypes.byref(o), buf, n + 1)
    return buf.value.decode()


def version() -> int:
    return load().pbat_version()


from .autograd import PBATReliability, reliability_torch  # noqa: E402,F401
