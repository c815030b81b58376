"""Splitting one enumeration across processes (one GPU each).

PBAT's equal division (arXiv 2209.09711 Sec. 4.3, Eq. 6) at the top level:
with chi = 2^bits divisions of the state space, rank r of w takes the
contiguous block of divisions [r*chi/w, (r+1)*chi/w) and runs it through the
engine's range option.  Partial R, N_k and dR/dp of disjoint division
blocks add up exactly to the whole (Eq. 1 is a sum over states), so the
only exchange is a sum-reduce of 1 + m floating-point numbers and m + 1
integer counts after the enumeration (PBAT STEP 3).
"""
from __future__ import annotations

from typing import Callable, List, Optional, Tuple

import numpy as np


def shard_range(m: int, world: int, rank: int, bits: Optional[int] = None) -> Tuple[int, int, int]:
    """(range_bits, lo, hi) of rank's block of equal divisions."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    if bits is None:
        bits = 0
        while (1 << bits) < world and bits < m:
            bits += 1
        bits = min(m, bits + 4)   # a few divisions per rank for balance
    chi = 1 << bits
    lo = rank * chi // world
    hi = (rank + 1) * chi // world
    return bits, lo, hi


def pack(R: float, Nk: List[int], grad: Optional[List[float]]) -> Tuple[np.ndarray, np.ndarray]:
    """The two vectors of a sum-reduce: float64 [R, dR/dp...] and int64
    [N_0..N_m].  N_k travel as integers so that the reduce stays bit-exact:
    a count can exceed 2^53 (C(63, 31) is about 9.2e17), and a sum of
    disjoint blocks' counts is at most the whole network's, below 2^63."""
    g = [] if grad is None else list(grad)
    return (np.asarray([R] + g, dtype=np.float64), np.asarray(list(Nk), dtype=np.int64))


def unpack(fv: np.ndarray, nv: np.ndarray, with_grad: bool):
    R = float(fv[0])
    Nk = [int(x) for x in nv]
    grad = [float(x) for x in fv[1:]] if with_grad else None
    return R, Nk, grad


def reliability_sharded(net, compute: Callable, world: int, rank: int,
                        all_reduce: Callable[[np.ndarray], np.ndarray], grad: bool = False,
                        bits: Optional[int] = None):
    """Run this rank's block through `compute(net, range_bits, lo, hi, grad)`
    -> (R, Nk, grad or None), sum-reduce with `all_reduce` (once for the
    float64 vector, once for the int64 counts), return the whole
    (R, Nk, grad)."""
    b, lo, hi = shard_range(net.m, world, rank, bits)
    R, Nk, g = compute(net, b, lo, hi, grad)
    fv, nv = pack(R, Nk, g if grad else None)
    return unpack(all_reduce(fv), all_reduce(nv), grad)


def gpu_compute(net, range_bits: int, lo: int, hi: int, grad: bool, stream: int = 0):
    """The engine on this process's current CUDA device."""
    from . import options, reliability_net
    r = reliability_net(net, grad=grad, stream=stream,
                        opts=options(range_bits=range_bits, range_lo=lo, range_hi=hi))
    return r.R, r.Nk, (list(r.grad) if grad else None)


def torch_all_reduce(group=None) -> Callable[[np.ndarray], np.ndarray]:
    """Sum-reduce through torch.distributed (float64 or int64, on the
    backend's device)."""
    import torch
    import torch.distributed as dist

    def f(v: np.ndarray) -> np.ndarray:
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        t = torch.from_numpy(v).to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t.cpu().numpy()
    return f
