"""Splitting one enumeration across processes (one GPU each).

PBAT's equal division (arXiv 2209.09711 Sec. 4.3, Eq. 6) at the top level:
with chi = 2^bits divisions of the state space, rank r of w takes the
contiguous block of divisions [r*chi/w, (r+1)*chi/w) and runs it through the
engine's range option.  Partial R, N_k and dR/dp of disjoint division
blocks add up exactly to the whole (Eq. 1 is a sum over states), so the
only exchange is one sum-reduce of 1 + (m + 1) + m numbers after the
enumeration (PBAT STEP 3).
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


def pack(R: float, Nk: List[int], grad: Optional[List[float]]) -> np.ndarray:
    """One float64 vector [R, N_0..N_m, dR/dp...] for a sum-reduce (N_k stay
    exact: each is below 2^53 for m <= 52, and the reduce is over a handful
    of ranks)."""
    g = [] if grad is None else list(grad)
    return np.asarray([R] + [float(x) for x in Nk] + g, dtype=np.float64)


def unpack(v: np.ndarray, m: int, with_grad: bool):
    R = float(v[0])
    Nk = [int(round(x)) for x in v[1:m + 2]]
    grad = [float(x) for x in v[m + 2:]] if with_grad else None
    return R, Nk, grad


def reliability_sharded(net, compute: Callable, world: int, rank: int,
                        all_reduce: Callable[[np.ndarray], np.ndarray], grad: bool = False,
                        bits: Optional[int] = None):
    """Run this rank's block through `compute(net, range_bits, lo, hi, grad)`
    -> (R, Nk, grad or None), sum-reduce with `all_reduce`, return the whole
    (R, Nk, grad)."""
    b, lo, hi = shard_range(net.m, world, rank, bits)
    R, Nk, g = compute(net, b, lo, hi, grad)
    total = all_reduce(pack(R, Nk, g if grad else None))
    return unpack(total, net.m, grad)


def gpu_compute(net, range_bits: int, lo: int, hi: int, grad: bool, stream: int = 0):
    """The engine on this process's current CUDA device."""
    from . import options, reliability_net
    r = reliability_net(net, grad=grad, stream=stream,
                        opts=options(range_bits=range_bits, range_lo=lo, range_hi=hi))
    return r.R, r.Nk, (list(r.grad) if grad else None)


def torch_all_reduce(group=None) -> Callable[[np.ndarray], np.ndarray]:
    """Sum-reduce through torch.distributed (float64 on the backend's device)."""
    import torch
    import torch.distributed as dist

    def f(v: np.ndarray) -> np.ndarray:
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        t = torch.from_numpy(v).to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t.cpu().numpy()
    return f
