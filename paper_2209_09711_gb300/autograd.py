"""torch.autograd.Function over the PBAT engine.

Forward runs the R-only enumeration; backward re-runs the enumeration with
the fused R + dR/dp kernel instead of storing any state (R is affine in every
p_k, so the gradient is exact, not a finite difference).  PyTorch is only
used here for tensors and the current CUDA stream.
"""
from __future__ import annotations

import torch

from . import reliability


def _stream_of(t: torch.Tensor) -> int:
    if t.is_cuda:
        return torch.cuda.current_stream(t.device).cuda_stream
    return 0


class PBATReliability(torch.autograd.Function):
    """R = PBATReliability.apply(p, network[, opts]); p is a float64 tensor
    of arc reliabilities in input arc order."""

    @staticmethod
    def forward(ctx, p: torch.Tensor, network, opts=None):
        pc = p.detach().to("cpu", torch.float64).contiguous().numpy()
        res = reliability(network.n, network.tail, network.head, pc, network.source,
                          network.sink, network.directed, grad=False, opts=opts,
                          stream=_stream_of(p))
        ctx.network = network
        ctx.opts = opts
        ctx.save_for_backward(p)
        return torch.tensor(res.R, dtype=torch.float64, device=p.device)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (p,) = ctx.saved_tensors
        net = ctx.network
        pc = p.detach().to("cpu", torch.float64).contiguous().numpy()
        res = reliability(net.n, net.tail, net.head, pc, net.source, net.sink, net.directed,
                          grad=True, opts=ctx.opts, stream=_stream_of(p))
        g = torch.from_numpy(res.grad).to(device=p.device, dtype=p.dtype)
        return grad_out * g, None, None


def reliability_torch(p: torch.Tensor, network, opts=None) -> torch.Tensor:
    return PBATReliability.apply(p, network, opts)
