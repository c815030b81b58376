"""Multi-process path on CPU: two gloo ranks split the equal divisions of
one network, each computes its block (here with the oracle standing in for
the per-rank GPU call), and one sum-reduce gives the whole R, N_k, dR/dp."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as tmp

import oracle
import synth
from paper_2209_09711_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _oracle_compute(net, bits, lo, hi, grad):
    r = oracle.enumerate_states(net, prefix_bits=bits, prefix_lo=lo, prefix_hi=hi, grad=grad)
    return r.R, r.Nk, (r.grad_t1t0 if grad else None)


class _Big:
    m = 63


_BIG_BASE = [3 ** 37 + 2 * k for k in range(64)]   # 3^37 > 2^58


def _big_compute(net, bits, lo, hi, grad):
    # a stand-in rank result: odd-sized counts that differ per block
    return 1e-3 * lo, [c + lo for c in _BIG_BASE], None


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = []
        for net in (synth.workload_small_random(), synth.figure1(True), synth.bridge([0.9] * 5)):
            R, Nk, g = shard.reliability_sharded(net, _oracle_compute, world, rank,
                                                 shard.torch_all_reduce(), grad=True)
            out.append((R, Nk, g))
        # counts above 2^53 (a 63-arc network's middle N_k reach C(63, 31)):
        # a float64 reduce would round them, the int64 one must not
        big = shard.reliability_sharded(_Big(), _big_compute, world, rank,
                                        shard.torch_all_reduce(), grad=False)
        q.put((rank, out, big))
    finally:
        dist.destroy_process_group()


def test_shard_ranges_cover_the_space():
    for m in (1, 5, 16, 40):
        for world in (1, 2, 3, 8):
            blocks = [shard.shard_range(m, world, r) for r in range(world)]
            bits = blocks[0][0]
            assert all(b[0] == bits for b in blocks)
            assert blocks[0][1] == 0 and blocks[-1][2] == 1 << bits
            assert all(blocks[i][2] == blocks[i + 1][1] for i in range(world - 1))


def test_two_gloo_ranks_match_the_whole():
    world = 2
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    results = {r: out for r, out, _ in got}
    bigs = {r: big for r, _, big in got}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    nets = (synth.workload_small_random(), synth.figure1(True), synth.bridge([0.9] * 5))
    for i, net in enumerate(nets):
        ref = oracle.enumerate_states(net, grad=True)
        for rank in range(world):
            R, Nk, g = results[rank][i]
            assert Nk == ref.Nk
            assert abs(R - ref.R) <= 1e-14
            assert max(abs(a - b) for a, b in zip(g, ref.grad_t1t0)) <= 1e-14
    blocks = [shard.shard_range(63, world, r)[1] for r in range(world)]
    want = [sum(c + lo for lo in blocks) for c in _BIG_BASE]
    assert max(want) > 2 ** 53
    for rank in range(world):
        R, Nk, g = bigs[rank]
        assert Nk == want
        assert g is None
