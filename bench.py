#!/usr/bin/env python3
"""PBAT benchmark: states/s of exact two-terminal reliability on one GB300.

A step is one pass of the whole enumeration (prefix split, exact monotone
prune, Gray walk, connectivity of every state, exact accumulation of R,
N_k and dR/dp into 256-bit fixed-point results) over the 2^m states of the
workload, with the tables already resident on the device.  The headline
workload is the largest single network, 24 nodes and 40 arcs (2^40
states).  ``value`` is 2^m / device time of the fused R + N_k + dR/dp step
(CUDA events on the launch stream, L2 flushed by a 256 MiB write between
steps, outside the events).  ``r_only`` is the same for the R + N_k kernel,
``unpruned`` the fused kernel with the prune off, and ``plain_gpu_bat`` the
one-state-per-thread frontier kernel (the plain GPU BAT, R and fused).
``e2e`` times the public C-ABI call with host buffers (planning, table
build, host -> device and device -> host copies included).  ``configs``
holds the same figures for every other workload of the scope: the 8-node
and 3x6-grid networks, the directed 34-arc network, and the batched
workload of 64 networks x 16 p-vectors.  ``cpu_baseline`` is the oracle
timed on the host cores; ``cpu_paper_pbat`` the paper's own PBAT in C on
every host core (cpu_pbat/).

--impl reference times the CPU oracle (test infrastructure: plain brute
force, long double) on the host cores over a bounded sample of the same
workload and reports it in the same metric.

Multi-GPU: one process per GPU (torchrun); the path does not shard across
GPUs here, so every rank runs an independent replica and ``value`` is the
states of all replicas over the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "states/s (2^m/time) for R and R+∇R vs plain GPU BAT, rel err ≤1e-12"
WORKLOADS = {
    "random-undirected-n24-m40": synth.workload_random_24_40,
    "grid-3x6": synth.workload_grid_3x6,
    "random-undirected-n8-m16": synth.workload_small_random,
    "random-directed-n20-m34": synth.workload_directed_20_34,
}
# the largest single-network workload (2^40 states) is the headline; the
# others (and the batched workload) are reported as sub-records
DEFAULT_WORKLOAD = "random-undirected-n24-m40"
BATCHED = "batched-64x16"
CONFIG_ORDER = ["random-undirected-n8-m16", "grid-3x6", "random-directed-n20-m34", BATCHED,
                "random-undirected-n24-m40"]

# Launch shapes (walk arcs L, threads per block, prune mode, occupancy,
# launches) the bench pins per workload and kernel, from shape sweeps on
# GB300, so that the timed launches are the ones the instruction counts below
# were taken from (--autotune lets the autotuner choose instead).  prune 2 =
# prune-aware prefix arcs; launches 2 = the first launch resolves what the
# prune can and defers the items left to walk to the second.
SHAPES = {
    "random-undirected-n24-m40": {"fused": (9, 256, 2, 2, 2), "r_only": (9, 128, 2, 0, 1)},
    "random-directed-n20-m34": {"fused": (7, 192, 2, 0, 2), "r_only": (7, 128, 2, 0, 2)},
    "grid-3x6": {"fused": (5, 128, 1, 0, 1), "r_only": (5, 64, 1, 0, 1)},
}

# Per generated kernel source (first 16 hex digits of its SHA-256, as
# pbat_kernel_source returns it): warp instructions executed per state
# (smsp__inst_executed.sum of one launch / 2^m) -- the per-unit figure of the
# issue-rate roofline -- and DRAM bytes per launch (dram__bytes_read.sum +
# dram__bytes_write.sum), from one ncu capture of that launch (bench.py
# --probe with the same workload and shape; summaries in profiles/).  A
# kernel whose source has changed since has no entry, and its roofline
# fraction is reported as null.
COUNTS = {
    # 24 nodes, 40 arcs: fused (L 9, 256 threads, prune 2, occupancy 2, its two launches
    # summed) and R-only (L 9, 128, 2, 0, one launch; four walk arcs unrolled)
    "b080d3e5392bd6e0": (12414443516 / 2**40, 1675264, "profiles/bs_kernel_grad_undirected24x40.md"),
    "0871ac197eac0d1d": (5902219352 / 2**40, 77568, "profiles/bs_kernel_undirected24x40.md"),
    # directed, 20 nodes, 34 arcs: fused (7, 192, 2, 0, two launches) and R-only
    # (7, 128, 2, 0, two launches)
    "8dff10689adf9178": (22081741 / 2**34, 98304, "profiles/bs_kernel_grad_directed20x34.md"),
    "fc32829a911d714a": (16006400 / 2**34, 74752, "profiles/bs_kernel_directed20x34.md"),
    # 3x6 grid: fused (5, 128, 1, 0, 1) and R-only (5, 64, 1, 0, 1)
    "23c0191c742fbc75": (15952825 / 2**27, 91904, "profiles/bs_kernel_grad_grid3x6.md"),
    "96d74f15c7df157a": (8078163 / 2**27, 51456, "profiles/bs_kernel_grid3x6.md"),
}

SM_COUNT = 152
ISSUE_PER_SM_CLK = 4          # warp instructions per clock per SM (4 schedulers)
SM_MAX_MHZ = 2070.0


def shape_opts(pb, workload: str, kind: str, **extra):
    """pbat_options of the pinned shape (the defaults if none is pinned)."""
    sh = SHAPES.get(workload, {}).get(kind)
    if sh is None:
        return pb.options(**extra)
    kw = dict(walk_bits=sh[0], block_threads=sh[1], prune=sh[2], occupancy=sh[3], launches=sh[4])
    kw.update(extra)
    return pb.options(**kw)


def source_key(pb, net, opts, grad: bool) -> str:
    """Hash of the generated kernel source a plan with these options runs."""
    src = pb.kernel_source(net, opts, grad=grad, p=net.p)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def workload_config(name: str, net, ws: int, l2: str) -> dict:
    """The workload as both arms name it in their JSON lines."""
    return {"workload": name, "n": net.n, "m": net.m, "states": 2**net.m,
            "outputs": "R, N_k, dR/dp", "directed": bool(net.directed),
            "parallelism": f"replicas x{ws}", "l2": l2}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def _oracle_division(args):
    name, bits, div, grad = args
    import oracle
    net = WORKLOADS[name]()
    t0 = time.perf_counter()
    oracle.enumerate_states(net, prefix_bits=bits, prefix_lo=div, prefix_hi=div + 1, grad=grad)
    return time.perf_counter() - t0


def oracle_rate(name: str, target_s: float, pool, cores: int, grad: bool = True):
    """States/s of the oracle on this host: calibrate one division, then run
    enough evenly spread divisions on every core to fill ~target_s."""
    net = WORKLOADS[name]()
    m = net.m
    sub = min(m, 12)                 # states per division: 2^sub
    bits = m - sub
    # calibrate with one division per process, all processes busy at once
    t0 = time.perf_counter()
    pool.map(_oracle_division, [(name, bits, (i * 7919) % (1 << bits), grad) for i in range(cores)])
    per = max(time.perf_counter() - t0, 1e-4)
    n_div = max(cores, int(target_s * cores / per))
    n_div = min(n_div, 1 << bits)
    step = max(1, (1 << bits) // n_div)
    divs = [(i * step) % (1 << bits) for i in range(n_div)]
    t0 = time.perf_counter()
    pool.map(_oracle_division, [(name, bits, d, grad) for d in divs])
    wall = time.perf_counter() - t0
    states = n_div * (1 << sub)
    return states / wall, dict(states=states, divisions=n_div, division_states=1 << sub,
                               wall_s=wall)


def run_reference(a):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    name = a.workload
    net = WORKLOADS[name]()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        for _ in range(a.warmup):
            oracle_rate(name, 1.0, pool, cores)
        rates, walls, samples = [], [], []
        for _ in range(a.steps):
            r, info = oracle_rate(name, a.ref_seconds, pool, cores)
            rates.append(r)
            walls.append(info["wall_s"])
            samples.append(info)
    value = statistics.median(rates)
    s0 = samples[0]
    sample = (f"{s0['divisions']} equal divisions of {s0['division_states']} states "
              f"(R, N_k, T1/T0 gradient) of {name}, spread over the 2^{net.m} space, "
              f"extrapolated as states/s")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "states/s",
        "n_gpus": 0, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1000.0 * statistics.mean(walls), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f80/f128 long double",
        "data": "synthetic",
        "config": workload_config(name, net, 1, "not applicable: host oracle"),
        "cpu_baseline": {"value": value, "unit": "states/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "states/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU path
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.t0 = self.t1 = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), max=float(f[2]), hw=f[5], hwt=f[6], swt=f[7],
                                 pcap=f[8]))
            except ValueError:
                continue
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, label in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                               ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(label)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["max"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows)}


def _time_plan(plan, steps, warmup, stream, flush, barrier):
    """Mean step time (CUDA events on the launch stream, L2 flushed between
    steps outside the events), the plan's own kernel time per launch, the
    wall time of the timed loop, and the last result."""
    import torch
    sp = stream.cuda_stream
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            plan.execute(sp)
        plan.read(sp)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            plan.execute(sp)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        barrier()
        res = plan.read(sp)
    step_ms = [s.elapsed_time(e) for s, e in ev]
    kern_ms = res.stats[4] / 1e6 / max(1, res.stats[7])
    return statistics.mean(step_ms), kern_ms, wall, res


def _peak():
    return SM_COUNT * ISSUE_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e9  # G warp-inst/s


def _roofline(kernel, key, states, kern_ms):
    """Issue-rate roofline of one kernel launch from its ncu counts."""
    cnt = COUNTS.get(key)
    ipc = cnt[0] if cnt else None
    achieved = ipc * states / (kern_ms / 1e3) / 1e9 if ipc is not None else None
    return {"bound": "alu", "achieved": achieved, "peak": _peak(), "unit": "Gwarp-inst/s",
            "frac": achieved / _peak() if achieved is not None else None,
            "traffic": cnt[1] if cnt else None, "kernel": kernel, "kernel_ms": kern_ms,
            "source_key": key, "counts_from": cnt[2] if cnt else "no capture of this source",
            "peak_source": "4 warp-inst/clk/SM x 152 SMs x 2070 MHz (derived)"}


def _single_record(pb, name, steps, warmup, stream, flush, barrier, ws):
    """Fused and R-only kernels of one network at its pinned shapes."""
    net = WORKLOADS[name]()
    states = 2**net.m
    rec = {"workload": name, "n": net.n, "m": net.m, "directed": bool(net.directed),
           "states": states}
    out = {}
    for kind, grad, kernel in (("fused", True, "bs_kernel_grad"), ("r_only", False, "bs_kernel")):
        opts = shape_opts(pb, name, kind)
        key = source_key(pb, net, opts, grad)
        plan = pb.Plan(net, grad=grad, opts=opts, stream=stream.cuda_stream)
        ms, kern, _, res = _time_plan(plan, steps, warmup, stream, flush, barrier)
        out[kind] = res
        rec[kind] = {"value": ws * states / (ms / 1e3), "ms_per_step": ms, "kernel_ms": kern,
                     "shape": dict(plan.describe(), prune=opts.prune, occupancy=opts.occupancy,
                                   launches=opts.launches),
                     "walked_fraction": res.stats[0] / states,
                     "roofline": _roofline(kernel, key, states, kern)}
        plan.close()
    assert out["fused"].Nk == out["r_only"].Nk, f"{name}: kernels disagree on N_k"
    rec["fused_over_r_only_time"] = rec["fused"]["ms_per_step"] / rec["r_only"]["ms_per_step"]
    rec["R"] = out["fused"].R
    return rec


def _batched_record(pb, steps, warmup, stream, ws):
    """The batched workload: 64 networks x 16 p-vectors through
    pbat_reliability_batched (one persistent launch replayed from a CUDA
    graph).  Device time from the library's events around the graph launch;
    the call time includes tables, upload and read-back."""
    import torch
    nets, pvecs = synth.workload_batched()
    K = len(pvecs[0])
    states = sum(2**n.m for n in nets)

    def timed(grad):
        o = pb.options()
        dev_ms, call_ms = [], []
        for i in range(warmup + steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            R, Nk, G = pb.reliability_batched(nets, pvecs, grad=grad, opts=o,
                                              stream=stream.cuda_stream)
            t1 = time.perf_counter()
            if i >= warmup:
                dev_ms.append(o.stats[4] / 1e6)
                call_ms.append(1e3 * (t1 - t0))
        return statistics.mean(dev_ms), statistics.mean(call_ms), R, Nk, int(o.stats[5])

    ms, call, R, Nk, launches = timed(False)
    gms, gcall, GR, GNk, glaunches = timed(True)
    assert GNk == Nk, "the gradient module disagrees with the R module on N_k"
    return {"workload": BATCHED, "networks": len(nets), "p_vectors": K, "states": states,
            "outputs": "R per (network, p-vector), N_k per network",
            "value": ws * states / (ms / 1e3), "pairs_per_s": ws * states * K / (ms / 1e3),
            "ms_per_step": ms, "call_ms": call, "launches": launches,
            "kernel": "bs_batch (one persistent launch, CUDA graph replay)", "R00": float(R[0][0]),
            "fused": {"value": ws * states / (gms / 1e3), "pairs_per_s": ws * states * K / (gms / 1e3),
                      "ms_per_step": gms, "call_ms": gcall, "launches": glaunches,
                      "outputs": "R, N_k and dR/dp per (network, p-vector)",
                      "kernel": "bs_batch_grad (one persistent launch, CUDA graph replay)"},
            "fused_over_r_only_time": gms / ms}


def run_ours(a):
    import torch
    ws, rank, local = _dist()
    cores = os.cpu_count() or 1
    pool = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        # the oracle's process pool is started before the first GPU call
        pool = mp.get_context("spawn").Pool(cores)
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2209_09711_gb300 import build
    build.build()
    import paper_2209_09711_gb300 as pb

    name = a.workload
    net = WORKLOADS[name]()
    m = net.m
    states = 2**m
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    sp = stream.cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    sampler = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                           if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit()
                           else local)

    def opts_for(kind, **extra):
        if a.autotune:
            return pb.options(**extra)
        o = shape_opts(pb, name, kind, **extra)
        if kind == "fused" and a.walk_bits is not None:
            o.walk_bits = a.walk_bits
        if kind == "fused" and a.block_threads is not None:
            o.block_threads = a.block_threads
        return o

    f_opts = opts_for("fused")
    fused = pb.Plan(net, grad=True, opts=f_opts, stream=sp)
    ms_f, kern_f, wall_f, res_f = _time_plan(fused, a.steps, a.warmup, stream, flush, barrier)
    clocks = sampler.stop()
    # the same fused kernel with the monotone prune off: every state walked
    nopr = pb.Plan(net, grad=True, opts=opts_for("fused", prune=0), stream=sp)
    ms_np, kern_np, _, res_np = _time_plan(nopr, max(3, a.steps // 10), min(a.warmup, 3), stream,
                                           flush, barrier)
    r_opts = opts_for("r_only")
    ronly = pb.Plan(net, grad=False, opts=r_opts, stream=sp)
    ms_r, kern_r, _, res_r = _time_plan(ronly, a.steps, a.warmup, stream, flush, barrier)
    # the plain GPU BAT: one state per thread, per-state PLSA frontier
    # expansion; above 2^34 states it runs on the first of 2^(m-34) equal
    # divisions (same per-state work) so that the bench stays within minutes
    plain_rb = max(0, m - 34)
    popt = dict(algo=pb.ALGO_FRONTIER, range_bits=plain_rb, range_lo=0, range_hi=1) if plain_rb \
        else dict(algo=pb.ALGO_FRONTIER)
    plain_states = states >> plain_rb
    plain = pb.Plan(net, grad=False, opts=pb.options(**popt), stream=sp)
    ms_p, _, _, res_p = _time_plan(plain, max(3, a.steps // 10), min(a.warmup, 3), stream, flush,
                                   barrier)
    plain_g = pb.Plan(net, grad=True, opts=pb.options(**popt), stream=sp)
    ms_pg, _, _, res_pg = _time_plan(plain_g, max(3, a.steps // 10), min(a.warmup, 3), stream,
                                     flush, barrier)
    assert res_r.Nk == res_f.Nk == res_np.Nk, "kernels disagree on N_k"
    if not plain_rb:
        assert res_r.Nk == res_p.Nk == res_pg.Nk, "kernels disagree on N_k"

    # e2e: the public call with host buffers, default options (the first
    # warm-up call runs the autotuner), copies included
    e2e_t = []
    o = pb.options()
    n_e2e = min(a.steps, 10)
    for i in range(a.warmup + n_e2e):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = pb.reliability_net(net, grad=True, opts=o, stream=sp)
        t1 = time.perf_counter()
        if i >= a.warmup:
            e2e_t.append(t1 - t0)
    e2e_s = statistics.mean(e2e_t)
    assert r.Nk == res_f.Nk, "the public call disagrees with the timed plan on N_k"

    # every other workload of the scope, at its pinned shapes
    configs = []
    if not a.no_configs:
        for cname in CONFIG_ORDER:
            if cname == name:
                continue
            if cname == BATCHED:
                configs.append(_batched_record(pb, min(a.steps, 10), min(a.warmup, 3), stream, ws))
            else:
                configs.append(_single_record(pb, cname, min(a.steps, 20), min(a.warmup, 3), stream,
                                              flush, barrier, ws))

    if ws > 1:
        t = torch.tensor([ms_f, ms_r, e2e_s, ms_p, ms_pg], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_f, ms_r, e2e_s, ms_p, ms_pg = t.tolist()

    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0

    cpu = cpu_paper = None
    if pool is not None:
        rate, info = oracle_rate(name, a.cpu_seconds, pool, cores)
        pool.close()
        cpu = {"value": rate, "unit": "states/s", "cores": cores, "kind": "oracle",
               "sample": f"{info['divisions']} equal divisions x {info['division_states']} states "
                         f"(R, N_k, T1/T0 gradient), {info['wall_s']:.1f} s wall on {cores} host "
                         f"processes, extrapolated to states/s"}
        import cpu_pbat
        prate, pinfo = cpu_pbat.rate(net, a.cpu_seconds, cores, grad=True)
        cpu_paper = {"value": prate, "unit": "states/s", "cores": cores, "kind": "pbat-cpu",
                     "what": "the paper's PBAT (Sec. 5.1): equal divisions on POSIX threads, "
                             "binary-addition order, PLSA test, FP64 Kahan sums; R, N_k and "
                             "T1/T0 per arc",
                     "cpu": _cpu_model(),
                     "sample": f"{pinfo['divisions']} evenly spread equal divisions x "
                               f"{pinfo['division_states']} states, {pinfo['wall_s']:.1f} s wall on "
                               f"{cores} threads, extrapolated to states/s"}

    roof = _roofline("bs_kernel_grad", source_key(pb, net, f_opts, True), states, kern_f)
    value = ws * states / (ms_f / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "states/s", "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_f, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u128", "data": "synthetic",
        "config": workload_config(name, net, ws,
                                  "flushed between steps (256 MiB write, outside the timed events)"),
        "roofline": roof,
        "fused_shape": dict(fused.describe(), prune=f_opts.prune, occupancy=f_opts.occupancy,
                            launches=f_opts.launches),
        "unpruned": {"value": ws * states / (ms_np / 1e3), "ms_per_step": ms_np, "kernel_ms": kern_np,
                     "what": "the fused kernel with the monotone prune off (every state walked)"},
        "r_only": {"value": ws * states / (ms_r / 1e3), "ms_per_step": ms_r, "kernel_ms": kern_r,
                   "kernel": "bs_kernel",
                   "shape": dict(ronly.describe(), prune=r_opts.prune, occupancy=r_opts.occupancy,
                                 launches=r_opts.launches),
                   "roofline": _roofline("bs_kernel", source_key(pb, net, r_opts, False), states,
                                         kern_r)},
        "plain_gpu_bat": {"value": ws * plain_states / (ms_p / 1e3), "ms_per_step": ms_p,
                          "kernel": "frontier_kernel (one state per thread, PLSA frontier)",
                          "states": plain_states,
                          "fused_value": ws * plain_states / (ms_pg / 1e3), "fused_ms_per_step": ms_pg},
        "fused_over_r_only_time": ms_f / ms_r,
        "speedup_over_plain_gpu_bat": {"R": (ms_p / plain_states) / (ms_r / states),
                                       "R+grad": (ms_pg / plain_states) / (ms_f / states)},
        "R": res_f.R, "pruned_states": res_f.stats[1], "walked_states": res_f.stats[0],
        "configs": configs,
        "cpu_baseline": cpu,
        "cpu_paper_pbat": cpu_paper,
        "e2e": {"value": ws * states / e2e_s, "unit": "states/s",
                "h2d_bytes_per_step": int(r.stats[2]), "d2h_bytes_per_step": int(r.stats[3]),
                "steps": n_e2e, "call": "pbat_reliability_grad, default options (autotuned)"},
        "gpu_launches": int(res_f.stats[5]),
        "clocks": clocks,
        "wall_s_timed": wall_f,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    for pl in (fused, nopr, ronly, plain, plain_g):
        pl.close()
    return 0


def run_shard(a):
    """One enumeration split across the ranks by equal divisions (Sec. 4.3,
    Eq. 6): each rank runs its contiguous block of divisions through the
    fused kernel at the workload's pinned shape, then one sum-reduce of the
    1 + m doubles (R, dR/dp) and the m + 1 int64 counts (N_k) over NCCL
    (PBAT STEP 3) gives every rank the whole result.  "scaling": "strong"
    (the total work is fixed); value = 2^m / the slowest rank's step."""
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2209_09711_gb300 import build
    build.build()
    import paper_2209_09711_gb300 as pb
    from paper_2209_09711_gb300 import shard
    name = a.workload
    net = WORKLOADS[name]()
    states = 2**net.m
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    bits, lo, hi = shard.shard_range(net.m, ws, rank)
    opts = shape_opts(pb, name, "fused", range_bits=bits, range_lo=lo, range_hi=hi)
    plan = pb.Plan(net, grad=True, opts=opts, stream=stream.cuda_stream)
    ms, kern, wall, res = _time_plan(plan, a.steps, a.warmup, stream, flush, barrier)
    # the exchange: one sum-reduce of each vector
    reduce = shard.torch_all_reduce() if ws > 1 else (lambda v: v)
    fv, nv = shard.pack(res.R, res.Nk, list(res.grad))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fsum, nsum = reduce(fv), reduce(nv)
    ex_ms = 1e3 * (time.perf_counter() - t0)
    R, Nk, g = shard.unpack(fsum, nsum, True)
    if ws > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = t.item()
    plan.close()
    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": states / ((ms + ex_ms) / 1e3), "unit": "states/s", "n_gpus": ws,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms + ex_ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u128", "data": "synthetic",
        "config": dict(workload_config(name, net, ws, "flushed between steps (256 MiB write)"),
                       parallelism=f"equal-division shards x{ws} (range_bits {bits})"),
        "shard_kernel_ms": ms, "exchange_ms": ex_ms, "R": R, "N_m": Nk[-1],
        "exchange": "NCCL all-reduce of 1 + m float64 and m + 1 int64" if ws > 1 else "none (one rank)",
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def _cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def run_probe(a):
    """One untimed launch of one kernel: the program ncu captures."""
    import torch
    torch.cuda.set_device(0)
    from paper_2209_09711_gb300 import build
    build.build()
    import paper_2209_09711_gb300 as pb
    net = WORKLOADS[a.workload]() if a.workload in WORKLOADS else None
    if a.probe in ("batched", "batched-fused"):
        nets, pvecs = synth.workload_batched()
        t0 = time.perf_counter()
        o = pb.options(algo=pb.ALGO_BITSLICE)
        R, Nk, _ = pb.reliability_batched(nets, pvecs, grad=a.probe == "batched-fused", opts=o)
        print(json.dumps({"probe": a.probe, "networks": len(nets), "p_vectors": len(pvecs[0]),
                          "states": sum(2**n.m for n in nets), "R00": R[0][0],
                          "kernel_ms": o.stats[4] / 1e6, "first_call_s": time.perf_counter() - t0}))
        return 0
    algo = pb.ALGO_FRONTIER if a.probe.startswith("plain") else pb.ALGO_AUTO
    grad = a.probe.endswith("fused")
    kind = "fused" if grad else "r_only"
    if algo == pb.ALGO_AUTO and not a.autotune:
        o = shape_opts(pb, a.workload, kind)
    else:
        o = pb.options(algo=algo)
    if a.walk_bits is not None:
        o.walk_bits = a.walk_bits
    if a.block_threads is not None:
        o.block_threads = a.block_threads
    key = source_key(pb, net, o, grad) if algo == pb.ALGO_AUTO else None
    plan = pb.Plan(net, grad=grad, opts=o)
    plan.execute(0)
    r = plan.read(0)
    print(json.dumps({"probe": a.probe, "workload": a.workload, "R": r.R, "source_key": key,
                      "kernel_ms": r.stats[4] / 1e6, "items": r.stats[6], "walked": r.stats[0],
                      "states": 2**net.m,
                      "shape": dict(plan.describe(), prune=o.prune, occupancy=o.occupancy,
                                    launches=o.launches)}))
    plan.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="target wall time of each CPU baseline sample (oracle, paper's PBAT)")
    ap.add_argument("--ref-seconds", type=float, default=6.0,
                    help="target wall time of one --impl reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="time the headline workload only (no sub-records of the other workloads)")
    ap.add_argument("--probe", choices=["fused", "r-only", "plain-r-only", "plain-fused", "batched",
                                        "batched-fused"],
                    help="run one untimed launch of that kernel (for profiler captures)")
    ap.add_argument("--walk-bits", type=int, default=None,
                    help="pin the walk length L (default: the tuned shape of the workload)")
    ap.add_argument("--block-threads", type=int, default=None,
                    help="pin the block size (default: the tuned shape of the workload)")
    ap.add_argument("--autotune", action="store_true",
                    help="let the autotuner pick the launch shapes instead of the recorded ones")
    ap.add_argument("--shard", action="store_true",
                    help="split one enumeration across the ranks by equal divisions (strong "
                         "scaling) instead of running replicas")
    a = ap.parse_args()
    if a.probe:
        return run_probe(a)
    if a.shard and a.impl == "ours":
        return run_shard(a)
    if a.warmup < 0 or a.steps < 1:
        ap.error("need --steps >= 1 and --warmup >= 0")
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
