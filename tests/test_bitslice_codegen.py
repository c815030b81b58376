"""The bit-sliced kernel's per-graph connectivity program, checked on the
CPU: the generated straight-line Boolean elimination (bs_inv then bs_var)
is evaluated in Python on 32-state words and compared, state by state, with
the oracle's PLSA connectivity.  Covers directed and undirected graphs,
parallel arcs, graphs smaller than a word, and the equal-division range."""
import re

import pytest

import oracle
import synth

LANE_PATTERNS = [0xAAAAAAAA, 0xCCCCCCCC, 0xF0F0F0F0, 0xFF00FF00, 0xFFFF0000]
FULL = 0xFFFFFFFF


@pytest.fixture(scope="module")
def pb():
    from paper_2209_09711_gb300 import build
    build.build()
    import paper_2209_09711_gb300 as mod
    return mod


def _parse(src):
    perm = [int(x) for x in src.splitlines()[0].split(":")[1].split()]
    defs = dict(re.findall(r"#define (BS_\w+) (\w+)", src))
    inv = src[src.index("void bs_inv"):]
    inv = inv[:inv.index("\n}\n")]
    var = src[src.index("u32 bs_var"):]
    var = var[:var.index("\n}\n")]
    return perm, {k: int(v.rstrip("u"), 0) for k, v in defs.items()}, inv, var


def _run(body, env):
    for line in body.splitlines()[1:]:
        line = line.strip()
        m = re.match(r"const u32 (v\d+) = (.*);$", line)
        if m:
            env[m.group(1)] = eval(m.group(2), {}, env) & FULL
            continue
        m = re.match(r"e\[(\d+)\] = (v\d+);$", line)
        if m:
            env["e"][int(m.group(1))] = env[m.group(2)]
            continue
        m = re.match(r"return (.*);$", line)
        if m:
            return eval(m.group(1).replace("0u", "0"), {}, env) & FULL
    return None


def _check(pb, net, seed, opts=None, trials=6):
    src = pb.kernel_source(net, opts)
    perm, D, inv, var = _parse(src)
    m, ell, tb, L, top = D["BS_M"], D["BS_ELL"], D["BS_TB"], D["BS_L"], D["BS_TOP"]
    rng = synth.SplitMix64(seed)
    for _ in range(trials):
        # a random assignment of every non-lane arc (internal positions)
        bits = [rng.below(2) for _ in range(m)]
        a = [0] * m
        for k in range(m):
            a[k] = LANE_PATTERNS[k] if k < ell else (FULL if bits[k] else 0)
        env = {"a": a, "e": [0] * max(1, D["BS_NCORE"])}
        _run(inv, env)
        w = [a[ell + tb + b] for b in range(L)]
        c = _run(var, {"e": env["e"], "w": w})
        for j in range(1 << ell):
            # the state: lane bits from j, others from `bits`; input arc order
            x = 0
            for k in range(m):
                on = ((j >> k) & 1) if k < ell else bits[k]
                if on:
                    x |= 1 << (m - 1 - perm[k])
            assert bool((c >> j) & 1) == oracle.connected(net, x), (net.name, j)


@pytest.mark.parametrize("directed", [False, True])
def test_generated_program_matches_oracle(pb, directed):
    for seed in range(25):
        rng = synth.SplitMix64(4242 + seed)
        n = 3 + rng.below(10)
        m = 1 + rng.below(30)
        net = synth.random_small(600 + seed, n=n, m=m, directed=directed)
        for walk in (-1, 0, 3):
            _check(pb, net, seed, pb.options(walk_bits=walk))


def test_generated_program_workloads(pb):
    for net in (synth.workload_grid_3x6(), synth.workload_directed_20_34(),
                synth.workload_random_24_40(), synth.workload_small_random(), synth.figure1()):
        _check(pb, net, 9, trials=4)
    net = synth.workload_random_24_40()
    _check(pb, net, 3, pb.options(range_bits=6, range_lo=5, range_hi=6), trials=3)
