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
    return perm, {k: int(v.rstrip("ul"), 0) for k, v in defs.items()}, inv, var


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


def test_plans_are_consistent_for_every_shape(pb):
    """Role assignment of the bit-sliced kernels: a permutation of the arcs,
    range arcs on top in input order, walk length within the free arcs --
    over sizes, ranges, walk requests and both kernels (a plan that broke
    these sent out-of-range arc indices to the device)."""
    checked = 0
    for seed in range(40):
        rng = synth.SplitMix64(31337 + seed)
        m = 1 + rng.below(63)
        n = 2 + rng.below(62)
        net = synth.random_small(12000 + seed, n=n, m=m, directed=bool(seed & 1))
        for grad in (False, True):
            for r in sorted({0, m // 2, max(0, m - 12), m}):
                if r and m - r < 0:
                    continue
                for walk in (-1, 0, 4, 10, 12):
                    o = pb.options(walk_bits=walk, range_bits=r, range_lo=0, range_hi=1 if r else 0)
                    src = pb.kernel_source(net, o, grad=grad)
                    perm, D, _, _ = _parse(src)
                    assert sorted(perm) == list(range(m)), (m, r, walk, grad)
                    assert all(perm[m - 1 - i] == i for i in range(r))
                    assert D["BS_D"] >= r and 0 <= D["BS_L"] <= 10
                    assert D["BS_ELL"] + D["BS_TB"] + D["BS_L"] + D["BS_D"] == m
                    checked += 1
    assert checked > 500


def test_generated_program_workloads(pb):
    for net in (synth.workload_grid_3x6(), synth.workload_directed_20_34(),
                synth.workload_random_24_40(), synth.workload_small_random(), synth.figure1()):
        _check(pb, net, 9, trials=4)
    net = synth.workload_random_24_40()
    _check(pb, net, 3, pb.options(range_bits=6, range_lo=5, range_hi=6), trials=3)


def _nvrtc_compile(src):
    import ctypes.util
    import os
    path = None
    for cand in ("/usr/local/cuda/lib64/libnvrtc.so", ctypes.util.find_library("nvrtc")):
        if cand and os.path.exists(cand):
            path = cand
            break
    if path is None:
        pytest.skip("NVRTC not found")
    import ctypes
    lib = ctypes.CDLL(path)
    prog = ctypes.c_void_p()
    lib.nvrtcCreateProgram(ctypes.byref(prog), src.encode(), b"gen.cu", 0, None, None)
    opts = (ctypes.c_char_p * 4)(b"-arch=sm_103a", b"-std=c++17", b"-lineinfo", b"-diag-suppress=177")
    rc = lib.nvrtcCompileProgram(prog, 4, opts)
    n = ctypes.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(max(1, n.value))
    lib.nvrtcGetProgramLog(prog, log)
    lib.nvrtcDestroyProgram(ctypes.byref(prog))
    errors = [l for l in log.value.decode(errors="replace").splitlines() if "error" in l]
    assert rc == 0, errors[:5]


def test_generated_sources_compile_with_nvrtc(pb):
    """Every kernel the engine generates at run time compiles for sm_103a
    (NVRTC runs on the CPU): R only, fused, and a batched module."""
    net = synth.workload_grid_3x6()
    for grad in (False, True):
        src = pb.kernel_source(net, grad=grad)
        _nvrtc_compile(src.split("\n", 1)[1])
    nets, _ = synth.workload_batched(6, 3)
    _nvrtc_compile(pb.batch_kernel_source(nets, 3))


def test_generated_source_holds_only_its_own_kernel(pb):
    """The R source carries no fused kernel and the fused source no R
    kernel, so a change to one kernel's template leaves the other's source
    (and the bench's instruction counts keyed by its hash) unchanged."""
    net = synth.workload_random_24_40()
    r_src = pb.kernel_source(net, grad=False)
    g_src = pb.kernel_source(net, grad=True)
    assert "bs_kernel_body" in r_src and "bs_kernel_grad_body" not in r_src
    assert "bs_kernel_grad_body" in g_src and "bs_kernel_body" not in g_src
    assert "extern \"C\" __global__ void KERNEL_BOUNDS bs_kernel(" in r_src
    assert "extern \"C\" __global__ void KERNEL_BOUNDS bs_kernel_grad(" in g_src


def test_every_template_variant_compiles_with_nvrtc(pb):
    """The generated source takes different template paths by shape: the
    fused kernel's accumulators in registers (short walks or small programs)
    or in global slots (long walks of large programs), two or three unrolled
    walk arcs (three or four in the R kernel), and with or without thread
    arcs.  Each combination compiles."""
    seen = set()
    cases = [(synth.workload_grid_3x6(), 5), (synth.workload_directed_20_34(), 10),
             (synth.workload_random_24_40(), 10), (synth.workload_random_24_40(), 4),
             (synth.random_small(31, n=5, m=7), 2)]
    for net, walk in cases:
        for grad in (False, True):
            src = pb.kernel_source(net, pb.options(walk_bits=walk), grad=grad)
            key = tuple(re.findall(r"#define (BS_GRAD|BS_ACC_REG|BS_IN_BITS|BS_TB) (\d+)", src))
            if key in seen:
                continue
            seen.add(key)
            _nvrtc_compile(src.split("\n", 1)[1])
    variants = {(dict(k)["BS_GRAD"], dict(k)["BS_ACC_REG"], dict(k)["BS_IN_BITS"]) for k in seen}
    assert ("1", "0", "2") in variants and ("1", "1", "3") in variants
    assert {v[2] for v in variants if v[0] == "0"} >= {"3", "4"}


@pytest.mark.parametrize("prune", [1, 2])
def test_batched_module_holds_each_network_program(pb, prune):
    """The batched module's per-network structs carry, in launch order
    (networks with the most work items first), exactly the connectivity
    programs emulated above for the single-network kernel with the batched
    walk length, and the plan constants that go with them."""
    nets, _ = synth.workload_batched(12, 2)
    bsrc = pb.batch_kernel_source(nets, 2, pb.options(prune=prune))
    singles = []
    for net in nets:
        src = pb.kernel_source(net, pb.options(walk_bits=5, block_threads=128, prune=prune))
        _, D, inv, var = _parse(src)
        singles.append((D, inv.split("\n", 1)[1], var.split("\n", 1)[1]))
    order = sorted(range(len(nets)), key=lambda i: -(1 << singles[i][0]["BS_D"]))
    for r, i in enumerate(order):
        start = bsrc.index(f"struct G{r} {{")
        body = bsrc[start:bsrc.index("\n};\n", start) + 1]   # ends with var's "}\n"
        consts = dict(re.findall(r"(\w+) = (\d+)", body.split("\n")[1]))
        D = singles[i][0]
        assert int(consts["M"]) == nets[i].m
        for key in ("ELL", "TB", "L", "D", "NCORE", "WALK0", "TOP"):
            assert int(consts[key]) == D["BS_" + key], (r, key)
        inv = body[body.index("void inv("):]
        inv = inv[:inv.index("\n}\n")].split("\n", 1)[1]
        var = body[body.index("u32 var("):]
        var = var[:var.index("\n}\n")].split("\n", 1)[1]
        assert inv and var
        assert inv == singles[i][1], r
        assert var == singles[i][2], r


@pytest.mark.parametrize("directed", [False, True])
def test_generated_program_at_maximum_sizes(pb, directed):
    """The generator at the ABI's limits: 63 arcs on 64 nodes and on 24
    nodes, seeded so that random states are a mix of connected and cut
    (roughly half connected), over the whole space, a deep equal-division range
    and the longest walk; the emulated program matches the oracle's
    connectivity, and the R and fused sources compile."""
    seeds = {False: (77000, 77000), True: (77028, 77002)}[directed]
    big = synth.random_small(seeds[0], n=64, m=63, directed=directed)
    mid = synth.random_small(seeds[1], n=24, m=63, directed=directed)
    for net in (big, mid):
        _check(pb, net, 5, trials=8)
        _check(pb, net, 6, pb.options(range_bits=40, range_lo=12345, range_hi=12346), trials=4)
        _check(pb, net, 7, pb.options(walk_bits=10), trials=4)
    _nvrtc_compile(pb.kernel_source(big, pb.options(walk_bits=10)))
    _nvrtc_compile(pb.kernel_source(mid, pb.options(walk_bits=10), grad=True))


# ---------------------------------------------------------------------------
# prune-aware prefix arcs (pbat_options.prune == 2)
# ---------------------------------------------------------------------------

def _prefix_arcs(src):
    perm, D, _, _ = _parse(src)
    return [perm[k] for k in range(D["BS_TOP"], D["BS_TOP"] + D["BS_D"])], D


def _resolved(net, prefix, values):
    """Items the monotone prune resolves (oracle connectivity): cut with
    every other arc working, or connected with every other arc failed."""
    m = net.m
    bit = {a: 1 << (m - 1 - a) for a in range(m)}
    rest = sum(bit[a] for a in range(m) if a not in prefix)
    n = 0
    for v in values:
        on = sum(bit[a] for j, a in enumerate(prefix) if (v >> j) & 1)
        if not oracle.connected(net, on | rest) or oracle.connected(net, on):
            n += 1
    return n


@pytest.mark.parametrize("grad", [False, True])
def test_prune_aware_prefix_resolves_more_items(pb, grad):
    """On the 34-arc directed network the default roles leave every small
    s-t cut partly among the walk arcs, so the prune resolves no item; the
    prune-aware prefix resolves most of them (counted exactly over all 2^14
    prefix values).  On the 40-arc network (sampled) and the 3x6 grid
    (exact) it resolves more than the default too."""
    import random
    for net, L, sample, floor in ((synth.workload_directed_20_34(), 10, None, 0.9),
                                  (synth.workload_random_24_40(), 10, 1024, 0.8),
                                  (synth.workload_grid_3x6(), 5, None, 0.6)):
        rates = {}
        for prune in (1, 2):
            src = pb.kernel_source(net, pb.options(walk_bits=L, prune=prune), grad=grad, p=net.p)
            pre, D = _prefix_arcs(src)
            vals = (range(1 << len(pre)) if sample is None
                    else random.Random(5).sample(range(1 << len(pre)), sample))
            rates[prune] = _resolved(net, pre, vals) / len(vals)
        assert rates[2] >= floor and rates[2] > rates[1], (net.name, rates)


def test_prune_aware_plans_are_exact_and_deterministic(pb):
    """Plans of the prune-aware mode: the emulated connectivity program
    matches the oracle, the role invariants hold (including a range and a
    gradient walk shortened by arcs with p at 0 or 1, whose extra prefix arcs
    come from the remaining ones), planning twice gives the same source, and
    the generated kernels compile."""
    for seed in range(8):
        rng = synth.SplitMix64(5150 + seed)
        net = synth.random_small(5200 + seed, n=4 + rng.below(12), m=12 + rng.below(30),
                                 directed=bool(seed & 1))
        for walk in (-1, 4, 10):
            _check(pb, net, seed, pb.options(walk_bits=walk, prune=2), trials=3)
    net = synth.workload_random_24_40()
    _check(pb, net, 2, pb.options(prune=2, range_bits=6, range_lo=5, range_hi=6), trials=3)
    # most arcs deterministic: too few eligible walk arcs for the fused plan
    p = [1.0 if k % 4 else 0.7 for k in range(net.m)]
    for r in (0, 6):
        o = pb.options(walk_bits=10, prune=2, range_bits=r, range_lo=0, range_hi=1 if r else 0)
        src = pb.kernel_source(net, o, grad=True, p=p)
        perm, D, _, _ = _parse(src)
        m = net.m
        assert sorted(perm) == list(range(m))
        assert all(perm[m - 1 - i] == i for i in range(r))
        walk = [perm[k] for k in range(D["BS_ELL"] + D["BS_TB"], D["BS_TOP"])]
        assert all(0 < p[a] < 1 for a in walk)
        assert D["BS_ELL"] + D["BS_TB"] + D["BS_L"] + D["BS_D"] == m
        assert D["BS_L"] < 10     # the shortened walk: extra prefix arcs were needed
        assert src == pb.kernel_source(net, o, grad=True, p=p)
    with pytest.raises(pb.PbatError):
        pb.kernel_source(net, pb.options(prune=3))
    # the mode's programs (walk cluster chosen for the fewest operations) compile
    for big in (synth.workload_random_24_40(), synth.workload_directed_20_34()):
        _nvrtc_compile(pb.kernel_source(big, pb.options(walk_bits=10, prune=2), grad=True, p=big.p))
        _nvrtc_compile(pb.kernel_source(big, pb.options(walk_bits=10, prune=2)))


def _walked_items_exact(net, prefix):
    """Items of a prefix that the prune leaves to walk, counted over every
    prefix value: 2^12 values at a time as the bits of Python integers
    (value i of a batch is bit i), reachability as a fixed point."""
    d, arcs = len(prefix), list(zip(net.tail, net.head))
    width = min(1 << 12, 1 << d)
    full = (1 << width) - 1

    def pattern(j, b):
        if j >= 12:
            return full if (b >> (j - 12)) & 1 else 0
        unit = ((1 << (1 << j)) - 1) << (1 << j)
        return sum(unit << s for s in range(0, width, 2 << j)) & full

    def reach(on):
        R = [0] * net.n
        R[net.source] = full
        grew = True
        while grew:
            grew = False
            for k, (u, v) in enumerate(arcs):
                for a, b in ((u, v), (v, u)) if not net.directed else ((u, v),):
                    nb = R[b] | (R[a] & on[k])
                    if nb != R[b]:
                        R[b], grew = nb, True
        return R[net.sink]

    pos = {a: j for j, a in enumerate(prefix)}
    walked = 0
    for b in range(max(1, (1 << d) >> 12)):
        up = [pattern(pos[k], b) if k in pos else full for k in range(net.m)]
        dn = [pattern(pos[k], b) if k in pos else 0 for k in range(net.m)]
        walked += bin(reach(up) & ~reach(dn) & full).count("1")
    return walked


def test_prune_aware_plan_resolves_the_whole_directed_network(pb):
    """Counted exactly: with the prune-aware prefix of 17 arcs (walk length
    7) the 34-arc directed network leaves no item to walk -- the prune alone
    decides all 2^34 states -- and at walk length 10 it leaves about 3%.
    The counter agrees with the oracle-based count on the grid."""
    net = synth.workload_directed_20_34()
    for L, most in ((7, 0), (10, 600)):
        src = pb.kernel_source(net, pb.options(walk_bits=L, prune=2), grad=True, p=net.p)
        pre, D = _prefix_arcs(src)
        assert D["BS_L"] == L
        assert _walked_items_exact(net, pre) <= most
    grid = synth.workload_grid_3x6()
    pre, _ = _prefix_arcs(pb.kernel_source(grid, pb.options(walk_bits=5, prune=2)))
    assert _walked_items_exact(grid, pre) == (1 << len(pre)) - _resolved(grid, pre, range(1 << len(pre)))


def test_batched_gradient_module_compiles_with_nvrtc(pb):
    """The batched gradient module (bs_batch_grad): every network's
    connectivity program and the kernel body, with walk arcs restricted to
    those whose p is inside [2^-20, 1 - 2^-20] under every p-vector."""
    nets, pvecs = synth.workload_batched(6, 3)
    src = pb.batch_grad_kernel_source(nets, pvecs)
    assert "bs_batch_grad(" in src and "bsb_finish_grad(" in src
    _nvrtc_compile(src)
    # an arc at p = 0 in one p-vector cannot be a walk arc of its network
    pv = [[list(v) for v in pvs] for pvs in pvecs]
    pv[0][1][0] = 0.0
    src0 = pb.batch_grad_kernel_source(nets, pv)
    _nvrtc_compile(src0)
