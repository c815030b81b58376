"""bench.py's reference arm (the CPU oracle timed on the host cores) prints
one JSON line with the keys the bench contract names; CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
         "--warmup", "0", "--ref-seconds", "0.5"],
        capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "states/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["data"] == "synthetic"
    cfg = d["config"]
    assert cfg["workload"] == "random-undirected-n24-m40" and cfg["m"] == 40 and cfg["states"] == 2**40
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_pinned_shapes_have_instruction_counts():
    """Every kernel the bench times at a pinned shape has an entry in
    bench.COUNTS under the hash of the source the library generates for it
    now, and the profile page named there exists and carries that hash: a
    kernel changed since its capture would otherwise report a null roofline
    fraction.  Source generation needs no GPU."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2209_09711_gb300 import build
    build.build()
    import paper_2209_09711_gb300 as pb
    for name, kinds in bench.SHAPES.items():
        net = bench.WORKLOADS[name]()
        for kind in kinds:
            key = bench.source_key(pb, net, bench.shape_opts(pb, name, kind), kind == "fused")
            assert key in bench.COUNTS, (name, kind, key)
            per_state, dram, page = bench.COUNTS[key]
            assert 0 < per_state < 1 and dram > 0
            with open(os.path.join(ROOT, page)) as f:
                assert key in f.read(), (page, key)
