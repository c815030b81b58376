"""Mutation check of the oracle's pins.

Each case plants one plausible mistake in a copy of the oracle's C source
(a swapped factor, a dropped or kept term, a wrong bit index, an arc read
the wrong way, an off-by-one range), builds it with the host C compiler on
the CPU, and runs the pin suite (test_oracle_pins.py) against that build.
Every mutant must make at least one pin fail; the unmodified copy, built the
same way, must pass them all.  The oracle's own file is never modified.

Mistakes that change only rounding (for instance dropping the compensation
term of the long double sums) are not listed: they move results by far less
than the 1e-12 tolerance the pins use, so no pin can or should see them.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pbat_oracle.c")

# name -> (original text, planted mistake); each original occurs exactly once
MUTANTS = {
    # Eq. 1: a working arc contributes p, a failed one 1 - p
    "state factor p and 1-p swapped": (
        "w *= orc_arc_on(x, m, k) ? (long double)p[k] : 1.0L - (long double)p[k];",
        "w *= orc_arc_on(x, m, k) ? 1.0L - (long double)p[k] : (long double)p[k];"),
    # prod_{j != i} of the gradient terms keeps arc i's own factor
    "excluded factor kept": (
        "    if (k == skip) continue;\n",
        "\n"),
    # Sec. 4.2: arc a_k is bit m-k of the index (x_1 most significant)
    "bit order reversed": (
        "return (int)((x >> (m - 1 - k)) & 1u);",
        "return (int)((x >> k) & 1u);"),
    # Sec. 3.2 on a directed network: arcs work tail -> head only
    "directed arcs used both ways": (
        "if (!directed && inprev[v] && !seen[u]) {",
        "if (inprev[v] && !seen[u]) {"),
    # ... and an undirected arc works both ways
    "undirected arcs used one way": (
        "if (!directed && inprev[v] && !seen[u]) {",
        "if (0 && inprev[v] && !seen[u]) {"),
    # arcs read head -> tail
    "arc direction reversed": (
        "if (inprev[u] && !seen[v]) {\n        seen[v] = 1;\n        nxt[nnxt++] = v;",
        "if (inprev[v] && !seen[u]) {\n        seen[u] = 1;\n        nxt[nnxt++] = u;"),
    # N_k indexes by the number of working arcs
    "N_k counts failed arcs": (
        "for (k = 0; k < m; ++k) c += orc_arc_on(x, m, k);",
        "for (k = 0; k < m; ++k) c += !orc_arc_on(x, m, k);"),
    # T1 collects x_i = 1, T0 collects x_i = 0
    "T1 and T0 exchanged": (
        "          orc_add(&T1[i], w);\n        else\n          orc_add(&T0[i], w);",
        "          orc_add(&T0[i], w);\n        else\n          orc_add(&T1[i], w);"),
    # critical state: X connected and X - e_i disconnected
    "critical test on X + e_i": (
        "if (orc_plsa(n, m, tail, head, directed, source, sink, x & ~bit, NULL)) continue;",
        "if (orc_plsa(n, m, tail, head, directed, source, sink, x | bit, NULL)) continue;"),
    "critical term keeps its own factor": (
        "orc_add(&G[i], orc_pr(m, p, x, i));",
        "orc_add(&G[i], orc_pr(m, p, x, -1));"),
    # Sec. 4.3 equal division: the range ends one state early
    "division end off by one": (
        "x1 = prefix_hi << (m - prefix_bits);",
        "x1 = (prefix_hi << (m - prefix_bits)) - 1;"),
    # Sec. 4.3 equal division: the range starts at the wrong state
    "division start shifted": (
        "x0 = prefix_lo << (m - prefix_bits);",
        "x0 = (prefix_lo << (m - prefix_bits)) >> 1;"),
    # Table 3: the layer a node is placed in
    "PLSA layer numbered from 0": (
        "for (i = 0; i < nnxt; ++i) layer_of[nxt[i]] = l;",
        "for (i = 0; i < nnxt; ++i) layer_of[nxt[i]] = l - 1;"),
    # Sec. 3.2 STEP P2/P3: a state whose sink is one layer away counted as cut
    "sink checked only among earlier layers": (
        "    if (seen[sink]) return 1;\n",
        "    if (seen[sink] && l > 2) return 1;\n"),
}


def _build(src_text, out_dir, tag):
    src = os.path.join(out_dir, f"oracle_{tag}.c")
    lib = os.path.join(out_dir, f"liboracle_{tag}.so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call([os.environ.get("CC", "gcc"), "-O2", "-std=c99", "-shared", "-fPIC",
                           "-o", lib, src])
    return lib


def _run_pins(lib):
    env = dict(os.environ, PBAT_ORACLE_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
           "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout + r.stderr


@pytest.mark.skipif(shutil.which(os.environ.get("CC", "gcc")) is None, reason="no C compiler")
def test_every_planted_mistake_fails_a_pin(tmp_path):
    base = open(SRC).read()
    builds = {"unmodified": _build(base, str(tmp_path), "unmodified")}
    for i, (name, (orig, bad)) in enumerate(MUTANTS.items()):
        assert base.count(orig) == 1, f"mutation site of '{name}' not found exactly once"
        builds[name] = _build(base.replace(orig, bad), str(tmp_path), f"m{i}")
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = dict(zip(builds, ex.map(_run_pins, builds.values())))
    rc, out = results.pop("unmodified")
    assert rc == 0, "the unmodified copy must pass every pin:\n" + out[-2000:]
    survivors = []
    for name, (rc, out) in results.items():
        # exit code 1 = tests ran and at least one failed (not a collection
        # or load error, which would say nothing about the pins)
        if rc != 1 or " failed" not in out:
            survivors.append(f"{name}: exit {rc}\n{out[-600:]}")
    assert not survivors, "mutants the pins did not catch:\n" + "\n".join(survivors)
