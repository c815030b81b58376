#!/usr/bin/env python3
"""Write the stored expected values of full-size workloads, from the oracle only.

    python tests/golden/make_golden.py grid-3x6

runs the CPU oracle (oracle/: plain brute force over every arc state, Eq. 1
with the PLSA test of Sec. 3.2, long double) over the whole state space of
the workload, split into equal divisions (Sec. 4.3) on a process pool, and
writes R, N_k and the T1/T0 sums of every arc to tests/golden/<name>_full.txt.
Floating values are stored as exact hex (float.hex) hi/lo pairs of the
oracle's long double sums; partial sums of the divisions are added in
Python with exact rational arithmetic, so the stored value does not depend
on the pool's order.  Nothing here reads or runs the CUDA engine.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOADS = {"grid-3x6": synth.workload_grid_3x6,
             "random-directed-n20-m34": synth.workload_directed_20_34}
DIV_BITS = 10


def _division(args):
    name, d = args
    import oracle
    net = WORKLOADS[name]()
    r = oracle.enumerate_states(net, prefix_bits=DIV_BITS, prefix_lo=d, prefix_hi=d + 1, grad=True)
    return d, r.R_hilo, r.Nk, r.T1_hilo, r.T0_hilo


def _exact(pairs):
    return sum((Fraction(h) + Fraction(l) for h, l in pairs), Fraction(0))


def _hilo(x: Fraction):
    hi = float(x)
    lo = float(x - Fraction(hi))
    return hi, lo


def make(name: str) -> str:
    net = WORKLOADS[name]()
    m = net.m
    t0 = time.time()
    procs = int(os.environ.get("GOLDEN_PROCS", os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_division, [(name, d) for d in range(1 << DIV_BITS)], chunksize=4)
    R = _exact([p[1] for p in parts])
    Nk = [sum(p[2][k] for p in parts) for k in range(m + 1)]
    T1 = [_exact([p[3][i] for p in parts]) for i in range(m)]
    T0 = [_exact([p[4][i] for p in parts]) for i in range(m)]
    path = os.path.join(HERE, f"{name}_full.txt")
    with open(path, "w") as f:
        f.write(f"# {name}: the oracle over all 2^{m} arc states (Eq. 1, PLSA of Sec. 3.2),\n")
        f.write("# written by tests/golden/make_golden.py from oracle/ alone.\n")
        f.write(f"# n {net.n} m {m} source {net.source} sink {net.sink} "
                f"directed {int(net.directed)}\n")
        f.write("# R: hi lo (float.hex); NK: N_0 .. N_m; T1 / T0: arc, hi, lo (input arc order)\n")
        f.write("R {} {}\n".format(*(v.hex() for v in _hilo(R))))
        f.write("NK " + " ".join(str(v) for v in Nk) + "\n")
        for i in range(m):
            f.write("T1 {} {} {}\n".format(i, *(v.hex() for v in _hilo(T1[i]))))
            f.write("T0 {} {} {}\n".format(i, *(v.hex() for v in _hilo(T0[i]))))
    print(f"{path}: R = {float(R):.15f}, {time.time() - t0:.1f} s")
    return path


if __name__ == "__main__":
    for nm in (sys.argv[1:] or list(WORKLOADS)):
        make(nm)
