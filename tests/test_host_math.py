"""The engine's host arithmetic against exact rationals (CPU only).

The bit-sliced kernels sum exact integers; what turns their tables and
results into and out of that fixed point runs on the host: rounding of
reliabilities to fixed point (walk masses, scale 2^127), the integer
floating point of the prefix masses (m * 2^(-63 - e)), the 256-bit results
(scale 2^250) read back as double-double, the binomials of the prune's
closed-form N_k and the reciprocals of the walk-arc gradient finish.  A
small C++ probe (host_math_probe.cpp) calls those functions of
pbat_engine.h; every answer is compared here with exact Fraction
arithmetic.
"""
import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2209_09711_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")
PROBE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "host_math_probe.cpp")
CXX = os.environ.get("CXX", "g++")

pytestmark = pytest.mark.skipif(shutil.which(CXX) is None, reason="no C++ compiler")


def _bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _dbl(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b))[0]


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("hostmath") / "probe")
    subprocess.check_call([CXX, "-O2", "-std=c++17", "-I", INCLUDE, "-I", CSRC, "-o", exe, PROBE])

    def run(lines, n_out=None):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             timeout=120, check=True).stdout.split("\n")
        return [o.split() for o in out[:len(lines) if n_out is None else n_out]]
    return run


def _round_half_up(q: Fraction) -> int:
    return math.floor(q + Fraction(1, 2))


def test_scaled_round_is_exact_round_half_up(probe):
    rng = random.Random(20909711)
    cases = []
    for _ in range(3000):
        x = rng.random() * 2.0 ** rng.randint(-80, 0)
        if x == 0.0:
            continue
        e = rng.randint(0, 127)
        if Fraction(x) * 2 ** e >= 2 ** 127:
            continue
        cases.append((x, e))
    # ties, exact powers and the smallest magnitudes
    cases += [(0.5, 0), (1.5, 0), (2.5, 0), (0.75, 1), (1.0, 127), (2.0 ** -1074, 1100),
              (5e-324, 1074), (5e-324, 1073), (2.0 ** -60 * 3, 59)]
    out = probe([f"S {_bits(x):x} {e}" for x, e in cases])
    for (x, e), (hi, lo) in zip(cases, out):
        got = (int(hi, 16) << 64) | int(lo, 16)
        assert got == _round_half_up(Fraction(x) * 2 ** e), (x, e)


def test_fixed127_within_one_unit(probe):
    rng = random.Random(7)
    cases = [(1.0, 0.0), (0.0, 0.0), (0.5, 2.0 ** -60), (0.9, -(2.0 ** -57))]
    for _ in range(2000):
        hi = rng.random()
        lo = (rng.random() - 0.5) * math.ulp(hi) if hi > 0 else 0.0
        cases.append((hi, lo))
    out = probe([f"F {_bits(h):x} {_bits(l):x}" for h, l in cases])
    for (h, l), (rh, rl) in zip(cases, out):
        got = (int(rh, 16) << 64) | int(rl, 16)
        exact = (Fraction(h) + Fraction(l)) * 2 ** 127
        # two half-unit roundings (hi and lo apart)
        assert abs(got - exact) <= 1, (h, l)
    assert int(out[0][0], 16) == 1 << 63 and int(out[0][1], 16) == 0   # 1.0 -> 2^127


def test_integer_floating_point_masses(probe):
    rng = random.Random(11)
    cases = [(1.0, 0.0), (0.5, 0.0), (0.0, 0.0), (1.0, 2.0 ** -60), (1.0, -(2.0 ** -70)),
             (2.0 ** -1000, 0.0), (2.0, 0.0), (3.5, 0.0)]
    for _ in range(3000):
        hi = rng.random() * 2.0 ** rng.randint(-300, 0)
        if hi == 0.0:
            continue
        lo = (rng.random() - 0.5) * math.ulp(hi)
        cases.append((hi, lo))
    out = probe([f"M {_bits(h):x} {_bits(l):x}" for h, l in cases])
    for (h, l), (ms, es) in zip(cases, out):
        m, e = int(ms, 16), int(es)
        v = Fraction(h) + Fraction(l)
        if v == 0:
            assert m == 0
            continue
        assert 2 ** 63 <= m < 2 ** 64 and e >= 0, (h, l, m, e)
        if v >= 2:
            # e would be negative: held at exactly 1 (a product of
            # reliabilities never comes near 2)
            assert m == 2 ** 63 and e == 0
            continue
        got = Fraction(m, 2 ** (63 + e))
        # two roundings of half a unit of m's last place each
        assert abs(got - v) <= Fraction(1, 2 ** (63 + e)), (h, l)


def test_256_bit_results_as_double_double(probe):
    rng = random.Random(13)
    cases = [[0] * 8, [1] + [0] * 7, [0] * 7 + [1 << 32], [(1 << 64) - 1] * 8]
    for _ in range(2000):
        # limbs as the kernels leave them: 32-bit chunks plus carries in the
        # upper halves; magnitudes from tiny to 2^6 (R, and gradient sums)
        top = rng.randint(0, 7)
        limbs = [rng.getrandbits(rng.choice((32, 40, 63, 64))) if i <= top else 0 for i in range(8)]
        cases.append(limbs)
    out = probe(["L " + " ".join(f"{x:x}" for x in c) for c in cases])
    for limbs, (hs, ls) in zip(cases, out):
        exact = Fraction(sum(x << (32 * i) for i, x in enumerate(limbs)), 2 ** 250)
        got = Fraction(_dbl(int(hs, 16))) + Fraction(_dbl(int(ls, 16)))
        if exact == 0:
            assert got == 0
        else:
            assert abs(got - exact) <= exact * Fraction(1, 2 ** 100), limbs


def test_binomials_of_the_prune(probe):
    cases = [(n, k) for n in range(0, 64) for k in range(-1, n + 2)]
    out = probe([f"B {n} {k}" for n, k in cases])
    for (n, k), (v,) in zip(cases, out):
        assert int(v, 16) == (math.comb(n, k) if 0 <= k <= n else 0), (n, k)


def test_reciprocals_of_walk_reliabilities(probe):
    rng = random.Random(17)
    xs = [1.0, 0.5, 2.0 ** -20, 1.0 - 2.0 ** -20, 0.9, 0.1, 1.0 / 3.0]
    xs += [rng.uniform(2.0 ** -20, 1.0) for _ in range(2000)]
    out = probe([f"R {_bits(x):x}" for x in xs])
    for x, (hs, ls) in zip(xs, out):
        y = Fraction(_dbl(int(hs, 16))) + Fraction(_dbl(int(ls, 16)))
        assert abs(y * Fraction(x) - 1) <= Fraction(1, 2 ** 100), x


def test_product_tables_of_arc_reliabilities(probe):
    """Every pattern's mass over up to 8 arcs, within 2^-100 of the exact
    product of p and 1 - p (the doubles as given)."""
    rng = random.Random(19)
    for n in (0, 1, 3, 5, 8):
        p = [rng.choice([0.0, 1.0, 0.5, rng.random(), 1 - 2.0 ** -30]) for _ in range(n)]
        out = probe(["P %d %s" % (n, " ".join(f"{_bits(x):x}" for x in p))], n_out=1 << n)
        for v, (hs, ls) in enumerate(out):
            exact = Fraction(1)
            for i, x in enumerate(p):
                exact *= Fraction(x) if (v >> i) & 1 else 1 - Fraction(x)
            got = Fraction(_dbl(int(hs, 16))) + Fraction(_dbl(int(ls, 16)))
            assert abs(got - exact) <= Fraction(1, 2 ** 100) * max(exact, Fraction(1, 2 ** 900)), (n, v)


def test_byte_tables_of_subset_sums(probe):
    """Lane and thread tables: entry v of byte b is the mass of the patterns
    in v's set bits at scale 2^62, within half a unit plus the 2^-126
    roundings of the (at most 8) weights; weights past n_valid count as 0."""
    rng = random.Random(23)
    for n in (32, 17, 5, 1):
        w = []
        for _ in range(n):
            hi = rng.random() / 32
            w.append((hi, (rng.random() - 0.5) * math.ulp(hi)))
        out = probe(["T %d %s" % (n, " ".join(f"{_bits(h):x} {_bits(l):x}" for h, l in w))],
                    n_out=1024)
        vals = [int(x[0], 16) for x in out]
        for b in range(4):
            assert vals[b * 256] == 0
            for v in range(1, 256):
                exact = sum((Fraction(w[8 * b + i][0]) + Fraction(w[8 * b + i][1])
                             for i in range(8) if (v >> i) & 1 and 8 * b + i < n), Fraction(0))
                err = abs(Fraction(vals[b * 256 + v], 2 ** 62) - exact)
                assert err <= Fraction(1, 2 ** 63) + Fraction(8, 2 ** 127), (n, b, v)


def test_fixed_point_rounding_of_double_doubles(probe):
    rng = random.Random(29)
    cases = [(1.0, 0.0, 63), (0.5, 2.0 ** -70, 63), (0.0, 0.0, 62)]
    for _ in range(1000):
        hi = rng.random()
        cases.append((hi, (rng.random() - 0.5) * math.ulp(hi) if hi else 0.0, rng.choice((62, 63))))
    out = probe([f"X {_bits(h):x} {_bits(l):x} {sc}" for h, l, sc in cases])
    for (h, l, sc), (v,) in zip(cases, out):
        exact = (Fraction(h) + Fraction(l)) * 2 ** sc
        assert abs(int(v, 16) - exact) <= 1, (h, l, sc)
