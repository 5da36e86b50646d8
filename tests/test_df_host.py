"""Double-float arithmetic of the integral kernels, checked on the host.

The kernels' double-float type (paper_1905_01381_gb300/csrc/cq_df.cuh: a
value is hi + lo, two FP32 numbers) is compiled into a small host program
(tests/df_host_check.cu) and every result is compared with exact rational
arithmetic (fractions.Fraction) on seeded operands spread over twelve
decades, with both signs and with near-cancelling sums:

* TwoSum is error-free: s + e equals a + b exactly, s = fl(a + b).
* Sum: error <= 2^-45 (|x| + |y|) -- the bound that matters for the sums of
  the recurrences, also under cancellation.
* Product: relative error <= 2^-45 (the double-word product ignores only
  lo*lo and two roundings of order u^2, u = 2^-24).
* Fused a*b + c: error <= 2^-45 (|a b| + |c|).
* Reciprocal: relative error <= 2^-44; square root: |r^2 / x - 1| <= 2^-43.
* Every result is normalised: |lo| <= ulp(hi) / 2.
"""
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1905_01381_gb300", "csrc")


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("df") / "df_host_check")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-ffp-contract=off", "-I", CSRC,
                        os.path.join(HERE, "df_host_check.cu"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def f32(x):
    return float(np.float32(x))


def bits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def unbits(u):
    return struct.unpack("<f", struct.pack("<I", u))[0]


def split(v):
    """Nearest double-float (hi, lo) of a double v."""
    hi = f32(v)
    return hi, f32(v - hi)


def value(p):
    return Fraction(p[0]) + Fraction(p[1])


def run(prog, cases):
    lines = "".join(f"{op} " + " ".join(f"{bits(x):08x}" for x in (*a, *b, *c)) + "\n" for op, a, b, c in cases)
    r = subprocess.run([prog], input=lines, capture_output=True, text=True, check=True)
    return [tuple(unbits(int(w, 16)) for w in ln.split()) for ln in r.stdout.splitlines()]


def operands(seed, n, positive=False):
    g = np.random.default_rng(seed)
    mag = 10.0 ** g.uniform(-6, 6, n)
    sign = np.ones(n) if positive else np.where(g.random(n) < 0.5, -1.0, 1.0)
    return [split(float(v)) for v in mag * sign * g.uniform(1, 2, n)]


def normalised(r):
    hi, lo = r
    return hi == 0.0 or abs(lo) <= abs(hi) * 2.0 ** -24


def test_two_sum_is_exact(prog):
    A, B = operands(1, 2000), operands(2, 2000)
    cases = [(0, a, b, (0.0, 0.0)) for a, b in zip(A, B)]
    for (op, a, b, _), r in zip(cases, run(prog, cases)):
        assert Fraction(r[0]) + Fraction(r[1]) == Fraction(a[0]) + Fraction(b[0])
        assert r[0] == f32(a[0] + b[0])


def test_sum(prog):
    A, B = operands(3, 2000), operands(4, 2000)
    # near-cancelling pairs: y = -x (1 + d), |d| down to 1e-9
    g = np.random.default_rng(5)
    C = [split(-float(value(a)) * (1 + float(d))) for a, d in zip(A, 10.0 ** g.uniform(-9, -1, 2000))]
    cases = [(1, a, b, (0.0, 0.0)) for a, b in zip(A, B)] + [(1, a, c, (0.0, 0.0)) for a, c in zip(A, C)]
    for (op, a, b, _), r in zip(cases, run(prog, cases)):
        x, y = value(a), value(b)
        assert abs(value(r) - (x + y)) <= Fraction(1, 2 ** 45) * (abs(x) + abs(y))
        assert normalised(r)


def test_product(prog):
    A, B = operands(6, 3000), operands(7, 3000)
    cases = [(2, a, b, (0.0, 0.0)) for a, b in zip(A, B)]
    for (op, a, b, _), r in zip(cases, run(prog, cases)):
        exact = value(a) * value(b)
        assert abs(value(r) - exact) <= Fraction(1, 2 ** 45) * abs(exact)
        assert normalised(r)


def test_fused_multiply_add(prog):
    A, B, C = operands(8, 3000), operands(9, 3000), operands(10, 3000)
    cases = [(3, a, b, c) for a, b, c in zip(A, B, C)]
    for (op, a, b, c), r in zip(cases, run(prog, cases)):
        ab, z = value(a) * value(b), value(c)
        assert abs(value(r) - (ab + z)) <= Fraction(1, 2 ** 45) * (abs(ab) + abs(z))
        assert normalised(r)


def test_reciprocal_and_square_root(prog):
    A = operands(11, 2000)
    P = operands(12, 2000, positive=True)
    cases = [(4, a, (0.0, 0.0), (0.0, 0.0)) for a in A] + [(5, p, (0.0, 0.0), (0.0, 0.0)) for p in P]
    out = run(prog, cases)
    for (op, a, _, _), r in zip(cases, out):
        x = value(a)
        if op == 4:
            assert abs(value(r) * x - 1) <= Fraction(1, 2 ** 44)
        else:
            assert abs(value(r) ** 2 / x - 1) <= Fraction(1, 2 ** 43)
        assert normalised(r)
