"""Pins of the double-float arithmetic the FP64 residual runs in
(paper_2301_05985_gb300/csrc/df32.cuh), on the host: sums, products and fused
multiply-adds of random pairs of floats, including sums that cancel almost completely,
against exact rational arithmetic.  The error bounds are those of the published
double-word algorithms (a few 2^-48 relative; the sum is exact when the hi parts cancel
exactly)."""
import os
import random
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("df") / "df_host_check")
    cmd = [nvcc, "-O2", "-std=c++17", "-Xcompiler", "-ffp-contract=off",
           "-I", os.path.join(ROOT, "paper_2301_05985_gb300", "csrc"),
           os.path.join(ROOT, "tests", "df_host_check.cu"), "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _df(rng, scale):
    """A normalised double-float: hi a float, lo below half an ulp of hi."""
    x = rng.uniform(-1.0, 1.0) * scale
    hi = np.float32(x)
    lo = np.float32((x - float(hi)) * rng.uniform(0.0, 1.0))
    hi2 = np.float32(float(hi) + float(lo))
    return hi2, np.float32(float(hi) + float(lo) - float(hi2))


def _exact(h, l):
    return Fraction(float(h)) + Fraction(float(l))


def test_double_float_operations_against_exact_arithmetic(driver):
    rng = random.Random(12345)
    cases = []
    for i in range(3000):
        sa, sb = 10.0 ** rng.uniform(-6, 6), 10.0 ** rng.uniform(-6, 6)
        a, b, c = _df(rng, sa), _df(rng, sb), _df(rng, sa * sb)
        if i % 5 == 0:  # b close to -a: the sum cancels
            b = (np.float32(-float(a[0]) * (1 + rng.uniform(-1e-6, 1e-6))), np.float32(rng.uniform(-1, 1) * 1e-9 * sa))
        cases.append((a, b, c))
    text = "\n".join(" ".join(float(x).hex() for pair in cs for x in pair) for cs in cases) + "\n"
    out = subprocess.run([driver], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    u2 = Fraction(1, 2 ** 48)
    worst = [0.0, 0.0, 0.0]
    for (a, b, c), line in zip(cases, out):
        r = [float.fromhex(t) for t in line.split()]
        A, B, Cc = _exact(*a), _exact(*b), _exact(*c)
        for k, (exact, got) in enumerate([(A + B, _exact(r[0], r[1])), (A * B, _exact(r[2], r[3])),
                                          (A * B + Cc, _exact(r[4], r[5]))]):
            err = abs(got - exact)
            bound = [3 * u2 * abs(exact), 5 * u2 * abs(exact), 8 * u2 * (abs(A * B) + abs(Cc))][k]
            assert err <= bound, (k, a, b, c, float(err), float(exact))
            if exact != 0:
                worst[k] = max(worst[k], float(err / abs(exact)))
    assert len(out) >= len(cases)
    # far below FP32 (2^-24), near the double-float unit
    assert max(worst[:2]) < 2.0 ** -45
