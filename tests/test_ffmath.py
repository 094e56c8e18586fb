"""The two-float helpers of the projection kernel (compensated camera transform and
perspective division), built for the host, against exact rational arithmetic."""
import ctypes
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def probe():
    d = tempfile.mkdtemp()
    so = os.path.join(d, "ff_probe.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                           "-I", os.path.join(ROOT, "paper_2607_02721_b300", "csrc"),
                           os.path.join(ROOT, "tests", "native", "ff_probe.cpp"), "-o", so])
    lib = ctypes.CDLL(so)
    P = ctypes.c_void_p
    lib.ff_dot3_plus.argtypes = [P, ctypes.c_float, P, P]
    lib.ff_persp.argtypes = [ctypes.c_float] * 6 + [P]
    return lib


def F(x):
    return Fraction(float(np.float32(x)))


def test_dot3_plus_is_accurate_to_two_floats(probe):
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(2000):
        r = rng.standard_normal(3).astype(np.float32)
        x = (rng.uniform(-4, 4, 3)).astype(np.float32)
        t = np.float32(rng.uniform(-15, 15))
        out = np.zeros(2, dtype=np.float32)
        probe.ff_dot3_plus(r.ctypes.data, t, x.ctypes.data, out.ctypes.data)
        exact = sum(F(r[k]) * F(x[k]) for k in range(3)) + F(t)
        got = F(out[0]) + F(out[1])
        scale = sum(abs(F(r[k]) * F(x[k])) for k in range(3)) + abs(F(t))
        worst = max(worst, float(abs(got - exact) / scale))
        # the high word is the correctly rounded value (or one ulp from it)
        assert abs(float(out[0]) - float(exact)) <= float(np.spacing(np.float32(abs(float(exact))))) + 1e-30
    assert worst < 2.0 ** -40


def test_perspective_mean_is_accurate_to_two_floats(probe):
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(2000):
        f = np.float32(rng.uniform(50, 2000))
        a_hi = np.float32(rng.uniform(-6, 6))
        a_lo = np.float32(float(a_hi) * rng.uniform(-2 ** -25, 2 ** -25))
        b_hi = np.float32(rng.uniform(1, 20))
        b_lo = np.float32(float(b_hi) * rng.uniform(-2 ** -25, 2 ** -25))
        c = np.float32(rng.uniform(0, 800))
        out = np.zeros(2, dtype=np.float32)
        probe.ff_persp(f, a_hi, a_lo, b_hi, b_lo, c, out.ctypes.data)
        exact = F(f) * (F(a_hi) + F(a_lo)) / (F(b_hi) + F(b_lo)) + F(c)
        got = F(out[0]) + F(out[1])
        mag = abs(F(f) * (F(a_hi) + F(a_lo)) / (F(b_hi) + F(b_lo))) + abs(F(c))
        worst = max(worst, float(abs(got - exact) / mag))
    assert worst < 2.0 ** -40
