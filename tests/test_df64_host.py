"""The df64 arithmetic (float pairs) of the reciprocal-energy branch, built
for the host with the same algorithms, against exact rational arithmetic on
the same float-pair inputs: relative error of sums (also under cancellation),
products and quotients below 2^-44."""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def df64_lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("df64") / "libdf64_check.so")
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", out,
                           os.path.join(HERE, "df64_check.cpp"),
                           "-I", os.path.join(ROOT, "paper_2608_12691_b300", "csrc"),
                           "-I", "/usr/local/cuda/include"])
    lib = ctypes.CDLL(out)
    lib.df64_ops.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
    return lib


def ops(lib, a, b):
    out = np.zeros(12)
    lib.df64_ops(a, b, out.ctypes.data)
    val = [Fraction(float(out[2 * k])) + Fraction(float(out[2 * k + 1])) for k in range(6)]
    return val[:4], val[4], val[5]


def test_df64_operations_against_exact_arithmetic(df64_lib):
    rng = np.random.default_rng(4)
    bound = Fraction(1, 2 ** 44)
    for t in range(3000):
        a = rng.normal() * 10.0 ** rng.integers(-6, 7)
        b = rng.normal() * 10.0 ** rng.integers(-6, 7)
        if t % 5 == 0:
            b = -a * (1.0 + rng.normal() * 1e-6)        # cancellation in a + b
        (s, d, p, q), x, y = ops(df64_lib, a, b)
        # the inputs as float pairs carry about 48 bits of a and b
        assert abs(x - Fraction(a)) <= abs(Fraction(a)) * Fraction(1, 2 ** 46)
        exact = [x + y, x - y, x * y, x / y]
        for got, want in zip((s, d, p, q), exact):
            if want != 0:
                assert abs(got - want) <= abs(want) * bound, (a, b, float(got), float(want))
            else:
                assert got == 0
