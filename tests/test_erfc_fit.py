"""The erfc approximation of the FP32 pair kernel (exp(-x^2) P(t), t = 1/(1 + p x),
P of degree 7): the coefficients compiled into the kernel are the least-squares
fit that fit_erfc.py reproduces, and the approximation meets its stated
relative error on [0, 4.2] in exact arithmetic and, evaluated by Horner's rule
in single precision, stays within a few float ulps of erfc."""
import os
import re

import numpy as np
from scipy.special import erfc

import fit_erfc

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2608_12691_b300", "csrc", "nonbonded.cu")


def kernel_coefficients():
    src = open(SRC).read()
    body = src[src.index("void erfc_exp(float x"):]
    body = body[:body.index("}")]
    p = float(re.search(r"fmaf\(([0-9.]+)f, x, 1\.0f\)", body).group(1))
    lead = float(re.search(r"float p = ([-0-9.e]+)f;", body).group(1))
    rest = [float(v) for v in re.findall(r"fmaf\(p, t, ([-0-9.e]+)f\)", body)]
    return p, np.array([lead] + rest)        # highest degree first


def test_kernel_coefficients_are_the_fit():
    p, c_hi_first = kernel_coefficients()
    assert p == fit_erfc.P and len(c_hi_first) == fit_erfc.DEG + 1
    c, rel = fit_erfc.fit()
    assert rel < 5e-8
    np.testing.assert_allclose(c_hi_first[::-1], c, rtol=1e-12, atol=0)


def test_approximation_error():
    p, c = kernel_coefficients()
    x = np.linspace(0.0, 4.2, 40001)
    # exact (double) evaluation of the fitted form
    t = 1.0 / (1.0 + p * x)
    approx = np.polyval(c, t) * np.exp(-x * x)
    assert np.max(np.abs(approx / erfc(x) - 1.0)) < 5e-8
    # single-precision Horner with the kernel's float coefficients (each fma
    # rounded once to float32) and the exact exponential
    x32 = x.astype(np.float32)
    t32 = (np.float32(1.0) / (np.float32(p) * x32 + np.float32(1.0))).astype(np.float32)
    acc = np.full_like(x32, np.float32(c[0]))
    for ck in c[1:]:
        acc = (acc.astype(np.float64) * t32 + np.float64(np.float32(ck))).astype(np.float32)
    y = acc.astype(np.float64) * np.exp(-x32.astype(np.float64) ** 2)
    rel = np.abs(y / erfc(x32.astype(np.float64)) - 1.0)
    assert rel.max() < 5e-7          # measured 3.6e-7, about six float ulps
