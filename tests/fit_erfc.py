"""Least-squares fit used by the FP32 pair kernel for erfc.

erfc(x) = exp(-x^2) P(t),  t = 1 / (1 + p x),  P a degree-7 polynomial, fitted
here to minimise the relative error of erfc on 0 <= x <= 4.2 (the form of
Hastings' approximations, Abramowitz & Stegun 7.1.26, with more terms and our
own coefficients).  Prints p, the coefficients and the maximum relative error
in double precision.
"""
import numpy as np
from scipy.special import erfc

XMAX = 4.2
P = 0.345
DEG = 7


def fit(p=P, deg=DEG, xmax=XMAX, n=20001):
    x = np.linspace(0.0, xmax, n)
    f = erfc(x) * np.exp(x * x)
    t = 1.0 / (1.0 + p * x)
    V = np.vander(t, deg + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V / f[:, None], np.ones_like(f), rcond=None)
    rel = np.abs((V @ c) / f - 1.0).max()
    return c, rel


if __name__ == "__main__":
    c, rel = fit()
    print(f"p = {P}, max relative error {rel:.3e}")
    print(", ".join(f"{v:.17g}" for v in c))
