"""Pins of the oracle's thermodynamic-integration estimator (Eq. 2).

The binning and the quadrature are checked against integrals known in closed
form: a linear mean-force profile is integrated exactly, a smooth one to the
quadrature's O(1/n^2), and for frozen atoms the mean force is
h_A'(lambda) U_uv + h_B'(lambda) U_soft, whose integral over [0, 1] is
U_uv (h_A goes from 0 to 1, h_B starts and ends at 0, Eq. 7-8).
"""
import math

import numpy as np
import pytest

from oracle import dynamics as D
from oracle import reference as R
from paper_2608_12691_b300 import systems as S


def test_bins_and_end_points():
    ti = D.TIAccumulator(10)
    ti.add(0.0, 1.0)
    ti.add(0.0999, 3.0)
    ti.add(0.1, 5.0)
    ti.add(1.0, 7.0)        # lambda = 1 belongs to the last bin
    assert ti.count.tolist() == [2, 1, 0, 0, 0, 0, 0, 0, 0, 1]
    m = ti.means()
    assert m[0] == 2.0 and m[1] == 5.0 and m[9] == 7.0 and np.isnan(m[5])


def test_linear_profile_integrates_exactly():
    ti = D.TIAccumulator(100)
    a, b = -37.5, 12.25
    rng = np.random.default_rng(1)
    for _ in range(20000):
        lam = rng.uniform(0.0, 1.0)
        b_idx = min(99, int(lam * 100))
        centre = (b_idx + 0.5) / 100
        ti.add(lam, a + b * centre)
    assert ti.delta_g() == pytest.approx(a + 0.5 * b, rel=1e-12)
    # two occupied bins only: the line through them is integrated exactly
    ti2 = D.TIAccumulator(100)
    ti2.add(0.305, a + b * 0.305)
    ti2.add(0.715, a + b * 0.715)
    assert ti2.delta_g() == pytest.approx(a + 0.5 * b, rel=1e-12)


def test_smooth_profile_quadrature_error():
    # mean force cos(3 lambda) sampled at the bin centres: error O(1/n^2)
    for n in (50, 100, 200):
        ti = D.TIAccumulator(n)
        for b in range(n):
            lam = (b + 0.5) / n
            ti.add(lam, math.cos(3 * lam))
        err = abs(ti.delta_g() - math.sin(3.0) / 3.0)
        assert err < 2.0 / n ** 2


def test_frozen_atoms_integrate_to_U_uv():
    # positions fixed: dU/dlambda(lambda) = h_A' U_uv + h_B' U_soft, so the
    # estimator must return U_uv (up to its quadrature error)
    d = S.make_water_box(seed=21, n_waters=101, box_len=1.45, solute="ring12", n_side=5,
                         r_cut=0.7, grid=16)
    E, _, _, _ = R.nonbonded(d, level=2, forces=False)
    ti = D.TIAccumulator(100)
    rng = np.random.default_rng(3)
    for lam in rng.uniform(0.0, 1.0, size=40000):
        _, _, dA, dB = R.switching(lam)
        ti.add(lam, dA * E["U_uv"] + dB * E["U_soft"])
    scale = abs(E["U_uv"]) + abs(E["U_soft"])
    assert abs(ti.delta_g() - E["U_uv"]) < 2e-3 * scale
