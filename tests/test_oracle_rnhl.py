"""Pins of the oracle's regulated Nose-Hoover-Langevin thermostat (the
extended variables' thermostat of Section 2.6) against what its invariant
density exp(-(U(x) + K(p) + Q v_eta^2 / 2) / kT), K(p) = n kT ln cosh(p /
sqrt(n m kT)), fixes in closed form:
  * K'(p) is the derivative of K (finite differences), is bounded by
    sqrt(n kT / m) and tends to p / m as n grows;
  * for a free variable, <p K'(p)> = kT, <v_eta^2> = kT / Q, and the
    momentum density proportional to cosh(y)^-n, y = p / sqrt(n m kT), has
    <y^2> = pi^2 / 4 (n = 1, hyperbolic secant) and pi^2 / 12 (n = 2,
    logistic);
  * in a harmonic well U = k x^2 / 2 the position marginal is Boltzmann:
    <x^2> = kT / k.
Many independent copies are stepped at once (numpy arrays)."""
import math

import numpy as np
import pytest

from oracle import dynamics as D

T, M, DT, TAU, GAMMA = 298.0, 20.0, 0.001, 0.04, 25.0
KT = D.KB * T


def test_regulated_velocity_is_the_kinetic_derivative_and_bounded():
    p = np.linspace(-40.0, 40.0, 81)
    for n in (1.0, 2.0, 5.0):
        K = lambda q: n * KT * np.log(np.cosh(q / np.sqrt(n * M * KT)))
        h = 1e-5
        fd = (K(p + h) - K(p - h)) / (2 * h)
        v = D.regulated_velocity(p, M, KT, n)
        assert np.allclose(v, fd, rtol=1e-7, atol=1e-10)
        assert np.all(np.abs(v) < math.sqrt(n * KT / M))
        assert np.allclose(D.regulated_velocity(-p, M, KT, n), -v)
    big = D.regulated_velocity(p, M, KT, 1e10)
    assert np.allclose(big, p / M, rtol=1e-8)


def run_free(n, steps=3000, burn=1000, copies=4000, seed=1):
    rng = np.random.default_rng(seed)
    x = np.zeros(copies)
    p = rng.choice([-1.0, 1.0], size=copies) * np.sqrt(M * KT)
    ve = np.zeros(copies)
    s_pv = s_p2 = s_v2 = 0.0
    cnt = 0
    for step in range(steps):
        x, p, ve = D.rnhl_step(x, p, ve, 0.0, M, DT, GAMMA, T, TAU, n, rng.standard_normal(copies))
        if step >= burn and step % 10 == 0:
            s_pv += (p * D.regulated_velocity(p, M, KT, n)).mean()
            s_p2 += (p * p).mean()
            s_v2 += (ve * ve).mean()
            cnt += 1
    return s_pv / cnt, s_p2 / cnt, s_v2 / cnt


@pytest.mark.parametrize("n,y2", [(1.0, math.pi ** 2 / 4.0), (2.0, math.pi ** 2 / 12.0)])
def test_free_variable_moments(n, y2):
    pv, p2, v2 = run_free(n)
    Q = KT * TAU * TAU
    assert pv == pytest.approx(KT, rel=0.02)
    assert v2 == pytest.approx(KT / Q, rel=0.03)
    assert p2 / (n * M * KT) == pytest.approx(y2, rel=0.03)


def test_harmonic_well_position_marginal_is_boltzmann():
    rng = np.random.default_rng(2)
    k = M * (2.0 * math.pi / 0.5) ** 2      # unregulated period 0.5 ps
    copies = 4000
    x = np.zeros(copies)
    p = rng.standard_normal(copies) * np.sqrt(M * KT)
    ve = np.zeros(copies)
    acc, cnt = 0.0, 0
    for step in range(4000):
        x, p, ve = D.rnhl_step(x, p, ve, -k * x, M, DT, GAMMA, T, TAU, 1.0, rng.standard_normal(copies))
        if step >= 1000 and step % 10 == 0:
            acc += (x * x).mean()
            cnt += 1
    assert acc / cnt == pytest.approx(KT / k, rel=0.03)


def test_theta_and_auxiliary_wrappers_wrap():
    th, p, ve = D.theta_step_rnhl(1.9999, 50.0, 0.0, 0.0, 1.0, 0.0, M, DT, GAMMA, T, TAU, 1.0, 0.0)
    assert 0.0 <= th < 2.0 and th < 0.01
    s, p, ve = D.dafed_step_rnhl(math.pi - 1e-4, 50.0, 0.0, 0.0, M, DT, GAMMA, T, TAU, 1.0, 0.0)
    assert -math.pi <= s < -math.pi + 0.01
