"""Pins of the oracle's d-AFED coupling (Eq. 15-16) and auxiliary integrator.

Forces and the auxiliary force are checked against central differences of the
energy, the energy's zero and periodicity, the dihedral gradient's zero total
force and torque, the mass formula against its closed form when only the end
atoms carry mass, and the auxiliary thermostat against equipartition at its
own temperature.
"""
import math

import numpy as np
import pytest

from oracle import dynamics as D
from paper_2608_12691_b300 import systems as S


@pytest.fixture(scope="module")
def frame():
    d = S.make_water_box(seed=7, n_waters=60, box_len=1.6, solute="dipeptide22", n_side=5,
                         r_cut=0.7, grid=20, phi_psi_chi=(-75.0, 150.0, 178.0))
    return d


def test_cvs_are_the_built_angles(frame):
    xi = [D.dihedral_grad(frame["pos"], idx, frame["box"])[0] for idx in S.DIPEPTIDE_CVS]
    want = np.radians([-75.0, 150.0, 178.0])
    # the Z-matrix builds each dihedral (same sign convention) up to the
    # float32 rounding of the coordinates
    assert np.allclose(np.vectorize(D.wrap_angle)(np.array(xi) - want), 0.0, atol=1e-5)


def test_forces_are_minus_gradient(frame):
    pos = frame["pos"]
    box = frame["box"]
    cvs = S.DIPEPTIDE_CVS
    s = np.array([3.1, -2.9, 0.4])          # near the periodic seam for the first two
    kappa = np.array([1000.0, 800.0, 600.0])
    U, F, Fs = D.dafed_energy_forces(pos, cvs, s, kappa, box)
    h = 1e-6
    for idx in cvs:
        for atom in idx:
            for k in range(3):
                pp = pos.copy(); pp[atom, k] += h
                pm = pos.copy(); pm[atom, k] -= h
                fd = -(D.dafed_energy_forces(pp, cvs, s, kappa, box)[0] -
                       D.dafed_energy_forces(pm, cvs, s, kappa, box)[0]) / (2 * h)
                assert F[atom, k] == pytest.approx(fd, rel=1e-5, abs=1e-4)
    for k in range(3):
        sp = s.copy(); sp[k] += h
        sm = s.copy(); sm[k] -= h
        fd = -(D.dafed_energy_forces(pos, cvs, sp, kappa, box)[0] -
               D.dafed_energy_forces(pos, cvs, sm, kappa, box)[0]) / (2 * h)
        assert Fs[k] == pytest.approx(fd, rel=1e-6, abs=1e-5)
    # zero total force and torque on each torsion
    assert np.allclose(F.sum(axis=0), 0.0, atol=1e-9)


def test_energy_zero_and_periodic(frame):
    pos, box = frame["pos"], frame["box"]
    cvs = S.DIPEPTIDE_CVS
    xi = np.array([D.dihedral_grad(pos, idx, box)[0] for idx in cvs])
    kappa = np.full(3, 1000.0)
    U0, F0, Fs0 = D.dafed_energy_forces(pos, cvs, xi, kappa, box)
    assert U0 == pytest.approx(0.0, abs=1e-20) and np.allclose(F0, 0.0) and np.allclose(Fs0, 0.0)
    s = xi + np.array([0.3, -0.2, 0.1])
    a = D.dafed_energy_forces(pos, cvs, s, kappa, box)
    b = D.dafed_energy_forces(pos, cvs, s + 2 * np.pi * np.array([1, -2, 3]), kappa, box)
    assert a[0] == pytest.approx(b[0], rel=1e-12)
    assert a[0] == pytest.approx(0.5 * 1000.0 * (0.09 + 0.04 + 0.01), rel=1e-10)


def test_gradient_has_no_net_torque(frame):
    pos, box = frame["pos"], frame["box"]
    for idx in S.DIPEPTIDE_CVS:
        _, g = D.dihedral_grad(pos, idx, box)
        r = np.array([pos[i] for i in idx])
        assert np.allclose(g.sum(axis=0), 0.0, atol=1e-10)
        assert np.allclose(np.cross(r, g).sum(axis=0), 0.0, atol=1e-9)


def test_mass_formula_closed_form(frame):
    # only the end atoms movable: |dxi/dr_a| = 1/(|b1| sin theta_abc),
    # |dxi/dr_d| = 1/(|b3| sin theta_bcd)
    pos, box = frame["pos"], frame["box"]
    idx = S.DIPEPTIDE_CVS[0]
    mass = np.zeros(len(pos))
    mass[idx[0]], mass[idx[3]] = 12.0, 14.0
    a, b, c, d = (pos[i] for i in idx)
    b1, b2, b3 = b - a, c - b, d - c
    sin1 = np.linalg.norm(np.cross(b1, b2)) / (np.linalg.norm(b1) * np.linalg.norm(b2))
    sin2 = np.linalg.norm(np.cross(b2, b3)) / (np.linalg.norm(b2) * np.linalg.norm(b3))
    want = 300.0 / (1 / (12.0 * (np.linalg.norm(b1) * sin1) ** 2) + 1 / (14.0 * (np.linalg.norm(b3) * sin2) ** 2))
    got = D.dafed_masses(pos, [idx], mass, 300.0, box)[0]
    assert got == pytest.approx(want, rel=1e-10)


def test_auxiliary_thermostat_equipartition():
    # a free auxiliary variable at 1000 K: <p^2 / m> = k_B T
    m, T, dt, gamma = 50.0, 1000.0, 0.002, 25.0
    s, p = 0.0, 0.0
    acc, nacc = 0.0, 0
    for step in range(30000):
        s, p = D.dafed_step(s, p, 0.0, m, dt, gamma, T, D.dafed_normal(0, step, 11))
        assert -math.pi <= s < math.pi
        if step > 2000:
            acc += p * p / m
            nacc += 1
    assert acc / nacc == pytest.approx(D.KB * T, rel=0.05)
