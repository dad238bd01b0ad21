"""Pins of the oracle's extended-variable loop (Eq. 3, 11-14), RNG and
constrained Langevin steps."""
import math

import numpy as np
import pytest

from oracle import dynamics as D
from oracle import reference as R
from paper_2608_12691_b300 import systems as S
from test_golden import rows as golden_rows


def test_philox_known_answers():
    # known-answer vectors of Philox4x32-10 (Salmon et al. 2011, Random123 KAT),
    # stored with their citation under tests/golden/
    kats = [r for r in golden_rows("philox4x32_10_kat.txt") if r[0] == "kat"]
    assert len(kats) == 3
    for r in kats:
        ctr = tuple(int(x, 16) for x in r[1:5])
        key = tuple(int(x, 16) for x in r[5:7])
        assert [f"{x:08x}" for x in D.philox4x32_10(ctr, key)] == r[7:11]


def test_box_muller_moments():
    z = np.array([D.normals3((i, 7, 0, 0), (12345, 0)) for i in range(20000)]).ravel()
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.03


def test_mirror_map():
    # Eq. 3 and the periodic wrap of theta into [0, 2)
    assert D.theta_to_lambda(0.3) == (0.3, 1.0)
    assert D.theta_to_lambda(1.0) == (1.0, 1.0)
    lam, s = D.theta_to_lambda(1.25)
    assert lam == pytest.approx(0.75) and s == -1.0
    lam, s = D.theta_to_lambda(2.1)
    assert lam == pytest.approx(0.1) and s == 1.0
    lam, s = D.theta_to_lambda(-0.2)
    assert lam == pytest.approx(0.2) and s == -1.0


def test_theta_force_continuous_at_folds():
    # dh_A/dlambda and dh_B/dlambda vanish at lambda = 0 and 1, so the
    # generalized force -(dlambda/dtheta) dU/dlambda is continuous at the folds
    for th in (1.0, 2.0 - 1e-12, 1e-12):
        lam_m, s_m = D.theta_to_lambda(th - 1e-7)
        lam_p, s_p = D.theta_to_lambda(th + 1e-7)
        for lam, s in ((lam_m, s_m), (lam_p, s_p)):
            _, _, dA, dB = R.switching(lam)
            assert abs(s * dA) < 1e-9 and abs(s * dB) < 1e-9


def test_opes_parameters_and_bounds():
    T = 298.0
    beta = 1.0 / (D.KB * T)
    dE = 30 * 4.184
    # a narrow kernel so that rho_hat at the far side of the period is far below eps
    std = D.Opes("std", dE, 0.05, T)
    exp = D.Opes("exp", 5 * 4.184, 0.05, T)
    assert std.gamma == pytest.approx(beta * dE)
    assert std.nu == pytest.approx(1 - 1 / std.gamma)
    assert exp.nu == pytest.approx(exp.gamma - 1)
    assert std.bias(0.4) == (0.0, 0.0)   # no kernels yet
    for b in (std, exp):
        b.deposit(0.4)
        # far from all kernels rho_hat -> 0 and V -> (nu/beta) ln(eps) = -Delta E
        Vfar, _ = b.bias(1.4)
        assert Vfar == pytest.approx((b.nu / b.beta) * math.log(b.eps), rel=1e-12)
        assert Vfar == pytest.approx(-(b.gamma / b.beta), rel=1e-9)
        # at the single centre rho_hat = rho_bar -> V = (nu/beta) ln(1 + eps)
        assert b.bias(0.4)[0] == pytest.approx(b.nu / b.beta * math.log(1 + b.eps), rel=1e-12)
        # the regularisation bounds the bias from below by -Delta E everywhere
        assert min(b.bias(t)[0] for t in np.linspace(0, 2, 101)) >= -(b.gamma / b.beta) - 1e-9


def test_opes_derivative_fd_and_periodicity():
    b = D.Opes("std", 30 * 4.184, 0.1, 298.0)
    for th in (0.05, 0.3, 0.33, 1.2, 1.9, 1.97):
        b.deposit(th)
    for th in (0.0, 0.2, 0.5, 1.0, 1.5, 1.99):
        h = 1e-6
        fd = (b.bias(th + h)[0] - b.bias(th - h)[0]) / (2 * h)
        assert b.bias(th)[1] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    assert b.bias(0.1)[0] == pytest.approx(b.bias(2.1)[0], rel=1e-12)
    # standard kernels are reweighted by exp(beta V) at deposition
    assert b.w[0] == 1.0 and b.w[1] != 1.0


def test_shake_converges_to_rigid_water():
    d = S.make_water_box(seed=3, n_waters=20, box_len=1.2, solute=None, n_side=3)
    pairs, lens = D.constraint_list(d)
    rng = np.random.default_rng(0)
    x_new = d["pos"] + rng.normal(scale=0.003, size=d["pos"].shape)
    w = 1.0 / d["mass"]
    x = D.shake(x_new, d["pos"], pairs, lens, w, d["box"])
    for (i, j), L in zip(pairs, lens):
        r = x[j] - x[i]
        r -= d["box"] * np.round(r / d["box"])
        assert np.linalg.norm(r) == pytest.approx(L, rel=1e-12)
    # constraint forces are internal: the mass-weighted displacement is unchanged
    m = d["mass"][:, None]
    assert np.allclose((m * (x - x_new)).sum(0), 0.0, atol=1e-12)


def test_nve_energy_drift_small_box():
    # gamma = 0: the middle scheme reduces to leapfrog with SHAKE; the total
    # energy of a small water box must not drift (dt 0.5 fs).  alpha is raised
    # so that erfc(alpha r_c) ~ 1e-6 and the Coulomb cutoff adds no jumps.
    d = S.make_water_box(seed=4, n_waters=27, box_len=1.25, solute=None, n_side=3,
                         r_cut=0.6, grid=24)
    d["alpha"] = 5.8
    pairs, lens = D.constraint_list(d)
    box = d["box"]
    dt = 0.0005
    zeros = np.zeros_like(d["pos"])
    rng = np.random.default_rng(1)

    def force(x):
        e = R.evaluate(d, 1.0, level=2, pos=x, with_bonded=False)
        return e["U"], e["F"]

    def ke(v):
        return 0.5 * (d["mass"][:, None] * v * v).sum()

    # relax the lattice start with friction, then switch it off
    x, v = d["pos"].copy(), np.zeros_like(d["pos"])
    for step in range(150):
        U, F = force(x)
        nrm = D.atom_normals(len(x), step, 99)
        x, v = D.langevin_middle_step(x, v, F, d["mass"], dt, 50.0, 298.0, nrm, box, pairs, lens)
    energies = []
    v_prev = v
    for step in range(300):
        U, F = force(x)
        x, v = D.langevin_middle_step(x, v_prev, F, d["mass"], dt, 0.0, 298.0, zeros, box, pairs, lens)
        # on-step kinetic energy: mean of the two half-step values
        energies.append(U + 0.5 * (ke(v_prev) + ke(v)))
        v_prev = v
    energies = np.array(energies)
    q = len(energies) // 4
    drift = abs(energies[-q:].mean() - energies[:q].mean())
    assert drift / ke(v) < 2e-3


# ---------------------------------------------------- lambda replica exchange

def test_hrex_delta_is_the_swapped_energy_difference():
    # the basis form of the swap energy equals the difference of four full
    # evaluations (Eq. 4 at both lambdas for both configurations)
    d = S.make_c0()
    rng = np.random.default_rng(5)
    xi = d["pos"]
    xj = S.f32(d["pos"] + rng.normal(0.0, 0.003, d["pos"].shape))
    a, b = 0.45, 0.8
    ei = R.evaluate(d, a, level=1, pos=xi, with_bonded=False)
    ej = R.evaluate(d, b, level=1, pos=xj, with_bonded=False)
    eib = R.evaluate(d, b, level=1, pos=xi, with_bonded=False)
    eja = R.evaluate(d, a, level=1, pos=xj, with_bonded=False)
    direct = (eib["U"] + eja["U"]) - (ei["U"] + ej["U"])
    Ei, Ej = R.nonbonded(d, level=1, pos=xi)[0], R.nonbonded(d, level=1, pos=xj)[0]
    basis = D.hrex_delta(a, b, Ei["U_uv"], Ei["U_soft"], Ej["U_uv"], Ej["U_soft"])
    assert basis == pytest.approx(direct, rel=1e-9, abs=1e-9)


def test_hrex_attempt_metropolis_rules():
    T, seed = 298.0, 11
    # equal configurations: Delta = 0, always accepted, lambdas swap pairwise
    acc, new = D.hrex_attempt([0.1, 0.5, 0.9, 1.0], [3.0] * 4, [2.0] * 4, T, seed, attempt=0)
    assert acc == [1, 0, 1] and new == [0.5, 0.1, 1.0, 0.9]
    # odd attempts try the other pairs
    acc, new = D.hrex_attempt([0.1, 0.5, 0.9, 1.0], [3.0] * 4, [2.0] * 4, T, seed, attempt=1)
    assert acc == [0, 1, 0] and new == [0.1, 0.9, 0.5, 1.0]
    # a huge uphill Delta is rejected
    acc, _ = D.hrex_attempt([0.5, 1.0], [1e6, 0.0], [0.0, 0.0], T, seed, attempt=0)
    assert D.hrex_delta(0.5, 1.0, 1e6, 0.0, 0.0, 0.0) > 0 and acc == [0]
    # the acceptance frequency of a fixed Delta matches exp(-beta Delta)
    lam = [0.6, 0.7]
    hA = [R.switching(x)[0] for x in lam]
    dU = 0.7 / (hA[1] - hA[0])          # U_uv difference that gives Delta = 0.7 kJ/mol
    delta = D.hrex_delta(0.6, 0.7, dU, 0.0, 0.0, 0.0)
    assert delta == pytest.approx(0.7)
    n = 4000
    hits = sum(D.hrex_attempt(lam, [dU, 0.0], [0.0, 0.0], T, seed, attempt=2 * t)[0][0] for t in range(n))
    p = math.exp(-0.7 / (0.0083144626 * T))
    assert abs(hits / n - p) < 4 * math.sqrt(p * (1 - p) / n)
