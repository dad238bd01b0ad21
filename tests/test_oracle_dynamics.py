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


# ------------------------------------------------- thermostat (O-step) pins
# Section 2.6: the atoms are held at 298 K by Langevin dynamics (friction
# 10 ps^-1) in the leapfrog "middle" scheme.  A correct thermostat gives
# equipartition, <m v_d^2> = k_B T per Cartesian component of a free atom and
# <p^2/m> = k_B T for a free extended variable; a wrong Ornstein-Uhlenbeck
# amplitude (a missing factor, 1 - a instead of 1 - a^2) or velocities that
# mix the pre- and post-noise half steps fail these.

def test_langevin_middle_equipartition_free_atoms():
    rng = np.random.default_rng(2608)
    n, T, dt, gamma = 6000, 298.0, 0.002, 10.0
    kT = D.KB * T
    masses = np.array([1.008, 12.011, 15.999])
    mass = masses[np.arange(n) % 3]
    box = np.array([3.0, 3.0, 3.0])
    x = rng.uniform(0.0, 3.0, (n, 3))
    v = np.zeros((n, 3))
    F = np.zeros((n, 3))
    acc = np.zeros(3)
    cnt = 0
    for step in range(900):
        x, v = D.langevin_middle_step(x, v, F, mass, dt, gamma, T, rng.standard_normal((n, 3)), box, [], [])
        if step >= 300:   # 6 relaxation times 1/gamma
            mv2 = mass[:, None] * v * v
            acc += np.array([mv2[k::3].mean() for k in range(3)])
            cnt += 1
    per_class = acc / cnt
    assert np.allclose(per_class, kT, rtol=0.03), per_class / kT


def test_langevin_middle_equipartition_rigid_dimers():
    # rigid X-H dimers (one constraint, 5 degrees of freedom each) with no
    # forces: <KE> = 5/2 k_B T per dimer
    rng = np.random.default_rng(7)
    nm, T, dt, gamma = 60, 298.0, 0.001, 10.0
    kT = D.KB * T
    box = np.array([6.0, 6.0, 6.0])
    d0 = 0.109
    centres = rng.uniform(0.5, 5.5, (nm, 3))
    u = rng.standard_normal((nm, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    x = np.empty((2 * nm, 3))
    x[0::2] = centres
    x[1::2] = centres + d0 * u
    mass = np.tile([12.011, 1.008], nm)
    pairs = [(2 * k, 2 * k + 1) for k in range(nm)]
    lens = [d0] * nm
    v = np.zeros_like(x)
    F = np.zeros_like(x)
    ke = []
    for step in range(700):
        x, v = D.langevin_middle_step(x, v, F, mass, dt, gamma, T, rng.standard_normal(x.shape), box, pairs, lens)
        if step >= 200:
            ke.append(0.5 * (mass[:, None] * v * v).sum() / nm)
    assert np.mean(ke) == pytest.approx(2.5 * kT, rel=0.08)


def test_theta_step_equipartition_free_theta():
    # a free alchemical variable (no force, no bias): <p_theta^2 / m> = k_B T
    rng = np.random.default_rng(11)
    m, T, dt, gamma = 20.0, 298.0, 0.002, 25.0
    kT = D.KB * T
    th, p = 0.5, 0.0
    acc, cnt = 0.0, 0
    for step in range(120000):
        th, p = D.theta_step(th, p, 0.0, 1.0, 0.0, m, dt, gamma, T, rng.standard_normal())
        if step >= 1000:
            acc += p * p / m
            cnt += 1
    assert acc / cnt == pytest.approx(kT, rel=0.04)


# ------------------------------------------------------ multi-kernel OPES
# Eq. 11-13 evaluated by hand for kernels at theta = 0.3, 0.5, 0.4 with width
# sigma = 0.1: the Gaussians between the centres are exp(-2) (distance 0.2)
# and exp(-1/2) (distance 0.1); their periodic images (distance >= 1.8)
# contribute exp(-162) and are dropped.

SIG = 0.1
E2, EH = math.exp(-2.0), math.exp(-0.5)


def _g(d):
    return math.exp(-0.5 * d * d / (SIG * SIG))


@pytest.mark.parametrize("kind", ["std", "exp"])
def test_opes_two_and_three_kernels_by_hand(kind):
    T = 298.0
    b = D.Opes(kind, 30 * 4.184 if kind == "std" else 5 * 4.184, SIG, T)
    nu, beta, eps = b.nu, b.beta, b.eps
    std = kind == "std"
    # first kernel: V = 0 before it, so its weight is 1 in both variants;
    # rho_hat = G(theta - 0.3), rho_bar = rho_hat(0.3) = 1
    b.deposit(0.3)
    assert b.w == [1.0] and b.rho_bar == pytest.approx(1.0, rel=1e-15)
    assert b.bias(0.5)[0] == pytest.approx(nu / beta * math.log(E2 + eps), rel=1e-12)
    # second kernel at 0.5, weight exp(beta V_1(0.5)) = (e^-2 + eps)^nu (Standard)
    w2 = (E2 + eps) ** nu if std else 1.0
    b.deposit(0.5)
    assert b.w[1] == pytest.approx(w2, rel=1e-12)
    # rho_bar = [rho_hat(0.3) + rho_hat(0.5)] / 2 = (1 + e^-2) / 2 for any w2
    assert b.rho_bar == pytest.approx((1.0 + E2) / 2.0, rel=1e-12)
    for th in (0.2, 0.4, 0.45, 0.7):
        rho = (_g(th - 0.3) + w2 * _g(th - 0.5)) / (1.0 + w2)
        V = nu / beta * math.log(rho / ((1.0 + E2) / 2.0) + eps)
        assert b.bias(th)[0] == pytest.approx(V, rel=1e-12, abs=1e-12)
    # third kernel at 0.4: rho_hat_2(0.4) = e^-1/2 for any w2, so its
    # Standard weight is (2 e^-1/2 / (1 + e^-2) + eps)^nu
    w3 = (2.0 * EH / (1.0 + E2) + eps) ** nu if std else 1.0
    b.deposit(0.4)
    assert b.w[2] == pytest.approx(w3, rel=1e-12)
    W = 1.0 + w2 + w3
    rho_c = [(1.0 + w2 * E2 + w3 * EH) / W,      # at 0.3
             (E2 + w2 + w3 * EH) / W,            # at 0.5
             (EH + w2 * EH + w3) / W]            # at 0.4
    rho_bar = sum(rho_c) / 3.0
    assert b.rho_bar == pytest.approx(rho_bar, rel=1e-12)
    for th, rho in zip((0.3, 0.5, 0.4), rho_c):
        assert b.bias(th)[0] == pytest.approx(nu / beta * math.log(rho / rho_bar + eps), rel=1e-12, abs=1e-12)


def test_opes_explore_equal_spacing_gives_equal_bias_at_centres():
    # unit weights at n equally spaced centres around the period: rho_hat is
    # periodic with period 2/n, so it is the same at every centre and
    # V(centre) = (nu/beta) ln(1 + eps) exactly
    b = D.Opes("exp", 5 * 4.184, 0.3, 298.0)
    n = 8
    for k in range(n):
        b.deposit(2.0 * k / n + 0.05)
    for k in range(n):
        assert b.bias(2.0 * k / n + 0.05)[0] == pytest.approx(b.nu / b.beta * math.log(1.0 + b.eps), rel=1e-12)


def test_opes_dual_bias_standard_weight_uses_the_total_bias():
    # Section 2.3: Standard kernels are reweighted so that rho_hat converges
    # to the unbiased distribution; in the dual protocol the trajectory runs
    # under V_std + V_exp (Eq. 14), so the reweighting factor of a Standard
    # kernel is exp(beta (V_std + V_exp)) at its centre, both biases taken
    # before either deposits; Explore kernels keep unit weight
    T = 298.0
    std = D.Opes("std", 30 * 4.184, SIG, T)
    exp = D.Opes("exp", 5 * 4.184, SIG, T)
    D.opes_dual_deposit(std, exp, 0.3)
    assert std.w == [1.0] and exp.w == [1.0]
    Vs, Ve = std.bias(0.45)[0], exp.bias(0.45)[0]
    assert Vs != 0.0 and Ve != 0.0
    D.opes_dual_deposit(std, exp, 0.45)
    assert std.w[1] == pytest.approx(math.exp(std.beta * (Vs + Ve)), rel=1e-12)
    assert exp.w[1] == 1.0
    # a single bias (the other switched off) reweights by its own bias only
    solo = D.Opes("std", 30 * 4.184, SIG, T)
    solo.deposit(0.3)
    V1 = solo.bias(0.45)[0]
    D.opes_dual_deposit(solo, None, 0.45)
    assert solo.w[1] == pytest.approx(math.exp(solo.beta * V1), rel=1e-12)
