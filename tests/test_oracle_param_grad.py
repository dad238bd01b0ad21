"""Pins of the oracle's parameter gradients (differentiation workload).

The class-resolved gradients dU_c/dp_i (p = charge, sigma, epsilon; c = own
class, uv, soft) are checked against what does not depend on their formula:
central finite differences of the oracle's energies, and the homogeneity
(Euler) identities of the energy in the charges and in epsilon.  A dropped
term (self, background, exclusion correction, 1-4 pair, reciprocal cross
potential), a wrong mixing-rule factor or a class mix-up fails one of them.
"""
import numpy as np
import pytest

from oracle import reference as R
from paper_2608_12691_b300 import systems as S


@pytest.fixture(scope="module")
def dip():
    # 22-atom flexible solute (exclusions and scaled 1-4 pairs) in 60 waters
    return S.make_water_box(seed=7, n_waters=60, box_len=1.6, solute="dipeptide22", n_side=5,
                            r_cut=0.7, grid=20)


def _classes(d, level, **over):
    dd = dict(d)
    dd.update(over)
    E, _, _, _ = R.nonbonded(dd, level=level, forces=False)
    return np.array([E["U_vv"] + E["U_uu"], E["U_uv"], E["U_soft"]]), E


@pytest.mark.parametrize("level", [1, 2])
def test_param_grad_matches_fd(dip, level):
    G = R.param_grad(dip, level=level)
    sol = np.flatnonzero(dip["solute"])
    atoms = list(sol[[0, 3, 7, 12, 21]]) + [30, 101, 150]
    for i in atoms:
        for p, key, h, tol in ((0, "charge", 1e-4, 1e-8), (1, "sigma", 1e-6, 2e-6), (2, "epsilon", 1e-6, 2e-6)):
            if key != "charge" and dip[key][i] == 0.0:
                continue
            a = dip[key].copy(); a[i] += h
            b = dip[key].copy(); b[i] -= h
            fd = (_classes(dip, level, **{key: a})[0] - _classes(dip, level, **{key: b})[0]) / (2 * h)
            scale = np.maximum(1.0, np.abs(fd))
            assert np.all(np.abs(G[i, p] - fd) <= tol * scale), (level, i, key, G[i, p], fd)


@pytest.mark.parametrize("level", [1, 2])
def test_euler_identities_in_the_solute_charges(dip, level):
    # U_uv^C is linear and U_uu^C quadratic in the solute charges, so
    # sum_u q_i dU_uv/dq_i = U_uv^C and sum_u q_i dU_uu/dq_i = 2 U_uu^C
    G = R.param_grad(dip, level=level)
    sol = dip["solute"].astype(bool)
    q = dip["charge"]
    _, E = _classes(dip, level)
    q0 = q.copy(); q0[sol] = 0.0
    _, E0 = _classes(dip, level, charge=q0)
    uvC = E["U_uv"] - E0["U_uv"]
    uuC = E["U_uu"] - E0["U_uu"]
    lhs_uv = np.sum(q[sol] * G[sol, 0, 1])
    lhs_uu = np.sum(q[sol] * G[sol, 0, 0])
    assert lhs_uv == pytest.approx(uvC, rel=1e-9, abs=1e-8)
    assert lhs_uu == pytest.approx(2.0 * uuC, rel=1e-9, abs=1e-8)
    # over every atom, each class Coulomb energy is quadratic in all charges
    _, Ez = _classes(dip, level, charge=np.zeros_like(q))
    allC = (E["U_vv"] + E["U_uu"] + E["U_uv"]) - (Ez["U_vv"] + Ez["U_uu"] + Ez["U_uv"])
    assert np.sum(q[:, None] * G[:, 0, :2]) == pytest.approx(2.0 * allC, rel=1e-9)


def test_euler_identity_in_the_solute_epsilon(dip):
    # eps_ij = sqrt(eps_i eps_j): the uv LJ and the soft basis are homogeneous
    # of degree 1/2 in the solute epsilons, the uu LJ of degree 1
    G = R.param_grad(dip, level=0)
    sol = dip["solute"].astype(bool)
    eps = dip["epsilon"]
    _, E = _classes(dip, 0)
    e0 = eps.copy(); e0[sol] = 0.0
    _, E0 = _classes(dip, 0, epsilon=e0)
    assert np.all(eps[sol] > 0)
    assert np.sum(eps[sol] * G[sol, 2, 1]) == pytest.approx(0.5 * (E["U_uv"] - E0["U_uv"]), rel=1e-10)
    assert np.sum(eps[sol] * G[sol, 2, 2]) == pytest.approx(0.5 * E["U_soft"], rel=1e-10)
    assert np.sum(eps[sol] * G[sol, 2, 0]) == pytest.approx(E["U_uu"] - E0["U_uu"], rel=1e-10)


def test_lambda_assembly_matches_fd_of_U_and_dUdl(dip):
    lam = 0.62
    G = R.param_grad(dip, level=2)
    dU, d2 = R.assemble_param_grad(G, lam)
    sol = np.flatnonzero(dip["solute"])
    for i in sol[[1, 9, 18]]:
        for p, key, h in ((0, "charge", 1e-4), (2, "epsilon", 1e-6)):
            a = dip[key].copy(); a[i] += h
            b = dip[key].copy(); b[i] -= h
            ea = R.evaluate(dict(dip, **{key: a}), lam, level=2, with_bonded=False)
            eb = R.evaluate(dict(dip, **{key: b}), lam, level=2, with_bonded=False)
            fdU = (ea["U"] - eb["U"]) / (2 * h)
            fdd = (ea["dUdl"] - eb["dUdl"]) / (2 * h)
            assert dU[i, p] == pytest.approx(fdU, rel=2e-6, abs=2e-6)
            assert d2[i, p] == pytest.approx(fdd, rel=2e-6, abs=2e-6)


def test_zero_epsilon_site_has_finite_zero_epsilon_gradient():
    d = dict(box=np.array([2.0, 2.0, 2.0]), pos=np.array([[0.3, 0.4, 0.5], [0.6, 0.5, 0.45]]),
             charge=np.array([0.4, -0.4]), sigma=np.array([0.3, 0.0]), epsilon=np.array([0.5, 0.0]),
             solute=np.array([1, 0], np.uint8), excl=np.zeros((0, 2), np.int32),
             pairs14=np.zeros((0, 2), np.int32), scale14=np.zeros((0, 2)),
             r_cut=0.9, r_switch=0.8, alpha=3.5, grid=[16] * 3, order=4)
    G = R.param_grad(d, level=0)
    assert np.all(np.isfinite(G))
    assert np.all(G[:, 1:, :] == 0.0)   # eps_ij = 0: no LJ, no soft term
    # two point charges, real space only: dU_uv/dq_0 = k_e q_1 erfc(a r)/r
    from math import erfc, sqrt
    r = sqrt(np.sum((d["pos"][1] - d["pos"][0]) ** 2))
    assert G[0, 0, 1] == pytest.approx(138.935458 * (-0.4) * erfc(3.5 * r) / r, rel=1e-14)
