"""GPU parity of d-AFED (Eq. 15-16): coupling forces and energy against the
oracle, the auxiliary masses of Eq. 16, captured steps of atoms, theta and the
auxiliary angles against the oracle's steps, and bit-exact checkpoint resume
with the auxiliary state."""
import numpy as np
import pytest

from oracle import dynamics as D
from oracle import reference as R
from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

CVS = S.DIPEPTIDE_CVS
KAPPA = np.array([1000.0, 900.0, 800.0])
MASS_S = np.array([50.0, 40.0, 30.0])
SEED = 91


def frame():
    return S.make_c4_frame(frame=9)


@pytest.mark.parametrize("precision,tolF", [(lfe.LFE_FP64, 1e-9), (lfe.LFE_FP32_MIXED, 1e-5)])
def test_coupling_forces_and_energy_match_oracle(precision, tolF):
    d = frame()
    box = d["box"]
    xi = np.array([D.dihedral_grad(d["pos"], idx, box)[0] for idx in CVS])
    s0 = xi + np.array([0.3, -0.5, 2.9])
    g = lfe.System(d, precision=precision, seed=SEED)
    g.set_dafed(CVS, KAPPA, MASS_S, temperature=1000.0, friction=25.0, s0=s0)
    s, p, xig = g.dafed_state()
    assert np.allclose(s, np.vectorize(D.wrap_angle)(s0), atol=1e-14) and np.all(p == 0)
    assert np.allclose(xig, xi, atol=1e-9)
    lam = 0.4
    t, F = g.eval(lam)
    o = R.evaluate(d, lam, level=2)
    Ud, Fd, Fs = D.dafed_energy_forces(d["pos"], CVS, s0, KAPPA, box)
    Fo = o["F"] + Fd
    assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) <= tolF
    # the solute atoms carry the coupling: check them on their own too
    sol = np.flatnonzero(d["solute"])
    assert np.linalg.norm(F[sol] - Fo[sol]) / np.linalg.norm(Fo[sol]) <= 10 * tolF
    E = o["E"]
    # U sums large terms of both signs (self energies, exclusion corrections,
    # real and reciprocal parts): its error is measured against their magnitudes
    parts = [f"{q}_{c}" for q in ("coul_real", "rec", "bg", "lj", "excl") for c in ("vv", "uu", "uv")]
    parts += ["self_vv", "self_uu", "p14_vv", "p14_uu", "U_soft"]
    scale = sum(abs(E[k]) for k in parts) + abs(o["U_bonded"]) + Ud
    assert abs(t["U"] - (o["U"] + Ud)) <= (1e-9 if precision == lfe.LFE_FP64 else 1e-6) * scale
    g.set_dafed(np.zeros((0, 4)), [], [])
    t2, _ = g.eval(lam)
    assert abs(t2["U"] - o["U"]) <= (1e-9 if precision == lfe.LFE_FP64 else 1e-6) * scale


def test_masses_of_eq16_match_oracle():
    d = frame()
    g = lfe.System(d, precision=lfe.LFE_FP64)
    m = g.dafed_masses(CVS, c=300.0)
    mo = D.dafed_masses(d["pos"], CVS, d["mass"], 300.0, d["box"])
    assert np.allclose(m, mo, rtol=1e-10)


def small_dipeptide():
    d = S.make_water_box(seed=7, n_waters=60, box_len=1.6, solute="dipeptide22", n_side=5, r_cut=0.7,
                         grid=20, lam=0.62, frozen_solute=False, phi_psi_chi=(-75.0, 150.0, 178.0))
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=2,
             opes_dE_std=30 * 4.184, opes_dE_exp=5 * 4.184, opes_sigma=0.1)
    return d


def oracle_steps(d, nsteps, s0):
    pairs, lens = D.constraint_list(d)
    x = d["pos"].copy()
    v = np.zeros_like(x)
    th, pth = d["lam"], 0.0
    s, ps = s0.copy(), np.zeros(len(CVS))
    std = D.Opes("std", d["opes_dE_std"], d["opes_sigma"], d["temperature"])
    exp = D.Opes("exp", d["opes_dE_exp"], d["opes_sigma"], d["temperature"])
    for step in range(nsteps):
        lam, dl = D.theta_to_lambda(th)
        e = R.evaluate(d, lam, level=2, pos=x)
        _, Fd, Fs = D.dafed_energy_forces(x, CVS, s, KAPPA, d["box"])
        nrm = D.atom_normals(len(x), step, SEED)
        x, v = D.langevin_middle_step(x, v, e["F"] + Fd, d["mass"], d["dt"], d["friction"], d["temperature"],
                                      nrm, d["box"], pairs, lens)
        dV = std.bias(th)[1] + exp.bias(th)[1]
        th, pth = D.theta_step(th, pth, e["dUdl"], dl, dV, d["lambda_mass"], d["dt"], d["lambda_friction"],
                               d["temperature"], D.theta_normal(step, SEED))
        for k in range(len(CVS)):
            s[k], ps[k] = D.dafed_step(s[k], ps[k], Fs[k], MASS_S[k], d["dt"], 25.0, 1000.0,
                                       D.dafed_normal(k, step, SEED))
        if (step + 1) % d["opes_stride"] == 0:
            D.opes_dual_deposit(std, exp, th)
    return x, th, s, ps


def test_steps_with_dafed_match_oracle():
    d = small_dipeptide()
    xi = np.array([D.dihedral_grad(d["pos"], idx, d["box"])[0] for idx in CVS])
    s0 = xi + np.array([0.4, -0.3, 0.2])
    g = lfe.System(d, precision=lfe.LFE_FP64, seed=SEED)
    g.set_dafed(CVS, KAPPA, MASS_S, temperature=1000.0, friction=25.0, s0=s0)
    n = 4
    g.step(n)
    pos, _, ext = g.get_state()
    s, ps, _ = g.dafed_state()
    xo, tho, so, pso = oracle_steps(d, n, s0)
    dx = pos - xo
    dx -= d["box"] * np.round(dx / d["box"])
    assert np.abs(dx).max() <= 2e-8
    assert abs(ext["theta"] - tho) <= 1e-9
    assert np.allclose(s, so, atol=1e-9) and np.allclose(ps, pso, rtol=1e-7, atol=1e-9)


def test_checkpoint_resume_with_dafed_is_bitwise(tmp_path):
    d = small_dipeptide()
    g = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    g.set_dafed(CVS, KAPPA, MASS_S)
    g.step(3)
    path = tmp_path / "dafed.ckpt"
    g.checkpoint(path)
    g.step(3)
    pa, va, ea = g.get_state()
    sa, psa, _ = g.dafed_state()
    h = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    h.set_dafed(CVS, KAPPA, MASS_S)
    h.restore(path)
    h.step(3)
    pb, vb, eb = h.get_state()
    sb, psb, _ = h.dafed_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    assert np.array_equal(sa, sb) and np.array_equal(psa, psb)
    assert ea["theta"] == eb["theta"]
