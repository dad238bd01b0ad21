"""GPU parity of the regulated Nose-Hoover-Langevin thermostat of the
extended variables (Section 2.6): captured steps of theta under the dual
OPES bias, and of theta with the d-AFED auxiliary angles, against the
oracle's steps (same Philox counters, the oracle's rnhl_step); bit-exact
checkpoint resume with the thermostat velocities; argument checks."""
import numpy as np
import pytest

from oracle import dynamics as D
from oracle import reference as R
from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

SEED = 57
TAU, NREG = 0.04, 1.0
CVS = S.DIPEPTIDE_CVS
KAPPA = np.array([1000.0, 900.0, 800.0])
MASS_S = np.array([50.0, 40.0, 30.0])


def water_system():
    d = S.make_water_box(seed=21, n_waters=101, box_len=1.45, solute="ring12", n_side=5,
                         r_cut=0.7, grid=16, lam=0.62)
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=2,
             opes_dE_std=30 * 4.184, opes_dE_exp=5 * 4.184, opes_sigma=0.1)
    return d


def dipeptide_system():
    d = S.make_water_box(seed=7, n_waters=60, box_len=1.6, solute="dipeptide22", n_side=5, r_cut=0.7,
                         grid=20, lam=0.62, frozen_solute=False, phi_psi_chi=(-75.0, 150.0, 178.0))
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=2,
             opes_dE_std=30 * 4.184, opes_dE_exp=5 * 4.184, opes_sigma=0.1)
    return d


def oracle_steps(d, nsteps, s0=None):
    pairs, lens = D.constraint_list(d)
    x = d["pos"].copy()
    v = np.zeros_like(x)
    th, pth, vth = d["lam"], 0.0, 0.0
    ncv = 0 if s0 is None else len(CVS)
    s, ps, vs = (s0.copy() if ncv else np.zeros(0)), np.zeros(ncv), np.zeros(ncv)
    std = D.Opes("std", d["opes_dE_std"], d["opes_sigma"], d["temperature"])
    exp = D.Opes("exp", d["opes_dE_exp"], d["opes_sigma"], d["temperature"])
    for step in range(nsteps):
        lam, dl = D.theta_to_lambda(th)
        e = R.evaluate(d, lam, level=2, pos=x)
        F = e["F"]
        if ncv:
            _, Fd, Fs = D.dafed_energy_forces(x, CVS, s, KAPPA, d["box"])
            F = F + Fd
        nrm = D.atom_normals(len(x), step, SEED)
        x, v = D.langevin_middle_step(x, v, F, d["mass"], d["dt"], d["friction"], d["temperature"],
                                      nrm, d["box"], pairs, lens)
        dV = std.bias(th)[1] + exp.bias(th)[1]
        th, pth, vth = D.theta_step_rnhl(th, pth, vth, e["dUdl"], dl, dV, d["lambda_mass"], d["dt"],
                                         d["lambda_friction"], d["temperature"], TAU, NREG,
                                         D.theta_normal(step, SEED))
        for k in range(ncv):
            s[k], ps[k], vs[k] = D.dafed_step_rnhl(s[k], ps[k], vs[k], Fs[k], MASS_S[k], d["dt"], 25.0, 1000.0,
                                                   TAU, NREG, D.dafed_normal(k, step, SEED))
        if (step + 1) % d["opes_stride"] == 0:
            D.opes_dual_deposit(std, exp, th)
    return x, th, pth, vth, s, ps, vs


@pytest.mark.parametrize("precision,tx,tth", [(lfe.LFE_FP64, 2e-8, 1e-9), (lfe.LFE_FP32_MIXED, 5e-6, 1e-6)])
def test_theta_steps_under_rnhl_match_oracle(precision, tx, tth):
    d = water_system()
    n = 6
    g = lfe.System(d, precision=precision, seed=SEED)
    g.set_ext_thermostat(lfe.LFE_EXT_RNHL, TAU, NREG)
    g.step(n)
    pos, _, ext = g.get_state()
    vth, _ = g.ext_thermostat_state()
    xo, tho, pto, vto, _, _, _ = oracle_steps(d, n)
    dx = pos - xo
    dx -= d["box"] * np.round(dx / d["box"])
    assert np.abs(dx).max() <= tx
    assert abs(ext["theta"] - tho) <= tth
    assert ext["p_theta"] == pytest.approx(pto, rel=1e-6 if precision == lfe.LFE_FP64 else 1e-4, abs=1e-9)
    assert vth == pytest.approx(vto, rel=1e-6 if precision == lfe.LFE_FP64 else 1e-4, abs=1e-9)
    assert vto != 0.0


def test_theta_and_auxiliary_angles_under_rnhl_match_oracle():
    d = dipeptide_system()
    xi = np.array([D.dihedral_grad(d["pos"], idx, d["box"])[0] for idx in CVS])
    s0 = xi + np.array([0.4, -0.3, 0.2])
    g = lfe.System(d, precision=lfe.LFE_FP64, seed=SEED)
    g.set_dafed(CVS, KAPPA, MASS_S, temperature=1000.0, friction=25.0, s0=s0)
    g.set_ext_thermostat(lfe.LFE_EXT_RNHL, TAU, NREG)
    n = 4
    g.step(n)
    pos, _, ext = g.get_state()
    s, ps, _ = g.dafed_state()
    vth, vs = g.ext_thermostat_state()
    xo, tho, pto, vto, so, pso, vso = oracle_steps(d, n, s0)
    dx = pos - xo
    dx -= d["box"] * np.round(dx / d["box"])
    assert np.abs(dx).max() <= 2e-8
    assert abs(ext["theta"] - tho) <= 1e-9 and vth == pytest.approx(vto, rel=1e-6, abs=1e-9)
    assert np.allclose(s, so, atol=1e-9) and np.allclose(ps, pso, rtol=1e-7, atol=1e-9)
    assert np.allclose(vs, vso, rtol=1e-6, atol=1e-9) and np.all(vso != 0.0)


def test_checkpoint_resume_under_rnhl_is_bitwise(tmp_path):
    d = dipeptide_system()

    def make():
        g = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
        g.set_dafed(CVS, KAPPA, MASS_S, temperature=1000.0, friction=25.0)
        g.set_ext_thermostat(lfe.LFE_EXT_RNHL, TAU, NREG)
        return g

    g = make()
    g.step(3)
    path = tmp_path / "rnhl.ckpt"
    g.checkpoint(path)
    g.step(3)
    pa, va, ea = g.get_state()
    sa, psa, _ = g.dafed_state()
    ta, aa = g.ext_thermostat_state()
    h = make()
    h.restore(path)
    h.step(3)
    pb, vb, eb = h.get_state()
    sb, psb, _ = h.dafed_state()
    tb, ab = h.ext_thermostat_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    assert np.array_equal(sa, sb) and np.array_equal(psa, psb)
    assert ta == tb and np.array_equal(aa, ab) and ta != 0.0
    assert all(ea[k] == eb[k] for k in ea)


def test_bad_thermostat_arguments_are_rejected():
    d = water_system()
    g = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    for args in ((2, TAU, NREG), (lfe.LFE_EXT_RNHL, 0.0, NREG), (lfe.LFE_EXT_RNHL, TAU, -1.0),
                 (lfe.LFE_EXT_RNHL, float("nan"), NREG)):
        with pytest.raises(lfe.LfeError) as e:
            g.set_ext_thermostat(*args)
        assert e.value.code == lfe.LFE_ERR_ARG
    # back to Langevin: the thermostat velocity stays 0 while stepping
    g.set_ext_thermostat(lfe.LFE_EXT_LANGEVIN)
    g.step(3)
    assert g.ext_thermostat_state()[0] == 0.0
