"""GPU dynamics parity: captured steps of the CUDA path (Langevin middle
scheme with rigid waters, theta under the dual OPES bias) against the same
steps taken by the oracle (level-2 forces, SHAKE to convergence, the same
Philox4x32-10 counters), plus bit-exact checkpoint / resume."""
import math

import numpy as np
import pytest

from oracle import dynamics as D
from oracle import reference as R
from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

SEED = 77


def water_system():
    d = S.make_water_box(seed=21, n_waters=101, box_len=1.45, solute="ring12", n_side=5,
                         r_cut=0.7, grid=16, lam=0.62)
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=2,
             opes_dE_std=30 * 4.184, opes_dE_exp=5 * 4.184, opes_sigma=0.1)
    return d


def oracle_steps(d, nsteps):
    pairs, lens = D.constraint_list(d)
    x = d["pos"].copy()
    v = np.zeros_like(x)
    th, p = d["lam"], 0.0
    std = D.Opes("std", d["opes_dE_std"], d["opes_sigma"], d["temperature"])
    exp = D.Opes("exp", d["opes_dE_exp"], d["opes_sigma"], d["temperature"])
    ti = D.TIAccumulator()
    for step in range(nsteps):
        lam, dl = D.theta_to_lambda(th)
        e = R.evaluate(d, lam, level=2, pos=x)
        ti.add(lam, e["dUdl"])
        nrm = D.atom_normals(len(x), step, SEED)
        x, v = D.langevin_middle_step(x, v, e["F"], d["mass"], d["dt"], d["friction"], d["temperature"],
                                      nrm, d["box"], pairs, lens)
        dV = std.bias(th)[1] + exp.bias(th)[1]
        th, p = D.theta_step(th, p, e["dUdl"], dl, dV, d["lambda_mass"], d["dt"], d["lambda_friction"],
                             d.get("lambda_temperature") or d["temperature"], D.theta_normal(step, SEED))
        if d["opes_stride"] and (step + 1) % d["opes_stride"] == 0:
            D.opes_dual_deposit(std, exp, th)
    oracle_steps.ti = ti
    return x, v, th, p, std, exp


def min_image(a, box):
    return a - box * np.round(a / box)


def octanol_system():
    # the octanol workload in small: 36 octanol-like chains (masses x 0.1,
    # X-H bonds constrained as stars, bonds/angles/torsions, 1-2/1-3
    # exclusions, scaled 1-4 pairs) around the frozen 20-atom solute,
    # 992 atoms in a 2.8 nm box, stepped at the octanol time step (1 fs)
    d = S.make_octanol_box(seed=31, n_chains=36, box_len=2.8, nx=6, ny=6, nz=2, r_cut=0.9, grid=24,
                           lam=0.55)
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=2,
             opes_dE_std=30 * 4.184, opes_dE_exp=5 * 4.184, opes_sigma=0.1)
    return d


@pytest.mark.parametrize("precision,tx,tv", [(lfe.LFE_FP64, 2e-8, 1e-6), (lfe.LFE_FP32_MIXED, 5e-6, 5e-3)])
def test_octanol_steps_match_oracle(precision, tx, tv):
    d = octanol_system()
    n = 4
    g = lfe.System(d, precision=precision, seed=SEED)
    g.step(n)
    pos, vel, ext = g.get_state()
    x, v, th, p, std, exp = oracle_steps(d, n)
    dx = np.abs(min_image(pos - x, d["box"])).max()
    assert dx < tx, dx
    assert np.abs(vel - v).max() < tv * np.abs(v).max()
    assert ext["step"] == n
    assert ext["n_kernels_std"] == len(std.c) and ext["n_kernels_exp"] == len(exp.c)
    assert ext["theta"] == pytest.approx(th, abs=1e-8 if precision == lfe.LFE_FP64 else 1e-5)


def test_kinetic_temperature_matches_the_thermostat():
    # Section 2.6: 298 K.  101 rigid waters (6 degrees of freedom each, the
    # solute frozen) stepped at 1 fs with friction 10 ps^-1: after 1 ps the
    # mean kinetic energy is 6/2 k_B T per water (equipartition)
    d = water_system()
    d.update(opes_stride=0)
    g = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    g.step(1000)
    kT = D.KB * d["temperature"]
    ke = []
    for _ in range(100):
        g.step(20)
        _, vel, _ = g.get_state()
        ke.append(0.5 * (d["mass"][:, None] * vel * vel).sum())
    n_w = len(d["waters"])
    assert np.mean(ke) == pytest.approx(3.0 * n_w * kT, rel=0.04)


@pytest.mark.parametrize("precision,tx,tv", [(lfe.LFE_FP64, 2e-8, 1e-6), (lfe.LFE_FP32_MIXED, 5e-6, 5e-3)])
def test_steps_match_oracle(precision, tx, tv):
    d = water_system()
    n = 4
    g = lfe.System(d, precision=precision, seed=SEED)
    g.step(n)
    pos, vel, ext = g.get_state()
    x, v, th, p, std, exp = oracle_steps(d, n)
    dx = np.abs(min_image(pos - x, d["box"])).max()
    assert dx < tx, dx
    vs = np.abs(v).max()
    assert np.abs(vel - v).max() < tv * vs
    assert ext["step"] == n
    assert ext["n_kernels_std"] == len(std.c) and ext["n_kernels_exp"] == len(exp.c)
    assert ext["theta"] == pytest.approx(th, abs=1e-8 if precision == lfe.LFE_FP64 else 1e-5)
    assert ext["p_theta"] == pytest.approx(p, rel=1e-6 if precision == lfe.LFE_FP64 else 2e-3, abs=1e-9)


@pytest.mark.parametrize("precision,tx", [(lfe.LFE_FP64, 2e-8), (lfe.LFE_FP32_MIXED, 5e-6)])
def test_hot_theta_steps_match_oracle(precision, tx):
    # lambda-d-AFED (Section 3.2): theta thermostatted at 5000 K with a heavy
    # mass, no OPES deposits; the atoms stay at the physical temperature
    d = water_system()
    d.update(lambda_temperature=5000.0, lambda_mass=1e4, opes_stride=0)
    n = 4
    g = lfe.System(d, precision=precision, seed=SEED)
    g.step(n)
    pos, vel, ext = g.get_state()
    x, v, th, p, std, exp = oracle_steps(d, n)
    assert np.abs(min_image(pos - x, d["box"])).max() < tx
    assert ext["n_kernels_std"] == 0 and ext["n_kernels_exp"] == 0
    assert ext["theta"] == pytest.approx(th, abs=1e-8 if precision == lfe.LFE_FP64 else 1e-5)
    assert ext["p_theta"] == pytest.approx(p, rel=1e-6 if precision == lfe.LFE_FP64 else 2e-3, abs=1e-9)
    # the same steps at the physical temperature move theta differently
    d2 = dict(d, lambda_temperature=0.0)
    _, _, th2, p2, _, _ = oracle_steps(d2, n)
    assert abs(p2 - p) > 1e-3 * abs(p)


def test_constraints_hold_after_many_steps():
    d = water_system()
    g = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    g.step(200)
    pos, vel, ext = g.get_state()
    w = d["waters"]
    for (o, h1, h2) in w:
        r1 = np.linalg.norm(min_image(pos[h1] - pos[o], d["box"]))
        r2 = np.linalg.norm(min_image(pos[h2] - pos[o], d["box"]))
        r3 = np.linalg.norm(min_image(pos[h2] - pos[h1], d["box"]))
        assert abs(r1 - 0.09572) < 1e-5 and abs(r2 - 0.09572) < 1e-5
        assert abs(r3 - 2 * 0.09572 * math.sin(math.radians(104.52) / 2)) < 2e-5
    assert 0.0 <= ext["theta"] < 2.0
    assert np.isfinite(vel).all()


def test_checkpoint_resume_is_bitwise(tmp_path):
    d = water_system()
    a = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    a.step(30)
    a.checkpoint(tmp_path / "c.bin")
    a.step(30)
    pa, va, ea = a.get_state()
    b = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    b.restore(tmp_path / "c.bin")
    b.step(30)
    pb, vb, eb = b.get_state()
    assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    assert ea["theta"] == eb["theta"] and ea["p_theta"] == eb["p_theta"]
    # a damaged checkpoint is refused
    raw = bytearray((tmp_path / "c.bin").read_bytes())
    raw[100] ^= 0xFF
    (tmp_path / "bad.bin").write_bytes(bytes(raw))
    with pytest.raises(lfe.LfeError):
        b.restore(tmp_path / "bad.bin")


@pytest.mark.parametrize("precision", [lfe.LFE_FP64, lfe.LFE_FP32_MIXED])
def test_forces_stay_exact_when_atoms_cross_the_box_between_builds(precision):
    # every atom moves 0.03 nm (< skin/2, so the list is kept) and the
    # positions are re-wrapped into the box, so the atoms next to the faces
    # jump by a box length; then a few steps follow.  The forces must stay
    # those of the oracle at the same positions.
    d = water_system()
    g = lfe.System(d, precision=precision, seed=SEED)
    box = d["box"]
    moved = S.f32(d["pos"] + np.array([0.03, -0.03, 0.03]))
    wrapped = S.f32(moved - box * np.floor(moved / box))
    wrapped[wrapped >= box] = 0.0
    assert np.any(np.floor(moved / box) != 0), "no atom crossed a face"
    g.set_positions(wrapped)
    lam = 0.45
    tol = 1e-9 if precision == lfe.LFE_FP64 else 1e-5
    t, F = g.eval(lam)
    o = R.evaluate(d, lam, level=2, pos=wrapped)
    assert np.linalg.norm(F - o["F"]) / np.linalg.norm(o["F"]) <= tol
    g.step(5)
    pos, _, _ = g.get_state()
    t, F = g.eval(lam)
    o = R.evaluate(d, lam, level=2, pos=pos)
    assert np.linalg.norm(F - o["F"]) / np.linalg.norm(o["F"]) <= tol


def test_ti_accumulators_match_oracle_and_survive_checkpoint(tmp_path):
    # the mean force of every step lands in the same lambda bin with the same
    # value as in the oracle's steps; a checkpoint carries the accumulators
    d = water_system()
    n = 4
    g = lfe.System(d, precision=lfe.LFE_FP64, seed=SEED)
    g.step(n)
    mean, count, dg = g.ti()
    oracle_steps(d, n)
    ti = oracle_steps.ti
    assert np.array_equal(count, ti.count.astype(float))
    occ = ti.count > 0
    om = ti.means()
    # the trajectories agree to ~1e-8 nm after these steps (test_steps_match_oracle),
    # so the sampled dU/dlambda agree to ~1e-7 relative
    assert np.all(np.abs(mean[occ] - om[occ]) <= 1e-6 * np.maximum(1.0, np.abs(om[occ])))
    assert np.all(np.isnan(mean[~occ]))
    assert dg == pytest.approx(ti.delta_g(), rel=1e-6, abs=1e-6)
    path = tmp_path / "ti.ckpt"
    g.checkpoint(path)
    g2 = lfe.System(d, precision=lfe.LFE_FP64, seed=SEED)
    g2.restore(path)
    mean2, count2, dg2 = g2.ti(reset=True)
    assert np.array_equal(count2, count) and dg2 == dg
    _, count3, _ = g2.ti()
    assert count3.sum() == 0


@pytest.mark.parametrize("precision", [lfe.LFE_FP64, lfe.LFE_FP32_MIXED])
def test_eval_after_a_step_rebuilds_the_pending_list(precision):
    # a step rebuilds the neighbour list at its start when the step before
    # left an atom more than skin/2 from the build positions, so the last
    # step of a call can leave a rebuild pending; an evaluation after it
    # rebuilds first, and its forces are the oracle's at the current positions
    d = water_system()
    g = lfe.System(d, precision=precision, seed=SEED)
    lam = 0.4
    tol = 1e-9 if precision == lfe.LFE_FP64 else 1e-5
    seen = 0
    for _ in range(400):
        g.step(1)
        pos, _, e0 = g.get_state()
        t, F = g.eval(lam)
        _, _, e1 = g.get_state()
        if e1["n_rebuilds"] > e0["n_rebuilds"]:
            seen += 1
            o = R.evaluate(d, lam, level=2, pos=pos)
            assert np.linalg.norm(F - o["F"]) / np.linalg.norm(o["F"]) <= tol
            if seen == 2:
                break
    assert seen == 2, "no rebuild was left pending by a step"
