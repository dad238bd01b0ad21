"""Soft-core coupling on the GPU (sc_alpha > 0: the Beutler form of the
solute-solvent LJ at lambda, Coulomb under h_A) against the oracle's same
option: forces, U and dU/dlambda of both precision modes at lambdas across
[0, 1] on the plain FP64 workload (alpha = 0.5, p = 1) and the small water
box; captured steps of atoms and theta (driven by the soft-core dU/dlambda)
against the oracle's steps; and the refusals of the calls that need the
linear basis."""
import numpy as np
import pytest

from oracle import dynamics as D
from oracle import reference as R
from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

TOL = {lfe.LFE_FP32_MIXED: dict(F=1e-5, dU=1e-6, U=1e-6), lfe.LFE_FP64: dict(F=1e-9, dU=1e-8, U=1e-9)}


def with_sc(d):
    d = dict(d)
    d["sc_alpha"], d["sc_power"] = 0.5, 1.0
    return d


def small_water():
    return S.make_water_box(seed=21, n_waters=101, box_len=1.45, solute="ring12", n_side=5,
                            r_cut=0.7, grid=16, lam=0.62)


@pytest.mark.parametrize("precision", [lfe.LFE_FP64, lfe.LFE_FP32_MIXED])
@pytest.mark.parametrize("make", [S.make_c0, small_water])
def test_softcore_evaluation_matches_oracle(make, precision):
    d = with_sc(make())
    g = lfe.System(d, precision=precision)
    tol = TOL[precision]
    for lam in (0.0, 0.2, 0.5, 0.8, 1.0):
        terms, F = g.eval(lam)
        o = R.evaluate(d, lam, level=2)
        rel = np.linalg.norm(F - o["F"]) / np.linalg.norm(o["F"])
        assert rel <= tol["F"], (lam, rel)
        E = o["E"]
        scale = abs(o["dhA"] * E["U_uv"]) + abs(E["dUsc_dl"]) + 1e-12
        assert abs(terms["dUdl"] - o["dUdl"]) <= tol["dU"] * max(abs(o["dUdl"]), scale), (lam, terms["dUdl"], o["dUdl"])
        assert terms["U_soft"] == pytest.approx(E["U_soft"], rel=tol["U"], abs=tol["U"] * 10)
        mag = sum(abs(E[k]) for k in ("coul_real_vv", "rec_vv", "self_vv", "excl_vv", "lj_vv", "coul_real_uv",
                                      "rec_uv", "bg_uv"))
        assert abs(terms["U"] - o["U"]) <= tol["U"] * mag, (lam, terms["U"], o["U"])


@pytest.mark.parametrize("precision,tx", [(lfe.LFE_FP64, 2e-8), (lfe.LFE_FP32_MIXED, 5e-6)])
def test_softcore_steps_match_oracle(precision, tx):
    seed = 77
    d = with_sc(small_water())
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=0)
    n = 4
    g = lfe.System(d, precision=precision, seed=seed)
    g.step(n)
    pos, vel, ext = g.get_state()
    pairs, lens = D.constraint_list(d)
    x, v = d["pos"].copy(), np.zeros_like(d["pos"])
    th, p = d["lam"], 0.0
    for step in range(n):
        lam, dl = D.theta_to_lambda(th)
        e = R.evaluate(d, lam, level=2, pos=x)
        x, v = D.langevin_middle_step(x, v, e["F"], d["mass"], d["dt"], d["friction"], d["temperature"],
                                      D.atom_normals(len(x), step, seed), d["box"], pairs, lens)
        th, p = D.theta_step(th, p, e["dUdl"], dl, 0.0, d["lambda_mass"], d["dt"], d["lambda_friction"],
                             d["temperature"], D.theta_normal(step, seed))
    dx = pos - x
    dx -= d["box"] * np.round(dx / d["box"])
    assert np.abs(dx).max() < tx
    assert ext["theta"] == pytest.approx(th, abs=1e-8 if precision == lfe.LFE_FP64 else 1e-5)


def test_softcore_refuses_linear_basis_calls():
    d = with_sc(small_water())
    g = lfe.System(d, precision=lfe.LFE_FP64)
    with pytest.raises(lfe.LfeError) as e:
        g.param_grad(0.5)
    assert e.value.code == lfe.LFE_ERR_STATE
    d2 = dict(d, lambda_mass=0.0)
    a = lfe.System(dict(d2, lam=0.3), precision=lfe.LFE_FP64, theta0=0.3)
    b = lfe.System(dict(d2, lam=0.7), precision=lfe.LFE_FP64, theta0=0.7)
    batch = lfe.Batch([a, b])
    with pytest.raises(lfe.LfeError) as e:
        batch.exchange([0, 1], 298.0, 1, 0)
    assert e.value.code == lfe.LFE_ERR_STATE
    bad = dict(d, sc_power=0.5)
    with pytest.raises(lfe.LfeError) as e:
        lfe.System(bad)
    assert e.value.code == lfe.LFE_ERR_ARG
