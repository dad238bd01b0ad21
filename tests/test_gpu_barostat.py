"""Monte Carlo barostat on the GPU (lfe_mc_volume_move) against the oracle's
volume moves (oracle/barostat.py) with the same Philox uniforms: the same
accept/reject decisions, the same boxes and scaled positions, and energies
equal to the level-2 oracle at the old and the proposed state; after a move
the forces match the oracle in the new box, and a rejected move leaves the
system as it was.  Checkpoints carry the box."""
import math

import numpy as np
import pytest

from oracle import barostat as B
from oracle import dynamics as D
from oracle import reference as R
from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

SEED = 4044


def water_system():
    # 101 rigid waters around a frozen 12-atom ring (a massless molecule) in a
    # 1.45 nm box, cutoff 0.7 nm: r_cut stays below half the box for the moves
    d = S.make_water_box(seed=21, n_waters=101, box_len=1.45, solute="ring12", n_side=5,
                         r_cut=0.7, grid=16, lam=0.62)
    d.update(dt=0.001, opes_stride=0)
    return d


def oracle_energy(d, lam):
    return lambda pos, box: R.evaluate(dict(d, box=np.asarray(box, dtype=np.float64)), lam, level=2, pos=pos)["U"]


@pytest.mark.parametrize("precision,tx,te", [(lfe.LFE_FP64, 1e-10, 1e-9), (lfe.LFE_FP32_MIXED, 2e-6, 1e-5)])
def test_volume_moves_match_the_oracle(precision, tx, te):
    d = water_system()
    lam = d["lam"]
    g = lfe.System(d, precision=precision)
    mass = np.asarray(d["mass"], dtype=np.float64)
    mol = B.molecule_ids(len(d["charge"]), d["excl"])
    n_mol = int(np.unique(mol).size)
    kT = D.KB * d["temperature"]
    x = np.asarray(d["pos"], dtype=np.float64)
    box = np.asarray(d["box"], dtype=np.float64)
    energy = oracle_energy(d, lam)
    U = energy(x, box)
    seen = set()
    for attempt, (p_bar, dv) in enumerate([(1.0, 0.02), (1.0, 0.02), (3000.0, 0.05), (-3000.0, 0.05),
                                           (1.0, 0.3), (1.0, 0.02)]):
        acc, box_g, (u0, u1) = g.mc_volume_move(p_bar, dv, SEED, attempt)
        # the oracle's move with the same uniforms, step by step
        u = D.uniforms((attempt & 0xFFFFFFFF, attempt >> 32, 0, 4), D.seed_key(SEED))
        V = float(np.prod(box))
        Vn = V + dv * (2.0 * u[0] - 1.0)
        x_new, box_new = B.scale_molecules(x, mass, mol, box, (Vn / V) ** (1.0 / 3.0))
        U_new = energy(x_new, box_new)
        p = B.accept_probability(U_new - U, p_bar * B.BAR, V, Vn, n_mol, kT)
        acc_o = u[1] < p
        assert u0 == pytest.approx(U, rel=te, abs=te * 1e3)
        assert u1 == pytest.approx(U_new, rel=te, abs=te * 1e3)
        assert abs(p - u[1]) > 1e-3, "decision too close to call at this precision"
        assert acc == acc_o, (attempt, acc, acc_o, p, u[1])
        seen.add(acc)
        if acc_o:
            x, box, U = x_new, box_new, U_new
        assert np.allclose(box_g, box, rtol=1e-14, atol=0)
        pos, _, _ = g.get_state()
        dx = pos - x
        dx -= box * np.round(dx / box)
        assert np.abs(dx).max() < tx, (attempt, np.abs(dx).max())
    assert seen == {True, False}
    # forces in the final box against the oracle
    terms, F = g.eval(lam)
    o = R.evaluate(dict(d, box=box), lam, level=2, pos=x)
    assert np.linalg.norm(F - o["F"]) / np.linalg.norm(o["F"]) < (1e-9 if precision == lfe.LFE_FP64 else 1e-5)


def test_rejected_move_restores_state_and_box_survives_checkpoint(tmp_path):
    d = water_system()
    g = lfe.System(d, precision=lfe.LFE_FP64)
    p0, v0, _ = g.get_state()
    t0, F0 = g.eval(d["lam"])
    # a huge pressure against an expansion, or a huge negative one against a
    # compression: find an attempt whose proposal is rejected
    for attempt in range(20):
        u = D.uniforms((attempt, 0, 0, 4), D.seed_key(SEED))
        if u[0] > 0.5:
            break
    acc, box, _ = g.mc_volume_move(1e6, 0.05, SEED, attempt)
    assert not acc and np.array_equal(box, np.asarray(d["box"], dtype=np.float64))
    p1, v1, _ = g.get_state()
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1)
    t1, F1 = g.eval(d["lam"])
    assert t1["U"] == pytest.approx(t0["U"], rel=1e-12) and np.allclose(F1, F0, rtol=0, atol=1e-9)
    # an accepted move (negative pressure favours the expansion), then a checkpoint
    acc, box, _ = g.mc_volume_move(-1e6, 0.05, SEED, attempt)
    assert acc and box[0] > d["box"][0]
    g.checkpoint(tmp_path / "npt.ckpt")
    t2, F2 = g.eval(d["lam"])
    h = lfe.System(d, precision=lfe.LFE_FP64)
    h.restore(tmp_path / "npt.ckpt")
    t3, F3 = h.eval(d["lam"])
    assert t3["U"] == pytest.approx(t2["U"], rel=1e-12)
    assert np.allclose(F3, F2, rtol=0, atol=1e-8)
