"""Neighbour-list overflow recovery on the GPU: a list capacity far below what
the system needs (lfe_set_list_capacity) makes the rebuilds inside captured
steps overflow; the skipped steps are replayed after the list grows, and the
results equal those of an uncapped system.  The overflow is a host-visible
flag set by the build kernels, which never write past the capacity."""
import numpy as np
import pytest

from oracle import reference as R
from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

SEED = 5


def water_system():
    d = S.make_water_box(seed=21, n_waters=101, box_len=1.45, solute="ring12", n_side=5,
                         r_cut=0.7, grid=16, lam=0.62)
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=2,
             opes_dE_std=30 * 4.184, opes_dE_exp=5 * 4.184, opes_sigma=0.1)
    return d


@pytest.mark.parametrize("n_steps", [40, 150])
def test_overflowing_steps_replay_to_the_uncapped_trajectory(n_steps):
    d = water_system()
    ref = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    ref.step(n_steps)
    p0, v0, e0 = ref.get_state()
    g = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    g.set_list_capacity(8)
    g.step(n_steps)
    p1, v1, e1 = g.get_state()
    assert e1["step"] == n_steps
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1)
    assert e1["theta"] == e0["theta"] and e1["p_theta"] == e0["p_theta"]
    assert e1["n_kernels_std"] == e0["n_kernels_std"]


def test_small_capacity_eval_and_far_move_match_oracle():
    d = water_system()
    g = lfe.System(d, precision=lfe.LFE_FP32_MIXED)
    with pytest.raises(lfe.LfeError) as e:
        g.set_list_capacity(0)
    assert e.value.code == lfe.LFE_ERR_ARG
    for pos in (d["pos"], S.f32(np.mod(d["pos"] + 0.31, d["box"]))):
        g.set_list_capacity(4)
        g.set_positions(pos)
        terms, F = g.eval(0.7)
        E, F0, Fuv, Fs = R.nonbonded(dict(d, pos=pos), level=2)
        hA, hB, _, _ = R.switching(0.7)
        Fo = F0 + hA * Fuv + hB * Fs
        assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) < 1e-5
        assert terms["n_pairs"] == pytest.approx(E["n_pairs"], abs=2)
