"""Dynamic pruning of the neighbour list (lfe_set_list_prune): the step's
pair kernel runs on a list cut from the built one, and every pair within the
cutoff is still evaluated -- the pair count of each pruned step equals the
count of the built list at the same positions, exactly -- while the pruned
list is shorter.  Trajectories follow the unpruned ones to rounding order,
the host-I/O step prunes like lfe_step, and buffers that cannot prune
switch the pruning off."""
import numpy as np
import pytest

from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

SEED = 17


def octanol_system():
    # 36 octanol-like chains (X-H stars, bonded terms, scaled 1-4 pairs) around
    # the frozen 20-atom solute: 992 atoms, 2.8 nm box, r_cut 0.9 nm, 1 fs
    d = S.make_octanol_box(seed=31, n_chains=36, box_len=2.8, nx=6, ny=6, nz=2, r_cut=0.9, grid=24,
                           lam=0.55)
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=4,
             opes_dE_std=30 * 4.184, opes_dE_exp=5 * 4.184, opes_sigma=0.1)
    return d


def water_system():
    d = S.make_water_box(seed=21, n_waters=101, box_len=1.45, solute="ring12", n_side=5,
                         r_cut=0.7, grid=16, lam=0.62)
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=4,
             opes_dE_std=30 * 4.184, opes_dE_exp=5 * 4.184, opes_sigma=0.1)
    return d


@pytest.mark.parametrize("precision", [lfe.LFE_FP32_MIXED, lfe.LFE_FP64])
@pytest.mark.parametrize("make", [octanol_system, water_system])
def test_pruned_steps_count_every_pair_in_range(precision, make):
    # before each step an evaluation counts the pairs within r_cut on the
    # built list at the step's positions; the step's own count (its pair
    # kernel on the pruned list) must be the same number
    d = make()
    g = lfe.System(d, precision=precision, seed=SEED, skin=0.2)
    g.set_list_prune(0.03)   # pruned again every few steps
    pruned_tiles = set()
    for k in range(40):
        t, _ = g.eval(0.5, forces=False)
        g.step(1)
        _, _, e = g.get_state()
        assert e["n_pairs_step"] == t["n_pairs"], (k, e["n_pairs_step"], t["n_pairs"])
        assert 0 < e["n_tiles_pruned"] < e["n_tiles"]
        pruned_tiles.add(e["n_tiles_pruned"])
    assert len(pruned_tiles) > 1      # the list was cut again along the way
    assert e["step"] == 40


@pytest.mark.parametrize("precision,tol", [(lfe.LFE_FP32_MIXED, 2e-4), (lfe.LFE_FP64, 1e-9)])
def test_pruned_trajectory_follows_the_full_list(precision, tol):
    d = octanol_system()
    a = lfe.System(d, precision=precision, seed=SEED, skin=0.2)
    b = lfe.System(d, precision=precision, seed=SEED, skin=0.2)
    a.set_list_prune(0.05)
    a.step(30)
    b.step(30)
    pa, va, ea = a.get_state()
    pb, vb, eb = b.get_state()
    box = np.asarray(d["box"])
    dx = pa - pb
    dx -= box * np.round(dx / box)
    assert np.abs(dx).max() < tol
    assert abs(ea["theta"] - eb["theta"]) < 1e3 * tol
    assert ea["step"] == eb["step"] == 30
    assert ea["n_tiles_pruned"] < ea["n_tiles"] and eb["n_tiles_pruned"] == 0


def test_host_io_step_prunes_like_step():
    import torch
    d = water_system()
    n = len(d["charge"])
    a = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED, skin=0.2)
    b = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED, skin=0.2)
    a.set_list_prune(0.03)
    b.set_list_prune(0.03)
    pa, va = (torch.zeros((n, 3), dtype=torch.float64).pin_memory() for _ in range(2))
    pb, vb = (torch.zeros((n, 3), dtype=torch.float64).pin_memory() for _ in range(2))
    ea, eb = np.zeros(lfe.NEXT), np.zeros(lfe.NEXT)
    pb.copy_(torch.from_numpy(np.asarray(d["pos"], dtype=np.float64)))
    for _ in range(25):
        a.set_positions_ptr(pb.data_ptr(), 0)
        a.step(1)
        a.get_state_into(pa.data_ptr(), va.data_ptr(), ea.ctypes.data)
        b.step_io(pb.data_ptr(), pb.data_ptr(), vb.data_ptr(), eb.ctypes.data)
        assert torch.equal(pa, pb) and torch.equal(va, vb)
        assert np.array_equal(ea, eb)
    assert 0 < eb[11] < eb[9]


def test_buffers_that_cannot_prune_switch_it_off():
    d = water_system()
    g = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED, skin=0.1)
    with pytest.raises(lfe.LfeError) as e:
        g.set_list_prune(-0.01)
    assert e.value.code == lfe.LFE_ERR_ARG
    g.set_list_prune(0.1)     # not below the list buffer: no pruning
    g.step(5)
    assert g.get_state()[2]["n_tiles_pruned"] == 0
    g.set_list_prune(0.05)
    g.step(5)
    _, _, e = g.get_state()
    assert 0 < e["n_tiles_pruned"] <= e["n_tiles"]
    g.set_list_prune(0.0)     # off again: the step runs on the built list
    t, _ = g.eval(0.5, forces=False)
    g.step(1)
    assert g.get_state()[2]["n_pairs_step"] == t["n_pairs"]


def test_batched_replicas_prune_like_single_systems():
    # the batch's shared pair launch runs on each replica's pruned list: every
    # replica ends bit-identical to the same system stepped alone with pruning
    def replica(seed, nw, side, box, lam, prec):
        d = S.make_water_box(seed=seed, n_waters=nw, box_len=box, solute="ring12", n_side=side,
                             r_cut=0.7, grid=16, lam=lam)
        d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=5,
                 opes_dE_std=30 * 4.184, opes_dE_exp=5 * 4.184, opes_sigma=0.1)
        g = lfe.System(d, precision=prec, seed=seed, skin=0.2)
        g.set_list_prune(0.03)
        return g
    specs = [(31, 101, 5, 1.45, 0.2, lfe.LFE_FP32_MIXED), (32, 180, 6, 1.75, 0.55, lfe.LFE_FP32_MIXED),
             (33, 101, 5, 1.45, 0.9, lfe.LFE_FP64)]
    batched = [replica(*sp) for sp in specs]
    alone = [replica(*sp) for sp in specs]
    b = lfe.Batch(batched)
    b.step(30)
    for s in alone:
        s.step(30)
    for sb, sa in zip(batched, alone):
        pb, vb, eb = sb.get_state()
        pa, va, ea = sa.get_state()
        assert np.array_equal(pb, pa) and np.array_equal(vb, va)
        assert eb["theta"] == ea["theta"] and eb["step"] == ea["step"] == 30
        assert eb["n_prunes"] == ea["n_prunes"] > 1
        assert 0 < eb["n_tiles_pruned"] < eb["n_tiles"]
    b.close()
