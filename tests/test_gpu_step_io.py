"""The fused host-I/O step (lfe_step_io) against the three calls it stands
for: lfe_set_positions from host memory, lfe_step(1) and lfe_get_state, on
identical systems with the same seed -- positions, velocities and the scalar
state equal bit for bit after every step, also when the device keeps its own
positions (pos_in NULL) and when the neighbour list overflows inside the
step.  Host buffers that are not page-locked are refused."""
import numpy as np
import pytest

from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

SEED = 31


def water_system():
    d = S.make_water_box(seed=21, n_waters=101, box_len=1.45, solute="ring12", n_side=5,
                         r_cut=0.7, grid=16, lam=0.62)
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=4,
             opes_dE_std=30 * 4.184, opes_dE_exp=5 * 4.184, opes_sigma=0.1)
    return d


def pinned(shape):
    import torch
    return torch.zeros(shape, dtype=torch.float64).pin_memory()


@pytest.mark.parametrize("feed_positions,capacity", [(True, None), (False, None), (True, 8)])
def test_step_io_equals_the_three_calls(feed_positions, capacity):
    import torch
    d = water_system()
    n = len(d["charge"])
    a = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    b = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    if capacity:
        a.set_list_capacity(capacity)
        b.set_list_capacity(capacity)
    pa, va, ea = pinned((n, 3)), pinned((n, 3)), pinned(lfe.NEXT)
    pb, vb = pinned((n, 3)), pinned((n, 3))
    eb = np.zeros(lfe.NEXT)
    pa.copy_(torch.from_numpy(np.asarray(d["pos"], dtype=np.float64)))
    pb.copy_(pa)
    for _ in range(30):
        if feed_positions:
            a.set_positions_ptr(pa.data_ptr(), 0)
        a.step(1)
        a.get_state_into(pa.data_ptr(), va.data_ptr(), ea.data_ptr())
        b.step_io(pb.data_ptr() if feed_positions else None, pb.data_ptr(), vb.data_ptr(), eb.ctypes.data)
        assert torch.equal(pa, pb) and torch.equal(va, vb)
        assert np.array_equal(ea.numpy(), eb)
    assert eb[7] == 30      # step counter


def test_step_io_refuses_pageable_buffers_and_bad_positions():
    import torch
    d = water_system()
    n = len(d["charge"])
    g = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    pos = np.ascontiguousarray(d["pos"], dtype=np.float64)
    with pytest.raises(lfe.LfeError) as e:
        g.step_io(pos.ctypes.data, None, None, None)
    assert e.value.code == lfe.LFE_ERR_ARG
    p = pinned((n, 3))
    p.copy_(torch.from_numpy(pos))
    p[5, 2] = float("nan")
    with pytest.raises(lfe.LfeError) as e:
        g.step_io(p.data_ptr(), None, None, None)
    assert e.value.code == lfe.LFE_ERR_ARG
    # the system is unchanged and still steps
    _, _, ext = g.get_state()
    assert ext["step"] == 0
    g.step_io(None, None, None, None)
    assert g.get_state()[2]["step"] == 1


def test_refused_positions_leave_the_trajectory_as_it_was():
    # positions are checked on the device inside the captured step: a call
    # with a non-finite coordinate changes nothing, so a run with one refused
    # call in its middle equals a run without it, bit for bit
    import torch
    d = water_system()
    n = len(d["charge"])
    a = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    b = lfe.System(d, precision=lfe.LFE_FP32_MIXED, seed=SEED)
    pa, va, pb, vb = pinned((n, 3)), pinned((n, 3)), pinned((n, 3)), pinned((n, 3))
    bad = pinned((n, 3))
    ea, eb = np.zeros(lfe.NEXT), np.zeros(lfe.NEXT)
    pa.copy_(torch.from_numpy(np.asarray(d["pos"], dtype=np.float64)))
    pb.copy_(pa)
    for k in range(12):
        if k == 6:
            bad.copy_(pa)
            bad[17, 0] = float("inf")
            with pytest.raises(lfe.LfeError) as e:
                a.step_io(bad.data_ptr(), None, None, None)
            assert e.value.code == lfe.LFE_ERR_ARG
        a.step_io(pa.data_ptr(), pa.data_ptr(), va.data_ptr(), ea.ctypes.data)
        b.step_io(pb.data_ptr(), pb.data_ptr(), vb.data_ptr(), eb.ctypes.data)
        assert torch.equal(pa, pb) and torch.equal(va, vb)
        assert np.array_equal(ea, eb)
    assert eb[7] == 12


@pytest.mark.parametrize("precision,capacity", [(lfe.LFE_FP32_MIXED, None), (lfe.LFE_FP32_MIXED, 8),
                                                (lfe.LFE_FP64, None)])
def test_float_host_buffers_step_as_the_doubles(precision, capacity):
    # lfe_step_io_f32 fed the same floats as lfe_step_io gets widened to
    # double: the same trajectory, outputs equal to the doubles rounded to
    # float (exactly the doubles for an FP32 system, whose state is float)
    import torch
    d = water_system()
    n = len(d["charge"])
    a = lfe.System(d, precision=precision, seed=SEED)
    b = lfe.System(d, precision=precision, seed=SEED)
    if capacity:
        a.set_list_capacity(capacity)
        b.set_list_capacity(capacity)
    pa, va = pinned((n, 3)), pinned((n, 3))
    pin32 = torch.zeros((n, 3), dtype=torch.float32).pin_memory()
    pb, vb = (torch.zeros((n, 3), dtype=torch.float32).pin_memory() for _ in range(2))
    ea, eb = np.zeros(lfe.NEXT), np.zeros(lfe.NEXT)
    pin32.copy_(torch.from_numpy(np.asarray(d["pos"], dtype=np.float32)))
    for k in range(25):
        pa.copy_(pin32.double())
        feed = k % 5 != 4          # every fifth step keeps the device positions
        a.step_io(pa.data_ptr() if feed else None, pa.data_ptr(), va.data_ptr(), ea.ctypes.data)
        b.step_io_f32(pin32.data_ptr() if feed else None, pb.data_ptr(), vb.data_ptr(), eb.ctypes.data)
        assert torch.equal(pb, pa.float()) and torch.equal(vb, va.float())
        if precision == lfe.LFE_FP32_MIXED:
            assert torch.equal(pb.double(), pa) and torch.equal(vb.double(), va)
        assert np.array_equal(ea, eb)
        pin32.copy_(pb)
    assert eb[7] == 25
    # refusals as for the doubles
    pin32[3, 1] = float("inf")
    with pytest.raises(lfe.LfeError) as e:
        b.step_io_f32(pin32.data_ptr(), pb.data_ptr(), None, None)
    assert e.value.code == lfe.LFE_ERR_ARG
    assert b.get_state()[2]["step"] == 25
    with pytest.raises(lfe.LfeError):
        b.step_io_f32(np.zeros(3 * n, dtype=np.float32).ctypes.data, None, None, None)
