"""Lambda replica exchange on the GPU (lfe_batch_exchange) against the
oracle's Metropolis attempts on the same configurations."""
import numpy as np
import pytest

from oracle import dynamics as D
from oracle import reference as R
from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

LAMS = [0.3, 0.55, 0.7, 0.9]
T, SEED = 298.0, 31


def replicas(noise=0.004):
    d0 = S.make_water_box(seed=21, n_waters=101, box_len=1.45, solute="ring12", n_side=5, r_cut=0.7, grid=16)
    rng = np.random.default_rng(9)
    out = []
    for k, lam in enumerate(LAMS):
        d = dict(d0, pos=S.f32(d0["pos"] + rng.normal(0.0, noise, d0["pos"].shape)), lam=lam, lambda_mass=0.0)
        out.append(d)
    return out


def test_exchange_matches_oracle_attempts():
    ds = replicas()
    gs = [lfe.System(d, precision=lfe.LFE_FP64, theta0=d["lam"]) for d in ds]
    b = lfe.Batch(gs)
    E = [R.nonbonded(d, level=2)[0] for d in ds]
    ladder = np.arange(len(gs))
    lam_of = {k: LAMS[k] for k in range(len(gs))}      # replica -> lambda
    n_acc = n_rej = 0
    for attempt in range(8):
        order = list(ladder)
        acc_o, new_o = D.hrex_attempt([lam_of[r] for r in order], [E[r]["U_uv"] for r in order],
                                      [E[r]["U_soft"] for r in order], T, SEED, attempt)
        ladder, acc = b.exchange(ladder, T, SEED, attempt)
        assert list(acc) == acc_o
        for pos, r in enumerate(order):
            lam_of[r] = new_o[pos]
        for r, g in enumerate(gs):
            assert g.get_state()[2]["lambda"] == pytest.approx(lam_of[r], abs=1e-15)
        assert [lam_of[r] for r in ladder] == sorted(LAMS)
        tried = range(attempt % 2, len(gs) - 1, 2)
        n_acc += sum(acc_o[k] for k in tried)
        n_rej += sum(1 - acc_o[k] for k in tried)
    assert n_acc > 0 and n_rej > 0
    # an evaluation at a replica's new lambda
    t, F = gs[0].eval(lam_of[0])
    assert np.isfinite(F).all()
    b.close()
    for g in gs:
        g.close()


def test_exchange_rejects_bad_ladders():
    ds = replicas()[:2]
    gs = [lfe.System(d, precision=lfe.LFE_FP32_MIXED, theta0=d["lam"]) for d in ds]
    b = lfe.Batch(gs)
    with pytest.raises(lfe.LfeError):
        b.exchange([1, 0], T, SEED, 0)          # not in lambda order
    with pytest.raises(lfe.LfeError):
        b.exchange([0, 0], T, SEED, 0)          # repeated replica
    b.close()
    for g in gs:
        g.close()
    d = dict(ds[0], lambda_mass=20.0)
    g1 = lfe.System(d, theta0=0.3)
    g2 = lfe.System(ds[1], theta0=0.55)
    b = lfe.Batch([g1, g2])
    with pytest.raises(lfe.LfeError):
        b.exchange([0, 1], T, SEED, 0)          # dynamical theta
    b.close()
    g1.close()
    g2.close()


def test_device_exchange_inside_batch_steps_matches_oracle():
    # lfe_batch_set_exchange: an attempt after every batch step, decided on
    # the device from each replica's configuration after the step; the
    # oracle's attempt on the same configurations gives the same swaps
    ds = [dict(d, dt=0.001) for d in replicas()]
    gs = [lfe.System(d, precision=lfe.LFE_FP64, theta0=d["lam"], seed=100 + k) for k, d in enumerate(ds)]
    b = lfe.Batch(gs)
    ladder = list(range(len(gs)))
    lam_of = {k: LAMS[k] for k in range(len(gs))}
    b.set_exchange(ladder, T, SEED, 1)
    n_acc = n_rej = 0
    for attempt in range(6):
        b.step(1)
        pos = [g.get_state()[0] for g in gs]
        E = [R.nonbonded(dict(d, pos=p), level=2)[0] for d, p in zip(ds, pos)]
        order = list(ladder)
        acc_o, new_o = D.hrex_attempt([lam_of[r] for r in order], [E[r]["U_uv"] for r in order],
                                      [E[r]["U_soft"] for r in order], T, SEED, attempt)
        for p_, r in enumerate(order):
            lam_of[r] = new_o[p_]
        for k, a in enumerate(acc_o):
            if a:
                ladder[k], ladder[k + 1] = ladder[k + 1], ladder[k]
        lad_dev, attempts, acc = b.exchange_state()
        assert attempts == attempt + 1
        assert list(lad_dev) == ladder
        for r, g in enumerate(gs):
            assert g.get_state()[2]["lambda"] == pytest.approx(lam_of[r], abs=1e-15)
        tried = range(attempt % 2, len(gs) - 1, 2)
        n_acc += sum(acc_o[k] for k in tried)
        n_rej += sum(1 - acc_o[k] for k in tried)
    assert n_acc > 0 and n_rej > 0
    b.set_exchange(ladder, T, SEED, 0)      # off: plain batch steps again, no more attempts
    b.step(2)
    assert b.exchange_state()[1] == 6
    b.close()
    for g in gs:
        g.close()
