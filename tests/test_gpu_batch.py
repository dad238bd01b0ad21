"""Batched replicas: one graph launch per step advances several systems of
different sizes and precisions; every replica must end bit-identical to the
same system stepped on its own, and batched evaluation must equal single
evaluation."""
import numpy as np
import pytest

from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu


def replica(seed, n_waters, side, box, lam):
    d = S.make_water_box(seed=seed, n_waters=n_waters, box_len=box, solute="ring12", n_side=side,
                         r_cut=0.7, grid=16, lam=lam)
    d.update(dt=0.001, lambda_mass=20.0, lambda_friction=25.0, opes_stride=5,
             opes_dE_std=30 * 4.184, opes_dE_exp=5 * 4.184, opes_sigma=0.1)
    return d


SPECS = [(31, 101, 5, 1.45, 0.2, lfe.LFE_FP32_MIXED),
         (32, 180, 6, 1.75, 0.55, lfe.LFE_FP32_MIXED),
         (33, 101, 5, 1.45, 0.9, lfe.LFE_FP64)]


def make(spec):
    seed, nw, side, box, lam, prec = spec
    return lfe.System(replica(seed, nw, side, box, lam), precision=prec, seed=seed)


def test_batch_steps_match_single_systems():
    batched = [make(sp) for sp in SPECS]
    alone = [make(sp) for sp in SPECS]
    b = lfe.Batch(batched)
    b.step(30)
    b.step(20)
    for s in alone:
        s.step(50)
    for sb, sa in zip(batched, alone):
        pb, vb, eb = sb.get_state()
        pa, va, ea = sa.get_state()
        assert np.array_equal(pb, pa) and np.array_equal(vb, va)
        assert eb["theta"] == ea["theta"] and eb["step"] == ea["step"] == 50
        assert eb["n_kernels_std"] == ea["n_kernels_std"] == 10


def test_batch_eval_matches_single_eval():
    batched = [make(sp) for sp in SPECS]
    b = lfe.Batch(batched)
    lams = [0.1, 0.45, 0.8]
    terms = b.eval(lams)
    for s, lam, t in zip([make(sp) for sp in SPECS], lams, terms):
        ts, _ = s.eval(lam)
        for k in ("U", "dUdl", "U_uv", "U_soft", "n_pairs"):
            assert t[k] == ts[k]
