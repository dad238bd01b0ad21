"""The autotuner (lfe_autotune): chosen launch shapes are valid, the state is
left as it was, results stay within the precision mode's tolerance, and the
JSON cache returns the same choice for a system of the same kind."""
import json

import numpy as np
import pytest

from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu


def test_autotune_keeps_state_and_results(tmp_path):
    d = S.make_c2(seed=77)
    lam = 0.6
    g = lfe.System(d, precision=lfe.LFE_FP32_MIXED)
    t0, F0 = g.eval(lam)
    p0, v0, e0 = g.get_state()
    cache = tmp_path / "tune.json"
    ms, par = g.autotune(reps=5, cache_path=cache)
    assert ms > 0 and par["from_cache"] == 0
    assert 1 <= par["pair_blocks_per_sm"] <= 8
    assert par["uv_blocks"] >= 1 and par["df64_lines"] in (4, 16)
    p1, v1, e1 = g.get_state()
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1)
    assert e1["step"] == e0["step"] and e1["theta"] == e0["theta"]
    t1, F1 = g.eval(lam)
    assert np.linalg.norm(F1 - F0) / np.linalg.norm(F0) < 1e-6
    assert abs(t1["dUdl"] - t0["dUdl"]) <= 1e-9 * max(abs(t0["dUdl"]), 1.0)
    assert abs(t1["U"] - t0["U"]) <= 1e-7 * max(abs(t0["U"]), 1.0)
    assert t1["n_pairs"] == t0["n_pairs"]
    # the step graph is recaptured with the chosen shapes
    g.step(3)
    p2, _, e2 = g.get_state()
    assert np.isfinite(p2).all() and e2["step"] == e0["step"] + 3
    g.close()
    entries = json.loads(cache.read_text())["entries"]
    assert len(entries) == 1 and entries[0]["pair_blocks_per_sm"] == par["pair_blocks_per_sm"]
    # a system of the same kind takes the cached choice without timing
    h = lfe.System(S.make_c2(seed=78), precision=lfe.LFE_FP32_MIXED)
    ms2, par2 = h.autotune(reps=5, cache_path=cache)
    assert par2["from_cache"] == 1 and ms2 == pytest.approx(ms, rel=1e-5)
    assert {k: par2[k] for k in ("pair_blocks_per_sm", "uv_blocks", "df64_lines")} == \
        {k: par[k] for k in ("pair_blocks_per_sm", "uv_blocks", "df64_lines")}
    h.close()


def test_autotune_rejects_bad_reps():
    g = lfe.System(S.make_c0(), precision=lfe.LFE_FP32_MIXED)
    with pytest.raises(lfe.LfeError):
        g.autotune(reps=0)
    t, _ = g.eval(0.5)
    assert np.isfinite(t["U"])
    g.close()


def small_water(lam=0.62):
    d = S.make_water_box(seed=21, n_waters=101, box_len=1.45, solute="ring12", n_side=5,
                         r_cut=0.7, grid=16, lam=lam)
    d.update(dt=0.001, lambda_mass=0.0, opes_stride=0)
    return d


def test_autotune_chooses_the_list_buffer_when_left_to_it():
    d = small_water()
    g = lfe.System(d, precision=lfe.LFE_FP32_MIXED, skin=0.0)
    g.step(20)
    t0, F0 = g.eval(0.5)
    p0, v0, e0 = g.get_state()
    ms, par = g.autotune(reps=10)
    assert par["skin_pm"] in (100, 140, 180, 220, 260)
    p1, v1, e1 = g.get_state()
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1) and e1["step"] == e0["step"]
    t1, F1 = g.eval(0.5)
    assert np.linalg.norm(F1 - F0) / np.linalg.norm(F0) < 1e-6
    assert abs(t1["n_pairs"] - t0["n_pairs"]) <= 2
    g.step(20)
    assert np.isfinite(g.get_state()[0]).all()
    # a fixed buffer is never changed
    h = lfe.System(d, precision=lfe.LFE_FP32_MIXED, skin=0.12)
    h.step(20)
    _, ph = h.autotune(reps=10)
    assert ph["skin_pm"] == 120


def test_restore_into_a_narrower_buffer_rebuilds_the_list(tmp_path):
    # the writer's list (0.26 nm buffer) is only rebuilt after an atom moved
    # 0.13 nm; a reader with a 0.10 nm buffer rebuilds at the restored
    # positions, so its forces are those of the current configuration
    from oracle import reference as R
    d = small_water()
    a = lfe.System(d, precision=lfe.LFE_FP32_MIXED, skin=0.26, seed=3)
    a.step(60)
    path = tmp_path / "wide.ckpt"
    a.checkpoint(path)
    pos, _, _ = a.get_state()
    b = lfe.System(d, precision=lfe.LFE_FP32_MIXED, skin=0.10, seed=3)
    b.restore(path)
    t, F = b.eval(0.5)
    E, F0, Fuv, Fs = R.nonbonded(dict(d, pos=pos.astype(np.float32)), level=2)
    hA, hB, _, _ = R.switching(0.5)
    Fo = F0 + hA * Fuv + hB * Fs
    assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) < 1e-5
    assert abs(t["n_pairs"] - E["n_pairs"]) <= 2


@pytest.mark.parametrize("precision", [lfe.LFE_FP32_MIXED, lfe.LFE_FP64])
def test_stage_timer_lists_the_stages_and_leaves_results_alone(precision):
    d = small_water()
    g = lfe.System(d, precision=precision)
    t0, F0 = g.eval(0.4)
    st = g.time_stages(0.7, reps=3)
    names = ["nbl_build", "pairs", "pme_spread", "pme_fft_fwd", "pme_conv", "pme_fft_inv", "pme_gather",
             "excl_14", "bonded", "eval_out", "uv_energy_fp64"]
    assert list(st)[:11] == names and all(v > 0 for v in st.values())
    assert ("pairs_full" in st) == (precision == lfe.LFE_FP32_MIXED)
    t1, F1 = g.eval(0.4)
    assert np.array_equal(F0, F1) and t1["U"] == t0["U"] and t1["dUdl"] == t0["dUdl"]
