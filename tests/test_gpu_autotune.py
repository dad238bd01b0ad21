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
