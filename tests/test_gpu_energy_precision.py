"""Precision of the reciprocal-space class energies of FP32 systems.

The solute-solvent reciprocal energy is a large share of a small U_uv, so the
FP32 systems form the class energies in df64 (float pairs, about 48 bits).
On an ion lattice whose spacing exceeds r_cut + skin there are no real-space
pairs and no exclusions: U_uv is then the reciprocal cross term plus its
background share only, and the FP32 system's U_uv and dU/dlambda must match
the level-2 oracle (smooth PME on the same grid, FP64) far below the FP32
rounding level (1e-9: the fixed-point charge grid is the limit)."""
import numpy as np
import pytest

from oracle import reference as R
from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu


def ion_lattice(seed, n_side=4, spacing=0.75, n_solute=16, grid=32):
    rng = np.random.default_rng(seed)
    L = n_side * spacing
    g = np.arange(n_side) * spacing
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.2
    pos = S.f32(pos + rng.normal(0.0, 0.02, pos.shape))
    n = pos.shape[0]
    q = rng.uniform(-0.8, 0.8, n)
    q -= q.mean()
    d = dict(S.make_c0())
    z2 = np.zeros((0, 2))
    d.update(box=S.f32(np.array([L, L, L])), pos=pos, charge=S.f32(q), sigma=S.f32(np.full(n, 0.3)),
             epsilon=np.zeros(n), solute=(np.arange(n) < n_solute).astype(np.uint8), mass=np.ones(n),
             excl=np.zeros((0, 2), dtype=np.int64), pairs14=np.zeros((0, 2), dtype=np.int64), scale14=z2,
             waters=np.zeros((0, 3), dtype=np.int64), r_cut=0.5, r_switch=0.4, grid=[grid] * 3,
             name="ion_lattice")
    return d


@pytest.mark.parametrize("precision", [lfe.LFE_FP32_MIXED, lfe.LFE_FP64])
@pytest.mark.parametrize("seed", [3, 4])
def test_reciprocal_class_energies_far_below_fp32_rounding(seed, precision):
    d = ion_lattice(seed)
    E = R.nonbonded(d, level=2)[0]
    assert E["n_pairs"] == 0
    g = lfe.System(d, precision=precision)
    # both modes share the fixed-point charge grid (2^-36 e per point), which
    # sets the limit near 1e-10; FP32 transforms would give 1e-6 to 1e-7
    tol = 1e-9
    for lam in (0.2, 0.6, 0.9):
        t, F = g.eval(lam)
        assert t["n_pairs"] == 0
        hA, hB, dA, dB = R.switching(lam)
        assert abs(t["U_uv"] - E["U_uv"]) <= tol * abs(E["U_uv"])
        assert abs(t["U_vv"] - E["U_vv"]) <= tol * abs(E["U_vv"])
        assert abs(t["U_uu"] - E["U_uu"]) <= tol * abs(E["U_uu"])
        assert abs(t["dUdl"] - dA * E["U_uv"]) <= tol * max(abs(dA * E["U_uv"]), 1e-300)
    g.close()
