"""Host-side checks of the seeded workload generators: the octanol start has
no two atoms of different molecules (or a molecule and the solute) closer
than 0.13 nm for the seeds the batched replicas use, and a start without
such contacts is left exactly as drawn."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_2608_12691_b300 import systems as S


def closest_intermolecular(d):
    pos = d["pos"].astype(np.float64)
    box = d["box"].astype(np.float64)
    n = len(pos)
    n_u = int(d["solute"].sum())
    mol = np.concatenate([np.full(n_u, -1), np.arange(n - n_u) // 27])
    pr = cKDTree(np.mod(pos, box), boxsize=box).query_pairs(0.16, output_type="ndarray")
    pr = pr[mol[pr[:, 0]] != mol[pr[:, 1]]]
    dv = pos[pr[:, 1]] - pos[pr[:, 0]]
    dv -= box * np.round(dv / box)
    r = np.linalg.norm(dv, axis=1)
    return r.min() if r.size else np.inf


@pytest.mark.parametrize("seed", [6007, 6020])
def test_octanol_start_has_no_close_intermolecular_contact(seed):
    d = S.make_c1(seed=seed)
    assert len(d["charge"]) == 13520
    assert closest_intermolecular(d) >= 0.13


def test_octanol_chains_move_only_when_in_contact():
    # the 36-chain box has no contact below 0.13 nm as drawn: redrawing
    # leaves it (and its chain conformations) exactly as placed
    d = S.make_octanol_box(seed=31, n_chains=36, box_len=2.8, nx=6, ny=6, nz=2, r_cut=0.9, grid=24, lam=0.55)
    x = d["pos"]
    box = d["box"]
    n_u = int(d["solute"].sum())
    chains = [x[n_u + 27 * c: n_u + 27 * (c + 1)].astype(np.float64) for c in range(36)]
    out = S._separate_chains(31, chains, np.array([c.mean(axis=0) for c in chains]), x[:n_u].astype(np.float64),
                             box)
    assert all(np.array_equal(a, b) for a, b in zip(chains, out))
