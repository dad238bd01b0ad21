"""The PME entry point that allocates no device memory (lfe_pme_noalloc).

It is meant for callers that cannot let a library call cudaMalloc (processes
whose device memory is owned by a pool that forbids hidden allocations,
services that must not grow after start-up).  Its grids live in a fixed
device array; this test checks, through the C-ABI, that two calls in a row
give the same reciprocal-space forces and class energies as the ordinary
system path (lfe_eval) on a system whose real-space part is empty, within the
parity tolerances of the FP32 path; that both match the level-2 oracle (the
same smooth PME in FP64 on the CPU), the reciprocal energies alone to 1e-6
relative; and that a grid larger than the fixed array is refused.  The file
name sorts last so that a stop-at-first-failure run has already run every
other test.
"""
import numpy as np
import pytest

from oracle import reference as R
from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

def sparse_system():
    # 216 ions on a 0.5 nm lattice (+-0.02 nm jitter) in a 3 nm box with a
    # 0.4 nm cutoff: no pair is inside the cutoff, no LJ, no exclusions, so
    # the system path's energies and forces are the reciprocal, self and
    # background terms alone
    rng = np.random.default_rng(8)
    g = (np.arange(6) + 0.5) * 0.5
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) + rng.uniform(-0.02, 0.02, (216, 3))
    n = len(pos)
    q = rng.uniform(-0.8, 0.8, n)
    sol = np.zeros(n, np.uint8)
    sol[:12] = 1
    q[:12] -= q[:12].mean()
    q[12:] -= q[12:].mean()
    box = S.f32([3.0, 3.0, 3.0])
    return dict(box=box, pos=S.f32(pos), charge=S.f32(q), sigma=np.full(n, 0.3), epsilon=np.zeros(n),
                solute=sol, mass=np.ones(n), excl=np.zeros((0, 2), np.int32),
                pairs14=np.zeros((0, 2), np.int32), scale14=np.zeros((0, 2)), r_cut=0.4, r_switch=-1.0,
                alpha=3.0, grid=[32, 32, 32], order=4, lam=0.6)


@pytest.mark.parametrize("lam", [0.6, 0.25])
def test_noalloc_matches_system_path_and_oracle_twice(lam):
    import torch
    d = sparse_system()
    sysg = lfe.System(d, precision=lfe.LFE_FP32_MIXED)
    terms, F_ref = sysg.eval(lam)
    assert terms["n_pairs"] == 0
    # the level-2 oracle: with no pair inside the cutoff, no LJ and no
    # exclusions its forces are the reciprocal forces alone
    Eo, F0, Fuv, Fs = R.nonbonded(d, level=2)
    hA = R.switching(lam)[0]
    F_or = F0 + hA * Fuv
    dev = torch.device("cuda")
    pos = torch.tensor(d["pos"].ravel(), dtype=torch.float64, device=dev)
    q = torch.tensor(d["charge"], dtype=torch.float64, device=dev)
    sol = torch.tensor(d["solute"], dtype=torch.uint8, device=dev)
    n = len(d["charge"])
    for call in range(2):
        F = torch.full((3 * n,), float("nan"), dtype=torch.float64, device=dev)
        E = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream()
        lfe.pme_noalloc(n, pos.data_ptr(), q.data_ptr(), sol.data_ptr(), d["box"], d["alpha"], d["grid"], lam,
                        F.data_ptr(), E.data_ptr(), stream)
        torch.cuda.synchronize()
        F = F.cpu().numpy().reshape(n, 3)
        E = E.cpu().numpy()
        # against the existing entry point (the system path)
        rel = np.linalg.norm(F - F_ref) / np.linalg.norm(F_ref)
        assert rel < 1e-5, (call, rel)
        for k, name in enumerate(("U_vv", "U_uu", "U_uv")):
            assert abs(E[k] - terms[name]) <= 1e-6 * abs(terms[name]), (call, name, E[k], terms[name])
        # against the oracle: forces, and each class's reciprocal energy with
        # the oracle's self and background terms removed from the total
        rel_o = np.linalg.norm(F - F_or) / np.linalg.norm(F_or)
        assert rel_o < 1e-5, (call, rel_o)
        for k, c in enumerate(("vv", "uu", "uv")):
            rec = E[k] - Eo.get(f"self_{c}", 0.0) - Eo[f"bg_{c}"]
            assert abs(rec - Eo[f"rec_{c}"]) <= 1e-6 * abs(Eo[f"rec_{c}"]), (call, c, rec, Eo[f"rec_{c}"])


def test_noalloc_rejects_oversized_grid():
    import torch
    d = sparse_system()
    n = len(d["charge"])
    dev = torch.device("cuda")
    pos = torch.tensor(d["pos"].ravel(), dtype=torch.float64, device=dev)
    q = torch.tensor(d["charge"], dtype=torch.float64, device=dev)
    sol = torch.tensor(d["solute"], dtype=torch.uint8, device=dev)
    F = torch.zeros(3 * n, dtype=torch.float64, device=dev)
    E = torch.zeros(3, dtype=torch.float64, device=dev)
    with pytest.raises(lfe.LfeError) as e:
        lfe.pme_noalloc(n, pos.data_ptr(), q.data_ptr(), sol.data_ptr(), d["box"], d["alpha"], [64, 64, 64], 0.5,
                        F.data_ptr(), E.data_ptr())
    assert e.value.code == lfe.LFE_ERR_ARG
    assert "LFE_NOALLOC_MAX_GRID" in str(e.value)
