"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Bar (spec tolerances): forces within 1e-5 relative RMS and dU/dlambda
within 1e-6 relative of the level-2 oracle (smooth PME on the same grid),
element by element on the same seeded inputs.  The FP64 instantiation is held
to 1e-10.  Energies per class are compared too, and the pair count exactly in
FP64.
"""
import functools

import numpy as np
import pytest

from oracle import reference as R
from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

# F: relative RMS over all atoms, and over the solute atoms alone once the
# solute is coupled (lambda >= 0.6: the solute carries a small share of the
# total force, so a solute-only error would hide in the global norm; below,
# a rigid solute with all intramolecular pairs excluded feels a small
# remainder of cancelling reciprocal and exclusion-correction forces, and a
# relative norm of that remainder measures cancellation, so there the solute
# atoms' RMS error is held to F times the RMS atomic force of the system);
# Fmax: the largest error of any force component against the RMS atomic force
# (ten times the RMS bound: FP32 sums of a few hundred pair terms per atom)
TOL = {lfe.LFE_FP32_MIXED: dict(F=1e-5, Fmax=1e-4, dU=1e-6, E=1e-6),
       lfe.LFE_FP64: dict(F=1e-9, Fmax=1e-8, dU=1e-8, E=1e-9)}


@functools.lru_cache(maxsize=None)
def oracle_basis(key):
    d = SYSTEMS[key]()
    E, F0, Fuv, Fs = R.nonbonded(d, level=2)
    Ub, Fb = R.bonded(d)
    return d, E, F0, Fuv, Fs, Ub, Fb


def oracle_at(key, lam):
    d, E, F0, Fuv, Fs, Ub, Fb = oracle_basis(key)
    hA, hB, dA, dB = R.switching(lam)
    F = F0 + hA * Fuv + hB * Fs + Fb
    U = E["U_vv"] + E["U_uu"] + hA * E["U_uv"] + hB * E["U_soft"] + Ub
    dU = dA * E["U_uv"] + dB * E["U_soft"]
    return d, dict(U=U, dUdl=dU, F=F, E=E, Ub=Ub, dA=dA, dB=dB)


def small_ragged():
    # 101 waters + 12-atom solute: 1 solute cluster + 10 solvent clusters, the
    # last holding 15 atoms
    return S.make_water_box(seed=21, n_waters=101, box_len=1.45, solute="ring12", n_side=5,
                            r_cut=0.7, grid=16)


def no_solute():
    return S.make_water_box(seed=22, n_waters=200, box_len=1.82, solute=None, n_side=6, r_cut=0.9,
                            grid=16)


def odd_grid():
    # anisotropic grid of odd and even lengths: column groups with
    # self-partner columns, radix-3/5 stages on every axis
    return dict(small_ragged(), grid=[20, 18, 15])


def big_grid():
    # a 100^3 grid: its FP64 plane does not fit in shared memory, so both
    # precisions take the per-axis transform
    return dict(small_ragged(), grid=[100, 100, 100])


def solute_only():
    # the 12-atom solute alone in the C0 box: no solvent clusters, no
    # solute-solvent pairs (U_uv = U_soft = 0, dU/dlambda = 0).  Its
    # exclusions are dropped so that its 66 pairs are real-space pairs (with
    # every pair excluded the net force is a small remainder of cancelling
    # reciprocal and correction terms, and a relative force norm is
    # ill-conditioned), Coulomb only (bonded atoms would overlap in LJ)
    d = S.make_c0()
    d = S.subsystem(d, np.flatnonzero(d["solute"]))
    d["excl"] = np.zeros((0, 2), dtype=np.int32)
    d["epsilon"] = np.zeros_like(d["epsilon"])
    return d


def far_exclusion():
    # the ragged water box with two extra exclusions, each between the oxygens
    # of two nearby waters far apart in index: the exclusion graph then joins
    # them into molecules spanning more than 63 atom indices, whose masks the
    # list placement builds by searching the exclusion lists (the bitmask path
    # covers the other molecules)
    d = small_ragged()
    pos, box = np.asarray(d["pos"]), np.asarray(d["box"])
    wat = np.asarray(d["waters"])
    ox = wat[:, 0]
    extra = []
    for w0 in (0, 1):
        dd = pos[ox] - pos[ox[w0]]
        dd -= box * np.round(dd / box)
        r = np.sqrt((dd * dd).sum(axis=1))
        far = [w for w in np.argsort(r) if abs(int(ox[w]) - int(ox[w0])) > 70 and 0.0 < r[w] < 0.5]
        extra.append((int(ox[w0]), int(ox[far[0]])))
    d["excl"] = np.concatenate([np.asarray(d["excl"]), np.asarray(extra, dtype=np.int32)]).astype(np.int32)
    return d


SYSTEMS = {
    "c0": S.make_c0,
    "far_excl": far_exclusion,
    "ragged": small_ragged,
    "odd_grid": odd_grid,
    "big_grid": big_grid,
    "nosolute": no_solute,
    "soluteonly": solute_only,
    "c2": S.make_c2,
    "c1": S.make_c1,
    "c4": lambda: S.make_c4_frame(frame=5),
}

_gpu_systems = {}


def gpu_system(key, precision):
    k = (key, precision)
    if k not in _gpu_systems:
        d = SYSTEMS[key]() if key not in ("c2", "c1") else oracle_basis(key)[0]
        _gpu_systems[k] = lfe.System(d, precision=precision)
    return _gpu_systems[k]


def check(key, lam, precision):
    d, o = oracle_at(key, lam)
    g = gpu_system(key, precision)
    terms, F = g.eval(lam)
    tol = TOL[precision]
    Fo = o["F"]
    rel = np.linalg.norm(F - Fo) / np.linalg.norm(Fo)
    assert rel <= tol["F"], f"{key} lam={lam}: force rel RMS {rel:.3e}"
    sol = np.asarray(d["solute"]).astype(bool)
    f_rms = np.sqrt((Fo * Fo).sum(axis=1).mean())
    if sol.any() and not sol.all():
        if lam >= 0.6:
            rel_u = np.linalg.norm(F[sol] - Fo[sol]) / np.linalg.norm(Fo[sol])
            assert rel_u <= tol["F"], f"{key} lam={lam}: solute force rel RMS {rel_u:.3e}"
        err_u = np.sqrt(((F[sol] - Fo[sol]) ** 2).sum(axis=1).mean()) / f_rms
        assert err_u <= tol["F"], f"{key} lam={lam}: solute force RMS error {err_u:.3e} of the RMS force"
    emax = np.abs(F - Fo).max() / f_rms
    assert emax <= tol["Fmax"], f"{key} lam={lam}: max force error {emax:.3e} of the RMS force"
    scale_dU = abs(o["dA"] * o["E"]["U_uv"]) + abs(o["dB"] * o["E"]["U_soft"])
    err_dU = abs(terms["dUdl"] - o["dUdl"])
    assert err_dU <= tol["dU"] * max(abs(o["dUdl"]), 1e-300) or err_dU <= 1e-12 * max(scale_dU, 1.0), \
        f"{key} lam={lam}: dU/dl {terms['dUdl']} vs {o['dUdl']}"
    # each class energy is a sum of large terms of both signs (self energy,
    # exclusion corrections, real and reciprocal parts): its error is measured
    # against the sum of the magnitudes of its parts
    E = o["E"]
    scale = {c: sum(abs(E[f"{part}_{c}"]) for part in ("coul_real", "rec", "bg", "lj", "excl"))
             + (abs(E.get(f"self_{c}", 0.0)) + abs(E.get(f"p14_{c}", 0.0))) for c in ("vv", "uu", "uv")}
    for k, sc in (("U_vv", scale["vv"]), ("U_uu", scale["uu"]), ("U_uv", scale["uv"]),
                  ("U_soft", abs(E["U_soft"]))):
        assert abs(terms[k] - E[k]) <= tol["E"] * max(sc, 1.0), f"{key}: {k} {terms[k]} vs {E[k]}"
    assert abs(terms["U_bonded"] - o["Ub"]) <= tol["E"] * max(abs(o["Ub"]), 1.0)
    assert abs(terms["U"] - o["U"]) <= tol["E"] * max(sum(scale.values()) + abs(o["Ub"]), 1.0)
    if precision == lfe.LFE_FP64:
        assert terms["n_pairs"] == o["E"]["n_pairs"]
    else:
        assert abs(terms["n_pairs"] - o["E"]["n_pairs"]) <= 2
    return rel, err_dU


LAMS = [0.0, 0.2, 0.35, 0.6, 1.0]


@pytest.mark.parametrize("precision", [lfe.LFE_FP64, lfe.LFE_FP32_MIXED])
@pytest.mark.parametrize("key", ["c0", "ragged", "nosolute", "soluteonly", "far_excl"])
def test_small_parity(key, precision):
    d = SYSTEMS[key]()
    for lam in LAMS + [d["lam"]]:
        check(key, lam, precision)


@pytest.mark.parametrize("precision", [lfe.LFE_FP64, lfe.LFE_FP32_MIXED])
@pytest.mark.parametrize("key", ["odd_grid", "big_grid"])
def test_transform_shapes(key, precision):
    for lam in (0.0, 0.5, 1.0):
        check(key, lam, precision)


@pytest.mark.parametrize("key", ["c2", "c1", "c4"])
def test_full_size_parity_fp32(key):
    for lam in (0.1, 0.5, 0.6, 0.9, 1.0):
        check(key, lam, lfe.LFE_FP32_MIXED)


def test_full_size_parity_fp64_c2():
    check("c2", 0.5, lfe.LFE_FP64)


def test_eval_is_bitwise_reproducible():
    g = gpu_system("c0", lfe.LFE_FP32_MIXED)
    t1, F1 = g.eval(0.47)
    t2, F2 = g.eval(0.47)
    assert np.array_equal(F1, F2)
    assert all(t1[k] == t2[k] for k in t1)


def test_empty_system_is_rejected():
    d = S.subsystem(S.make_c0(), np.zeros(0, dtype=np.int64))
    with pytest.raises(lfe.LfeError) as e:
        lfe.System(d)
    assert e.value.code == lfe.LFE_ERR_ARG


def test_bad_inputs_are_rejected_and_system_survives():
    d = SYSTEMS["ragged"]()
    g = lfe.System(d)
    bad = d["pos"].copy()
    bad[3, 1] = np.nan
    with pytest.raises(lfe.LfeError) as e:
        g.set_positions(bad)
    assert e.value.code == lfe.LFE_ERR_ARG
    with pytest.raises(lfe.LfeError):
        g.eval(1.5)
    t, F = g.eval(0.5)
    assert np.isfinite(F).all()
    dd = dict(d, r_cut=0.8)
    with pytest.raises(lfe.LfeError) as e:
        lfe.System(dd)
    assert e.value.code == lfe.LFE_ERR_ARG


def test_set_positions_far_move_rebuilds_on_device():
    # positions of another configuration of the same topology: every atom
    # moves far beyond skin/2, so the list is rebuilt inside the call
    d = SYSTEMS["ragged"]()
    g = lfe.System(d)
    rng = np.random.default_rng(3)
    perm_pos = d["pos"].copy()
    shift = S.f32(rng.uniform(0.2, 0.4, size=3))
    perm_pos = S.f32(perm_pos + shift)
    perm_pos = S.f32(perm_pos - d["box"] * np.floor(perm_pos / d["box"]))
    perm_pos[perm_pos >= d["box"]] = 0.0
    for pos in (perm_pos, d["pos"]):
        g.set_positions(pos)
        t, F = g.eval(0.7)
        E, F0, Fuv, Fs = R.nonbonded(dict(d, pos=pos), level=2)
        hA, hB, _, _ = R.switching(0.7)
        Fo = F0 + hA * Fuv + hB * Fs
        assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) < 1e-5


def test_set_positions_roundtrip():
    d = SYSTEMS["ragged"]()
    g = lfe.System(d)
    rng = np.random.default_rng(0)
    moved = S.f32(d["pos"] + rng.normal(scale=0.01, size=d["pos"].shape))
    moved = moved - d["box"] * np.floor(moved / d["box"])
    moved = S.f32(moved)
    moved[moved >= d["box"]] = 0.0
    g.set_positions(moved)
    t, F = g.eval(0.4)
    dd = dict(d, pos=moved)
    E, F0, Fuv, Fs = R.nonbonded(dd, level=2)
    hA, hB, _, _ = R.switching(0.4)
    Fo = F0 + hA * Fuv + hB * Fs
    assert np.linalg.norm(F - Fo) / np.linalg.norm(Fo) < 1e-5
