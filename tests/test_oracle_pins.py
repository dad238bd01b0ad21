"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks a property that a plausible mistake in the oracle (a dropped
term, a wrong sign, index or coefficient, a transposed operand) would break:
closed forms (NaCl Madelung constant, dipole-lattice limit, LJ minimum),
invariants (alpha-independence of Ewald, forces = -grad U by central
differences, zero net force, lambda end points of Eq. 4), and the boundary
conditions the paper states for u_cap (Eq. 6) and the switching functions
(Eq. 7-10).
"""
import math

import numpy as np
import pytest

from oracle import reference as R
from paper_2608_12691_b300 import systems as S

KE = 138.935458


def polyfit_exact(f, deg, lo, hi):
    xs = np.linspace(lo, hi, deg + 1)
    ys = np.array([f(x) for x in xs])
    return np.polynomial.polynomial.polyfit(xs, ys, deg)


def poly_derivs_at(c, x, n):
    out = []
    p = np.polynomial.Polynomial(c)
    for k in range(n + 1):
        out.append(p(x))
        p = p.deriv()
    return out


# ---------------------------------------------------------------- Eq. 6

def test_ucap_cap_value_and_smooth_join():
    # the cap tends to 119.2 eps as r -> 0 (Section 2.2, Eq. 6)
    assert R.ucap(0.0)[0] == pytest.approx(119.2, abs=1e-12)
    # on [0,1) u_cap is a degree-6 polynomial; its value and first three
    # derivatives at x = 1 must equal those of 4x^-12 - 4x^-6: 0, -24, 456, -7392
    c = polyfit_exact(lambda x: R.ucap(x)[0], 6, 0.0, 0.999)
    d = poly_derivs_at(c, 1.0, 3)
    assert d[0] == pytest.approx(0.0, abs=1e-6)
    assert d[1] == pytest.approx(-24.0, rel=1e-7)
    assert d[2] == pytest.approx(456.0, rel=1e-7)
    assert d[3] == pytest.approx(-7392.0, rel=1e-7)
    # the cap is flat at x = 0 (no x, x^2, x^3 terms)
    assert np.allclose(c[1:4], 0.0, atol=1e-6)


def test_ucap_is_lj_beyond_sigma():
    # textbook LJ in reduced units: zero at x = 1, minimum -1 at x = 2^(1/6)
    xm = 2.0 ** (1.0 / 6.0)
    u, du = R.ucap(xm)
    assert u == pytest.approx(-1.0, rel=1e-12)
    assert du == pytest.approx(0.0, abs=1e-12)
    assert R.ucap(1.0)[0] == pytest.approx(0.0, abs=1e-12)
    # monotone decreasing cap on (0, 1)
    xs = np.linspace(0.01, 0.99, 50)
    assert all(R.ucap(x)[1] < 0 for x in xs)


def test_ucap_derivative_matches_fd():
    for x in (0.1, 0.5, 0.95, 1.0 + 1e-3, 1.3, 2.0):
        h = 1e-6
        fd = (R.ucap(x + h)[0] - R.ucap(x - h)[0]) / (2 * h)
        assert R.ucap(x)[1] == pytest.approx(fd, rel=1e-6, abs=1e-6)


# ------------------------------------------------------------- Eq. 7-10

def test_smoothsteps_vanishing_derivatives():
    # S_mn has m vanishing derivatives at x = 0 and n at x = 1 (Section 2.2)
    c22 = polyfit_exact(lambda x: R.S22(x)[0], 5, 0.001, 0.999)
    d0, d1 = poly_derivs_at(c22, 0.0, 2), poly_derivs_at(c22, 1.0, 2)
    assert np.allclose(d0, [0, 0, 0], atol=1e-7)
    assert np.allclose(d1, [1, 0, 0], atol=1e-6)
    c32 = polyfit_exact(lambda x: R.S32(x)[0], 6, 0.001, 0.999)
    d0, d1 = poly_derivs_at(c32, 0.0, 3), poly_derivs_at(c32, 1.0, 2)
    assert np.allclose(d0, [0, 0, 0, 0], atol=1e-6)
    assert np.allclose(d1, [1, 0, 0], atol=1e-5)
    assert R.S22(0.5)[0] == pytest.approx(0.5)
    assert R.S32(0.5)[0] == pytest.approx(0.34375)
    assert R.S32(-0.3)[0] == 0.0


def test_hA_hB_end_points():
    # h_A = 0 for lambda <= 0.35, h_A(1) = 1, h_B(1) = 0 (Section 2.2)
    for lam in (0.0, 0.1, 0.35):
        hA, hB, dA, dB = R.switching(lam)
        assert hA == 0.0 and dA == 0.0
    hA, hB, dA, dB = R.switching(1.0)
    assert (hA, hB) == (1.0, 0.0)
    assert dA == pytest.approx(0.0, abs=1e-14) and dB == pytest.approx(0.0, abs=1e-14)
    hA, hB, dA, dB = R.switching(0.0)
    assert hB == 0.0 and dB == 0.0
    for lam in (0.2, 0.36, 0.5, 0.8, 0.97):
        h = 1e-6
        a1, b1, _, _ = R.switching(lam + h)
        a0, b0, _, _ = R.switching(lam - h)
        _, _, dA, dB = R.switching(lam)
        assert dA == pytest.approx((a1 - a0) / (2 * h), rel=1e-6, abs=1e-9)
        assert dB == pytest.approx((b1 - b0) / (2 * h), rel=1e-6, abs=1e-9)


def test_lj_switch_boundary_conditions():
    rc, rs = 1.0, 0.9
    # fit in t = (r - r_sw)/(r_c - r_sw) for conditioning
    c = polyfit_exact(lambda t: R.lj_switch(rs + t * (rc - rs), rc, rs)[0], 5, 1e-3, 1 - 1e-3)
    d0, d1 = poly_derivs_at(c, 0.0, 2), poly_derivs_at(c, 1.0, 2)
    assert np.allclose(d0, [1, 0, 0], atol=1e-8)
    assert np.allclose(d1, [0, 0, 0], atol=1e-8)
    for r in (0.91, 0.95, 0.99):
        h = 1e-7
        fd = (R.lj_switch(r + h, rc, rs)[0] - R.lj_switch(r - h, rc, rs)[0]) / (2 * h)
        assert R.lj_switch(r, rc, rs)[1] == pytest.approx(fd, rel=1e-6)


# ------------------------------------------------------------------ Ewald

def nacl(a=0.5, cells=2, split_solute=False):
    pts = []
    qs = []
    for ix in range(2 * cells):
        for iy in range(2 * cells):
            for iz in range(2 * cells):
                pts.append([ix * a / 2, iy * a / 2, iz * a / 2])
                qs.append(1.0 if (ix + iy + iz) % 2 == 0 else -1.0)
    n = len(pts)
    sol = np.zeros(n, dtype=np.uint8)
    if split_solute:
        sol[: n // 2] = 1   # first half (not neutral per part is fine here)
    L = cells * a
    return dict(box=np.array([L] * 3), pos=np.array(pts, dtype=np.float64), charge=np.array(qs),
                sigma=np.zeros(n), epsilon=np.zeros(n), solute=sol,
                excl=np.zeros((0, 2), np.int32), pairs14=np.zeros((0, 2), np.int32),
                scale14=np.zeros((0, 2)), r_cut=L / 2, r_switch=-1.0, alpha=9.2,
                grid=[32, 32, 32], order=4)


from test_golden import value as golden_value  # noqa: E402

MADELUNG_NACL = golden_value("madelung_nacl.txt", "madelung_nacl")[0]   # Kittel, ch. 3


def test_madelung_nacl_level1():
    a = 0.5
    d = nacl(a)
    E, F0, Fuv, Fs = R.nonbonded(d, level=1)
    total = E["U_vv"] + E["U_uu"] + E["U_uv"]
    expect = -64 * MADELUNG_NACL * KE / a
    assert total == pytest.approx(expect, rel=1e-8)
    # perfect lattice: zero force on every ion
    assert np.abs(F0).max() < 1e-6 * KE / a ** 2
    # the class split of the same lattice sums to the same total
    d2 = nacl(a, split_solute=True)
    E2, _, _, _ = R.nonbonded(d2, level=1)
    assert E2["U_vv"] + E2["U_uu"] + E2["U_uv"] == pytest.approx(expect, rel=1e-8)


def test_madelung_nacl_spme_converges():
    a = 0.5
    d = nacl(a)
    expect = -64 * MADELUNG_NACL * KE / a
    errs = []
    for K in (8, 16, 32):
        E, _, _, _ = R.nonbonded(d, level=2, grid=[K] * 3, alpha=8.0, r_cut=0.5)
        errs.append(abs(E["U_vv"] - expect) / abs(expect))
    assert errs[2] < 1e-6
    assert errs[0] > errs[1] > errs[2] or errs[2] < 1e-9


@pytest.fixture(scope="module")
def c0():
    return S.make_c0(seed=11)


def small_water(seed=5, n_side=4, box_len=1.3, solute="ring12"):
    # 64 sites, 40 waters + 12-atom solute, small enough for FD
    return S.make_water_box(seed=seed, n_waters=40, box_len=box_len, solute=solute, n_side=n_side,
                            r_cut=0.6, grid=16)


def test_alpha_independence_per_class(c0):
    # each class energy is a Coulomb energy of neutral charge subsets plus
    # alpha-free LJ: it must not depend on the Ewald splitting parameter
    E1, _, _, _ = R.nonbonded(c0, level=1, alpha=4.6)
    E2, _, _, _ = R.nonbonded(c0, level=1, alpha=5.6)
    for k in ("U_vv", "U_uu", "U_uv"):
        assert E1[k] == pytest.approx(E2[k], rel=2e-7, abs=1e-5), k
    assert E1["U_soft"] == pytest.approx(E2["U_soft"], rel=1e-12)


def test_background_needed_for_charged_box():
    d = dict(box=np.array([2.0, 2.0, 2.0]), pos=np.array([[0.3, 0.4, 0.5], [1.1, 0.9, 1.4]]),
             charge=np.array([1.0, 0.5]), sigma=np.zeros(2), epsilon=np.zeros(2),
             solute=np.array([1, 0], np.uint8), excl=np.zeros((0, 2), np.int32),
             pairs14=np.zeros((0, 2), np.int32), scale14=np.zeros((0, 2)),
             r_cut=1.0, r_switch=-1.0, alpha=5.0, grid=[16] * 3, order=4)
    tot = lambda E: E["U_vv"] + E["U_uu"] + E["U_uv"]
    Ea, _, _, _ = R.nonbonded(d, level=1, alpha=5.0)
    Eb, _, _, _ = R.nonbonded(d, level=1, alpha=6.0)
    assert tot(Ea) == pytest.approx(tot(Eb), rel=1e-8)
    for k in ("U_vv", "U_uu", "U_uv"):
        assert Ea[k] == pytest.approx(Eb[k], rel=1e-8, abs=1e-9)
    nobg = lambda E: tot(E) - E["bg_vv"] - E["bg_uu"] - E["bg_uv"]
    assert abs(nobg(Ea) - nobg(Eb)) > 1e5 * 1e-8 * abs(tot(Ea))


def test_isolated_water_dipole_lattice_limit():
    # one water, all intramolecular pairs excluded: what remains is the
    # interaction with its periodic images, which for a cubic lattice with
    # conducting boundary tends to -(2 pi / 3V) k_e mu^2 (point-dipole limit)
    geo = S.water_geometry()
    q = np.array(S.W_Q)
    mu = np.linalg.norm((q[:, None] * geo).sum(0))
    vals = []
    for L in (3.0, 4.0):
        d = dict(box=np.array([L] * 3), pos=geo + L / 2, charge=q, sigma=np.zeros(3),
                 epsilon=np.zeros(3), solute=np.zeros(3, np.uint8),
                 excl=np.array([[0, 1], [0, 2], [1, 2]], np.int32),
                 pairs14=np.zeros((0, 2), np.int32), scale14=np.zeros((0, 2)),
                 r_cut=1.2, r_switch=-1.0, alpha=3.5, grid=[16] * 3, order=4)
        E, _, _, _ = R.nonbonded(d, level=1)
        vals.append(E["U_vv"] * L ** 3)
    limit = -(2 * math.pi / 3) * KE * mu ** 2
    assert vals[1] == pytest.approx(limit, rel=0.02)
    assert abs(vals[1] - limit) < abs(vals[0] - limit) + 1e-12


def test_pair14_unit_scale_equals_plain_pair():
    pos = np.array([[0.5, 0.5, 0.5], [0.75, 0.6, 0.55]])
    base = dict(box=np.array([3.0] * 3), pos=pos, charge=np.array([0.4, -0.3]),
                sigma=np.array([0.3, 0.32]), epsilon=np.array([0.5, 0.8]),
                solute=np.zeros(2, np.uint8), r_cut=1.2, r_switch=1.0, alpha=3.0,
                grid=[16] * 3, order=4)
    plain = dict(base, excl=np.zeros((0, 2), np.int32), pairs14=np.zeros((0, 2), np.int32),
                 scale14=np.zeros((0, 2)))
    as14 = dict(base, excl=np.array([[0, 1]], np.int32), pairs14=np.array([[0, 1]], np.int32),
                scale14=np.array([[1.0, 1.0]]))
    Ea, Fa, _, _ = R.nonbonded(plain, level=1)
    Eb, Fb, _, _ = R.nonbonded(as14, level=1)
    assert Ea["U_vv"] == pytest.approx(Eb["U_vv"], rel=1e-12)
    assert np.allclose(Fa, Fb, rtol=1e-10, atol=1e-10)


def test_lj_minimum_with_mixing():
    si, sj, ei, ej = 0.28, 0.34, 0.3, 0.6
    s, e = 0.5 * (si + sj), math.sqrt(ei * ej)
    rmin = 2 ** (1 / 6) * s
    pos = np.array([[1.0, 1.0, 1.0], [1.0 + rmin, 1.0, 1.0]])
    d = dict(box=np.array([4.0] * 3), pos=pos, charge=np.zeros(2), sigma=np.array([si, sj]),
             epsilon=np.array([ei, ej]), solute=np.zeros(2, np.uint8),
             excl=np.zeros((0, 2), np.int32), pairs14=np.zeros((0, 2), np.int32),
             scale14=np.zeros((0, 2)), r_cut=1.5, r_switch=1.2, alpha=3.0, grid=[16] * 3, order=4)
    E, F0, _, _ = R.nonbonded(d, level=0)
    assert E["U_vv"] == pytest.approx(-e, rel=1e-12)
    assert np.abs(F0).max() < 1e-10
    # the same pair as solute-solvent: U_uv is the LJ and U_soft equals it (x >= 1)
    d["solute"] = np.array([1, 0], np.uint8)
    E, _, Fuv, Fs = R.nonbonded(d, level=0)
    assert E["U_uv"] == pytest.approx(-e, rel=1e-12)
    assert E["U_soft"] == pytest.approx(-e, rel=1e-12)
    # at r -> 0 the soft basis is capped at 119.2 eps_ij (Section 2.2)
    d["pos"] = np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 1.0 + 1e-9]])
    E, _, _, _ = R.nonbonded(d, level=0)
    assert E["U_soft"] == pytest.approx(119.2 * e, rel=1e-9)


def _fd_check(d, level, lam, atoms, h=1e-5, rtol=1e-6, **kw):
    ref = R.evaluate(d, lam, level=level, **kw)
    F = ref["F"]
    for i in atoms:
        for k in range(3):
            pp = d["pos"].copy(); pp[i, k] += h
            pm = d["pos"].copy(); pm[i, k] -= h
            ep = R.evaluate(d, lam, level=level, pos=pp, **kw)
            em = R.evaluate(d, lam, level=level, pos=pm, **kw)
            if ep["E"]["n_pairs"] != em["E"]["n_pairs"]:
                continue   # a pair crossed the cutoff: U is not differentiable there
            fd = -(ep["U"] - em["U"]) / (2 * h)
            scale = max(1.0, np.abs(F[i]).max())
            assert abs(F[i, k] - fd) <= rtol * scale, (i, k, F[i, k], fd)


@pytest.mark.parametrize("level", [1, 2])
def test_forces_are_minus_grad_U(level):
    d = small_water()
    solute_atoms = list(range(0, 3))
    water_atoms = [20, 41, 80]
    for lam in (0.2, 0.7):
        _fd_check(d, level, lam, solute_atoms + water_atoms)


def test_bonded_forces_and_equilibrium():
    d = S.make_c4_frame(frame=1)
    sub = S.subsystem(d, np.arange(22))
    U, F = R.bonded(sub)
    # bonds and angles are built at their equilibrium values: only torsions remain
    tors_only = dict(sub, bonds=sub["bonds"][:0], angles=sub["angles"][:0])
    Ut, _ = R.bonded(tors_only)
    assert U == pytest.approx(Ut, abs=1e-6)   # positions are float32-rounded
    rng = np.random.default_rng(3)
    pos = sub["pos"] + rng.normal(scale=0.01, size=sub["pos"].shape)
    U, F = R.bonded(sub, pos=pos)
    h = 1e-6
    for i in (0, 8, 14, 21):
        for k in range(3):
            pp = pos.copy(); pp[i, k] += h
            pm = pos.copy(); pm[i, k] -= h
            fd = -(R.bonded(sub, pos=pp)[0] - R.bonded(sub, pos=pm)[0]) / (2 * h)
            assert F[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    # zero net bonded force
    assert np.abs(F.sum(0)).max() < 1e-8


def test_dihedral_matches_construction():
    xyz = S.solute_dipeptide22(-63.0, 141.0, 55.0)
    box = np.array([10.0] * 3)
    # phi = C(ace)-N-CA-C = atoms 4, 6, 8, 14; psi = N-CA-C-N' = 6, 8, 14, 16
    phi = math.degrees(R.dihedral(xyz[4], xyz[6], xyz[8], xyz[14], box))
    psi = math.degrees(R.dihedral(xyz[6], xyz[8], xyz[14], xyz[16], box))
    chi = math.degrees(R.dihedral(xyz[6], xyz[8], xyz[10], xyz[11], box))
    assert phi == pytest.approx(-63.0, abs=1e-6)
    assert psi == pytest.approx(141.0, abs=1e-6)
    assert chi == pytest.approx(55.0, abs=1e-6)


@pytest.mark.parametrize("level", [1, 2])
def test_dUdlambda_matches_fd(level):
    d = small_water()
    for lam in (0.1, 0.34, 0.5, 0.9):
        h = 1e-4
        up = R.evaluate(d, lam + h, level=level, with_bonded=False)["U"]
        um = R.evaluate(d, lam - h, level=level, with_bonded=False)["U"]
        dU = R.evaluate(d, lam, level=level, with_bonded=False)["dUdl"]
        assert dU == pytest.approx((up - um) / (2 * h), rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("level", [1, 2])
def test_lambda_end_points(level):
    # lambda = 1: the fully interacting system (Section 2.2); lambda = 0: the
    # solvent and the solute each on their own in the same box
    d = small_water(seed=9)
    full = R.evaluate(d, 1.0, level=level, with_bonded=False)
    plain = R.evaluate(d, 1.0, level=level, with_bonded=False, solute=np.zeros_like(d["solute"]))
    assert full["U"] == pytest.approx(plain["U"], rel=1e-10)
    assert np.allclose(full["F"], plain["F"], rtol=1e-9, atol=1e-8)
    zero = R.evaluate(d, 0.0, level=level, with_bonded=False)
    ns = int(d["solute"].sum())
    idx_u = np.arange(ns)
    idx_v = np.arange(ns, len(d["charge"]))
    su = S.subsystem(d, idx_u)
    sv = S.subsystem(d, idx_v)
    eu = R.evaluate(su, 1.0, level=level, with_bonded=False, solute=np.zeros(ns, np.uint8))
    ev = R.evaluate(sv, 1.0, level=level, with_bonded=False)
    assert zero["U"] == pytest.approx(eu["U"] + ev["U"], rel=1e-10)
    assert np.allclose(zero["F"][idx_u], eu["F"], rtol=1e-9, atol=1e-8)
    assert np.allclose(zero["F"][idx_v], ev["F"], rtol=1e-9, atol=1e-8)


def test_zero_net_force_level1(c0):
    E, F0, Fuv, Fs = R.nonbonded(c0, level=1)
    for F in (F0, Fuv, Fs):
        scale = np.abs(F).max()
        assert np.abs(F.sum(0)).max() < 1e-9 * scale * len(F)


def test_spme_approaches_ewald(c0):
    E1, F1, U1, S1 = R.nonbonded(c0, level=1)
    errs = []
    for K in (16, 32):
        E2, F2, U2, S2 = R.nonbonded(c0, level=2, grid=[K] * 3)
        errs.append(np.linalg.norm(F2 - F1) / np.linalg.norm(F1))
        assert E2["U_soft"] == pytest.approx(E1["U_soft"], rel=1e-12)
    assert errs[1] < errs[0] / 4     # order-4 B-splines: error falls fast with K
    assert errs[1] < 1e-4


def test_bspline_partition_of_unity():
    # sum_k M_n(u - k) = 1 and the b-moduli are finite for even order
    for u in (0.0, 0.3, 0.77):
        assert sum(R.bspline(4, u + j) for j in range(4)) == pytest.approx(1.0, abs=1e-14)
    assert all(np.isfinite(R.bmod2(4, 48, m)) for m in range(48))
    assert R.bmod2(4, 16, 0) == pytest.approx(1.0)
