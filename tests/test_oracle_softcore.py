"""Pins of the oracle's optional soft-core coupling (the conventional
alternative that Section 2.2 sets the linear-basis method against; the
configuration of the plain FP64 workload names alpha = 0.5, p = 1).  With
soft-core coupling the solute-solvent Lennard-Jones term is the Beutler form
at lambda and the Coulomb terms keep the h_A weight.  Pinned by what the form
must reduce to: at lambda = 1 the fully coupled system (the linear-basis
potential at lambda = 1, where h_A = 1 and h_B = 0), at lambda = 0 the
decoupled one; dU/dlambda and the forces by central differences; and a
finite value at contact, where plain LJ diverges."""
import math

import numpy as np
import pytest

from oracle import reference as R
from paper_2608_12691_b300 import systems as S


def c0_softcore():
    d = S.make_c0()
    d["sc_alpha"], d["sc_power"] = 0.5, 1.0
    return d


@pytest.mark.parametrize("level", [1, 2])
def test_lambda_end_points_equal_the_linear_basis_end_points(level):
    d = c0_softcore()
    lbf = dict(d, sc_alpha=0.0)
    for lam in (0.0, 1.0):
        a = R.evaluate(d, lam, level=level)
        b = R.evaluate(lbf, lam, level=level)
        assert a["U"] == pytest.approx(b["U"], rel=1e-12, abs=1e-9)
        assert np.allclose(a["F"], b["F"], rtol=0, atol=1e-9 * np.abs(b["F"]).max())


def test_dudl_matches_central_differences():
    d = c0_softcore()
    h = 1e-5
    for lam in (0.05, 0.3, 0.5, 0.77, 0.95):
        e = R.evaluate(d, lam, level=2)
        fd = (R.evaluate(d, lam + h, level=2)["U"] - R.evaluate(d, lam - h, level=2)["U"]) / (2 * h)
        assert e["dUdl"] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    # at lambda = 0 the soft-core derivative is finite (p = 1): one-sided
    e0 = R.evaluate(d, 0.0, level=2)
    fd0 = (R.evaluate(d, 2e-6, level=2)["U"] - e0["U"]) / 2e-6
    assert math.isfinite(e0["dUdl"]) and e0["dUdl"] == pytest.approx(fd0, rel=1e-4, abs=1e-4)


def test_forces_are_minus_the_gradient():
    d = c0_softcore()
    lam = 0.55
    e = R.evaluate(d, lam, level=2)
    rng = np.random.default_rng(4)
    sol = np.flatnonzero(d["solute"])
    atoms = list(sol[:3]) + list(rng.choice(np.flatnonzero(~d["solute"].astype(bool)), 3, replace=False))
    h = 1e-6     # small enough that no pair crosses the cutoff between the two points
    for a in atoms:
        for k in range(3):
            p1 = d["pos"].astype(np.float64).copy()
            p2 = p1.copy()
            p1[a, k] += h
            p2[a, k] -= h
            fd = -(R.evaluate(d, lam, level=2, pos=p1)["U"] - R.evaluate(d, lam, level=2, pos=p2)["U"]) / (2 * h)
            assert e["F"][a, k] == pytest.approx(fd, rel=1e-5, abs=1e-4)


def test_two_atom_pair_is_finite_at_contact():
    # one solute atom 1e-3 nm from a solvent atom, no charges: plain LJ is
    # 4 eps (sigma/r)^12 ~ 1e30 eps there, the soft-core term at lambda < 1 is
    # 4 eps lambda^p (1/D^2 - 1/D) with D = alpha (1 - lambda) + (r/sigma)^6,
    # e.g. lambda = 0.5, alpha = 0.5: D = 0.25 + 1.5e-15 and U = 24 eps
    eps = 0.3
    d = dict(box=np.array([3.0, 3.0, 3.0]), pos=np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 1.001]]),
             charge=np.zeros(2), sigma=np.array([0.3, 0.3]), epsilon=np.array([eps, eps]),
             solute=np.array([1, 0], dtype=np.uint8), excl=np.zeros((0, 2), np.int32),
             pairs14=np.zeros((0, 2), np.int32), scale14=np.zeros((0, 2)), r_cut=0.9, r_switch=-1.0,
             alpha=3.0, grid=[16, 16, 16], order=4, sc_alpha=0.5, sc_power=1.0)
    e = R.evaluate(d, 0.5, level=0, with_bonded=False)
    assert e["E"]["U_soft"] == pytest.approx(24.0 * eps, rel=1e-12)
    # the force vanishes at contact like r^5 (dD/dr = 6 (r/sigma)^6 / r)
    assert np.abs(e["F"]).max() < 1e-9
