"""Pins of the Monte Carlo barostat oracle (Section 2.6's NPT runs) to what
statistical mechanics fixes: the ideal-gas volume distribution (a Gamma
distribution, which needs the N ln(V'/V) Jacobian and the sign of P dV), the
shift of the mean volume by an energy linear in V (the sign of dU), the molar
volume of an ideal gas at 25 C and 1 atm (the units of P), and rigid
molecules under centre-of-mass scaling."""
import numpy as np
import pytest

from oracle import barostat as B


def run_chain(n_mol, P, kT, dV_max, n_moves, energy, seed, V0):
    rng = np.random.default_rng(seed)
    L = V0 ** (1.0 / 3.0)
    box = np.array([L, L, L])
    pos = rng.uniform(0.0, L, size=(n_mol, 3))
    mass = np.ones(n_mol)
    mol = np.arange(n_mol)
    U = energy(pos, box)
    vols = np.empty(n_moves)
    n_acc = 0
    for k in range(n_moves):
        u = rng.random(2)
        pos, box, U, acc = B.volume_move(pos, box, mass, mol, energy, U, P, kT, dV_max, u[0], u[1])
        n_acc += acc
        vols[k] = np.prod(box)
    return vols, n_acc / n_moves


def test_ideal_gas_volume_distribution():
    # p(V) ~ V^N exp(-P V / kT): Gamma(N + 1, kT / P); mean 10, sd 4.47 here
    n_mol, kT = 4, 2.5
    P = (n_mol + 1) * kT / 10.0
    vols, acc = run_chain(n_mol, P, kT, 6.0, 60000, lambda x, b: 0.0, 11, 10.0)
    v = vols[2000:]
    assert 0.2 < acc < 0.9
    assert v.mean() == pytest.approx((n_mol + 1) * kT / P, rel=0.04)
    assert v.var() == pytest.approx((n_mol + 1) * (kT / P) ** 2, rel=0.15)
    # without the Jacobian the chain would sample Gamma(1, kT/P), mean 2
    assert v.mean() > 8.0


def test_energy_linear_in_volume_acts_as_pressure():
    # U = a V adds a to the pressure: mean volume (N + 1) kT / (P + a)
    n_mol, kT, P, a = 4, 2.5, 0.75, 0.5
    vols, _ = run_chain(n_mol, P, kT, 5.0, 60000, lambda x, b: a * float(np.prod(b)), 12, 8.0)
    assert vols[2000:].mean() == pytest.approx((n_mol + 1) * kT / (P + a), rel=0.04)


def test_ideal_gas_molar_volume_units():
    # molar volume of an ideal gas at 298.15 K and 1 atm: 24.465 L/mol
    v_nm3 = B.KB * 298.15 / B.ATM                   # per molecule, large-N limit
    assert v_nm3 * 6.02214076e23 * 1e-24 == pytest.approx(24.465, rel=1e-4)


def test_molecules_scale_rigidly():
    rng = np.random.default_rng(3)
    box = np.array([2.0, 2.2, 2.4])
    n_w = 20
    O = rng.uniform(0.0, 1.0, size=(n_w, 3)) * box
    O[:4] = box * 0.999                              # molecules across the boundary
    H1 = O + np.array([0.09572, 0.0, 0.0])
    H2 = O + np.array([-0.024, 0.0927, 0.0])
    pos = np.stack([O, H1, H2], axis=1).reshape(-1, 3)
    pos -= box * np.floor(pos / box)                 # wrapped, so some molecules are split
    mass = np.tile([15.999, 1.008, 1.008], n_w)
    waters = np.arange(3 * n_w).reshape(-1, 3)
    mol = B.molecule_ids(3 * n_w, np.concatenate([waters[:, [0, 1]], waters[:, [0, 2]]]))
    assert np.array_equal(mol, np.repeat(np.arange(n_w), 3))
    s = 1.03
    new, box_new = B.scale_molecules(pos, mass, mol, box, s)
    assert np.allclose(box_new, s * box)

    def whole(p, b):
        d = p[1:] - p[0]
        return d - b * np.round(d / b)

    for m in range(n_w):
        i = slice(3 * m, 3 * m + 3)
        assert np.allclose(whole(new[i], box_new), whole(pos[i], box), atol=1e-12)
        d0 = whole(pos[i], box)
        com0 = pos[3 * m] + (mass[i][1:, None] * d0).sum(0) / mass[i].sum()
        d1 = whole(new[i], box_new)
        com1 = new[3 * m] + (mass[i][1:, None] * d1).sum(0) / mass[i].sum()
        assert np.allclose(com1, s * com0, atol=1e-12)


def test_rejects_nonpositive_volume():
    assert B.accept_probability(0.0, 1.0, 1.0, 0.0, 3, 2.5) == 0.0
    box = np.array([0.5, 0.5, 0.5])
    pos = np.zeros((1, 3))
    out = B.volume_move(pos, box, np.ones(1), np.zeros(1, dtype=int), lambda x, b: 0.0, 0.0, 1.0, 2.5,
                        10.0, 0.0, 0.0)
    assert out[3] is False and out[1] is box


def test_massless_molecule_scales_about_its_geometric_centre():
    # a frozen rigid molecule (all masses 0) keeps its shape and its
    # geometric centre scales with the box
    box = np.array([3.0, 3.0, 3.0])
    ring = np.array([[0.14 * np.cos(a), 0.14 * np.sin(a), 0.0] for a in np.linspace(0, 2 * np.pi, 6, endpoint=False)])
    pos = np.vstack([ring + np.array([2.9, 1.0, 1.5]), [[0.5, 0.5, 0.5]]])
    pos -= box * np.floor(pos / box)                 # split across the x face
    mass = np.array([0.0] * 6 + [12.0])
    mol = np.array([0] * 6 + [1])
    s = 0.97
    new, box_new = B.scale_molecules(pos, mass, mol, box, s)
    d0 = pos[:6] - pos[0]
    d0 -= box * np.round(d0 / box)
    d1 = new[:6] - new[0]
    d1 -= box_new * np.round(d1 / box_new)
    assert np.allclose(d1, d0, atol=1e-12)
    c0 = pos[0] + d0.mean(axis=0)
    c1 = new[0] + d1.mean(axis=0)
    assert np.allclose(c1, s * c0, atol=1e-12)
    assert np.allclose(new[6], s * pos[6], atol=1e-12)
