"""Seeded synthetic systems (inputs only; no energy or force arithmetic).

The paper's systems (one solute in 500 waters or 80 octanols, built with
PACKMOL and GAFF/AMBER parameters, Section 2.6) are not available, so these
generators build stand-ins with the same kinds of structure: rigid 3-site
waters on a lattice with random orientations, near-trans all-atom
octanol-like chains packed in layers, rigid organic-like solutes and a
flexible 22-atom N-acetyl-amino-acid-amide-like solute built from backbone
dihedrals.  Every force-field number here is synthetic.

Conventions shared by both sides of every comparison:
  * the box lengths, all coordinates, charges, sigmas and epsilons are
    float32-representable doubles (the mixed-precision path stores them in
    float32, so both sides then see identical inputs) and every coordinate is
    wrapped into [0, L) per atom;
  * ``excl`` lists every pair left out of the ordinary pair sum (1-2, 1-3,
    1-4 and, for rigid solutes, all intramolecular pairs); ``pairs14`` is the
    subset that gets scaled 1-4 terms, with ``scale14`` = (s_LJ, s_C);
  * mass 0 marks a frozen atom (the rigid solutes of the dynamics workloads);
  * ``solute`` is 1 for solute atoms, 0 for solvent atoms.

This module holds geometry, topology and random draws only.  It is shared by
the tests, the benchmark and the smoke check as the single source of inputs.
"""
import math

import numpy as np

# per-element masses (amu)
M_H, M_C, M_N, M_O = 1.008, 12.011, 14.007, 15.999

# 3-site water (configuration text: O -0.834 e, H +0.417 e, r_OH 0.09572 nm,
# HOH 104.52 deg, O sigma 0.315 nm, eps 0.636 kJ/mol; H carries no LJ)
W_Q = (-0.834, 0.417, 0.417)
W_ROH = 0.09572
W_ANG = math.radians(104.52)
W_SIG = (0.315, 0.0, 0.0)
W_EPS = (0.636, 0.0, 0.0)


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _wrap(pos, box):
    p = pos - box * np.floor(pos / box)
    p = f32(p)
    for k in range(3):
        col = p[:, k]
        col[col >= box[k]] = 0.0
        col[col < 0.0] = 0.0
    return p


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def water_geometry():
    """O at the origin, H atoms in the xy plane, bisector along +x."""
    h = W_ANG / 2
    return np.array([
        [0.0, 0.0, 0.0],
        [W_ROH * math.cos(h), W_ROH * math.sin(h), 0.0],
        [W_ROH * math.cos(h), -W_ROH * math.sin(h), 0.0],
    ])


def _place_z(a, b, c, bond, angle, dihedral):
    """NeRF: place atom d bonded to c with angle b-c-d and dihedral a-b-c-d."""
    bc = c - b
    bc /= np.linalg.norm(bc)
    n = np.cross(b - a, bc)
    n /= np.linalg.norm(n)
    m = np.cross(n, bc)
    d2 = np.array([-bond * math.cos(angle),
                   bond * math.sin(angle) * math.cos(dihedral),
                   bond * math.sin(angle) * math.sin(dihedral)])
    return c + d2[0] * bc + d2[1] * m + d2[2] * n


def _build_zmatrix(zm):
    """zm: list of (bonded_to, bond, angle_ref, angle_deg, dihedral_ref, dihedral_deg)."""
    xyz = []
    for k, (i, r, j, ang, l, dih) in enumerate(zm):
        if k == 0:
            xyz.append(np.zeros(3))
        elif k == 1:
            xyz.append(xyz[i] + np.array([r, 0.0, 0.0]))
        elif k == 2:
            a = math.radians(ang)
            v = xyz[j] - xyz[i]
            v /= np.linalg.norm(v)
            perp = np.array([-v[1], v[0], 0.0])
            if np.linalg.norm(perp) < 1e-9:
                perp = np.array([0.0, 1.0, 0.0])
            perp /= np.linalg.norm(perp)
            xyz.append(xyz[i] + r * (math.cos(a) * v + math.sin(a) * perp))
        else:
            xyz.append(_place_z(xyz[l], xyz[j], xyz[i], r, math.radians(ang), math.radians(dih)))
    return np.array(xyz)


def _graph_lists(n, bonds):
    """1-2, 1-3 and 1-4 pairs (i < j) and angle / proper-torsion tuples of a molecule."""
    adj = [set() for _ in range(n)]
    for i, j in bonds:
        adj[i].add(j)
        adj[j].add(i)
    p12 = {tuple(sorted(b)) for b in bonds}
    angles = []
    p13 = set()
    for j in range(n):
        nb = sorted(adj[j])
        for a in range(len(nb)):
            for b in range(a + 1, len(nb)):
                angles.append((nb[a], j, nb[b]))
                p13.add(tuple(sorted((nb[a], nb[b]))))
    torsions = []
    p14 = set()
    for j, k in bonds:
        for i in adj[j]:
            if i == k:
                continue
            for l in adj[k]:
                if l == j or l == i:
                    continue
                torsions.append((i, j, k, l))
                p14.add(tuple(sorted((i, l))))
    p13 -= p12
    p14 -= p12 | p13
    return sorted(p12), sorted(p13), sorted(p14), angles, torsions


def _random_charges(rng, n, lo=-0.5, hi=0.5):
    """Uniform charges shifted to zero sum, redrawn until all lie in [lo, hi]."""
    while True:
        q = rng.uniform(lo, hi, size=n)
        q -= q.mean()
        if q.min() >= lo and q.max() <= hi:
            return q


# ------------------------------------------------------------------ solutes

def solute_ring12(rng):
    """Rigid benzene-like solute: 6-ring of heavy atoms (0.14 nm) + 6 H (0.108 nm)."""
    xyz = []
    for k in range(6):
        t = 2 * math.pi * k / 6
        xyz.append([0.14 * math.cos(t), 0.14 * math.sin(t), 0.0])
    for k in range(6):
        t = 2 * math.pi * k / 6
        xyz.append([(0.14 + 0.108) * math.cos(t), (0.14 + 0.108) * math.sin(t), 0.0])
    mass = np.array([M_C] * 6 + [M_H] * 6)
    return np.array(xyz), mass


def solute_rigid20(rng):
    """Rigid 20-atom organic-like solute: naphthalene skeleton with 6 H,
    one hydroxyl (O, H) and one nitrile-like (C, N) substituent."""
    a = 0.14
    # two fused hexagons sharing the bond (c0, c1) along y
    ring = []
    for k in range(6):
        t = math.pi / 6 + 2 * math.pi * k / 6
        ring.append([a * math.cos(t), a * math.sin(t), 0.0])
    ring = np.array(ring)
    shift = np.array([2 * a * math.cos(math.pi / 6), 0.0, 0.0])
    left = ring - shift / 2
    right = ring + shift / 2
    # left ring vertices 0 (upper right) and 5 (lower right) coincide with right ring 2 and 3
    heavy = [left[k] for k in range(6)] + [right[k] for k in (0, 1, 4, 5)]
    heavy = np.array(heavy)
    centre_l = -shift / 2
    centre_r = shift / 2
    # outer carbons: left 1,2,3,4 and right 0,1(=idx7),4(=idx8),5(=idx9) -> 8 positions
    outer = [(1, centre_l), (2, centre_l), (3, centre_l), (4, centre_l),
             (6, centre_r), (7, centre_r), (8, centre_r), (9, centre_r)]
    subs = []
    for idx, cen in outer:
        v = heavy[idx] - cen
        v /= np.linalg.norm(v)
        subs.append((idx, v))
    xyz = list(heavy)
    mass = [M_C] * 10
    for k, (idx, v) in enumerate(subs):
        if k == 0:      # hydroxyl
            o = heavy[idx] + 0.136 * v
            xyz.append(o)
            perp = np.cross(v, [0, 0, 1.0])
            xyz.append(o + 0.096 * (math.cos(math.radians(71)) * v + math.sin(math.radians(71)) * perp))
            mass += [M_O, M_H]
        elif k == 4:    # nitrile-like
            c = heavy[idx] + 0.144 * v
            xyz.append(c)
            xyz.append(c + 0.115 * v)
            mass += [M_C, M_N]
        else:
            xyz.append(heavy[idx] + 0.108 * v)
            mass += [M_H]
    xyz = np.array(xyz)
    assert xyz.shape[0] == 20
    return xyz - xyz.mean(axis=0), np.array(mass)


# Ac-X-NHMe-like 22-atom solute (alanine-dipeptide topology).  Atom order:
#  0 CH3(ace) 1-3 H  4 C(ace) 5 O  6 N 7 H 8 CA 9 HA 10 CB 11-13 HB
# 14 C 15 O 16 N 17 H 18 CH3(nme) 19-21 H
DIPEPTIDE_BONDS = [(0, 1), (0, 2), (0, 3), (0, 4), (4, 5), (4, 6), (6, 7), (6, 8), (8, 9),
                   (8, 10), (10, 11), (10, 12), (10, 13), (8, 14), (14, 15), (14, 16),
                   (16, 17), (16, 18), (18, 19), (18, 20), (18, 21)]
DIPEPTIDE_ELEM = ["C", "H", "H", "H", "C", "O", "N", "H", "C", "H", "C", "H", "H", "H",
                  "C", "O", "N", "H", "C", "H", "H", "H"]
# the torsions coupled to auxiliary variables (d-AFED): phi, psi, chi
DIPEPTIDE_CVS = [(4, 6, 8, 14), (6, 8, 14, 16), (6, 8, 10, 11)]


def solute_dipeptide22(phi, psi, chi):
    """Cartesian coordinates of the 22-atom solute for backbone phi, psi and
    side-chain chi (degrees), from a Z-matrix with standard-like geometry."""
    zm = [None] * 22
    zm[4] = (None,)
    # build order: C(ace)=4, CH3=0, O=5, N=6, CA=8, C=14, N'=16, ...
    order = {}
    rows = []

    def add(atom, i=None, r=None, j=None, a=None, l=None, d=None):
        order[atom] = len(rows)
        rows.append((atom, i, r, j, a, l, d))

    add(4)
    add(0, 4, 0.152)
    add(6, 4, 0.133, 0, 116.0)
    add(5, 4, 0.123, 6, 123.0, 0, 180.0)
    add(8, 6, 0.146, 4, 122.0, 0, 180.0)   # omega(ace)
    add(14, 8, 0.152, 6, 111.0, 4, phi)     # phi = C(ace)-N-CA-C
    add(16, 14, 0.133, 8, 116.0, 6, psi)    # psi = N-CA-C-N'
    add(15, 14, 0.123, 16, 123.0, 8, 180.0)
    add(18, 16, 0.146, 14, 122.0, 8, 180.0)  # omega
    add(7, 6, 0.101, 8, 119.0, 14, 180.0 + phi)
    add(9, 8, 0.109, 6, 109.5, 14, -120.0)
    add(10, 8, 0.153, 6, 110.5, 14, 120.0)
    add(11, 10, 0.109, 8, 109.5, 6, chi)     # chi = N-CA-CB-HB1
    add(12, 10, 0.109, 8, 109.5, 6, chi + 120.0)
    add(13, 10, 0.109, 8, 109.5, 6, chi - 120.0)
    add(17, 16, 0.101, 18, 119.0, 14, 180.0)
    add(1, 0, 0.109, 4, 109.5, 6, 0.0)
    add(2, 0, 0.109, 4, 109.5, 6, 120.0)
    add(3, 0, 0.109, 4, 109.5, 6, -120.0)
    add(19, 18, 0.109, 16, 109.5, 14, 60.0)
    add(20, 18, 0.109, 16, 109.5, 14, 180.0)
    add(21, 18, 0.109, 16, 109.5, 14, -60.0)
    zrows = []
    for atom, i, r, j, a, l, d in rows:
        zrows.append((order[i] if i is not None else 0, r, order[j] if j is not None else 0,
                      a, order[l] if l is not None else 0, d))
    xyz_b = _build_zmatrix(zrows)
    xyz = np.zeros((22, 3))
    for atom, k in order.items():
        xyz[atom] = xyz_b[k]
    return xyz - xyz.mean(axis=0)


# ------------------------------------------------------------------ helpers

class _Builder:
    def __init__(self, box):
        self.box = np.asarray(box, dtype=np.float64)
        self.pos, self.q, self.sig, self.eps, self.sol, self.mass = [], [], [], [], [], []
        self.excl, self.p14, self.s14, self.waters = [], [], [], []
        self.bonds, self.bond_par, self.angles, self.angle_par = [], [], [], []
        self.tors, self.tors_par, self.cons, self.cons_len = [], [], [], []

    @property
    def n(self):
        return len(self.pos)

    def add_atoms(self, xyz, q, sig, eps, mass, solute):
        base = self.n
        for k in range(len(xyz)):
            self.pos.append(np.asarray(xyz[k], dtype=np.float64))
            self.q.append(float(q[k]))
            self.sig.append(float(sig[k]))
            self.eps.append(float(eps[k]))
            self.mass.append(float(mass[k]))
            self.sol.append(1 if solute else 0)
        return base

    def add_water(self, xyz):
        b = self.add_atoms(xyz, W_Q, W_SIG, W_EPS, (M_O, M_H, M_H), False)
        self.waters.append((b, b + 1, b + 2))
        self.excl += [(b, b + 1), (b, b + 2), (b + 1, b + 2)]
        return b

    def finish(self, **params):
        n = self.n
        box = f32(self.box)
        d = dict(
            box=box,
            pos=_wrap(np.array(self.pos), box),
            charge=f32(np.array(self.q)),
            sigma=f32(np.array(self.sig)),
            epsilon=f32(np.array(self.eps)),
            solute=np.array(self.sol, dtype=np.uint8),
            mass=np.array(self.mass),
            excl=np.array(sorted(tuple(sorted(e)) for e in self.excl), dtype=np.int32).reshape(-1, 2),
            pairs14=np.array(self.p14, dtype=np.int32).reshape(-1, 2),
            scale14=np.array(self.s14, dtype=np.float64).reshape(-1, 2),
            waters=np.array(self.waters, dtype=np.int32).reshape(-1, 3),
            bonds=np.array(self.bonds, dtype=np.int32).reshape(-1, 2),
            bond_par=np.array(self.bond_par, dtype=np.float64).reshape(-1, 2),
            angles=np.array(self.angles, dtype=np.int32).reshape(-1, 3),
            angle_par=np.array(self.angle_par, dtype=np.float64).reshape(-1, 2),
            torsions=np.array(self.tors, dtype=np.int32).reshape(-1, 4),
            torsion_par=np.array(self.tors_par, dtype=np.float64).reshape(-1, 3),
            constraints=np.array(self.cons, dtype=np.int32).reshape(-1, 2),
            constraint_len=np.array(self.cons_len, dtype=np.float64),
        )
        assert d["pos"].shape == (n, 3)
        d.update(params)
        return d


def _lattice_sites(box, n_side):
    g = (np.arange(n_side) + 0.5) / n_side
    X, Y, Z = np.meshgrid(g * box[0], g * box[1], g * box[2], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _min_image_dist(a, b, box):
    d = b[None, :, :] - a[:, None, :]
    d -= box * np.round(d / box)
    return np.sqrt((d * d).sum(-1))


def _place_waters(B, rng, sites, n_keep, avoid_xyz, avoid_r, jitter, n_orient=12):
    """Put n_keep rigid waters on lattice sites that are at least avoid_r from
    every atom in avoid_xyz; orientations are picked among n_orient random
    draws to keep hydrogens of neighbouring waters apart."""
    box = B.box
    if len(avoid_xyz):
        dmin = _min_image_dist(sites, np.asarray(avoid_xyz), box).min(axis=1)
        ok = np.nonzero(dmin >= avoid_r)[0]
    else:
        ok = np.arange(len(sites))
    if len(ok) < n_keep:
        raise ValueError("not enough free lattice sites")
    chosen = np.sort(rng.choice(ok, size=n_keep, replace=False))
    geo = water_geometry()
    placed_h = []
    cell = 0.35
    grid = {}
    nc = np.maximum(1, np.floor(box / cell).astype(int))

    def key(p):
        c = np.floor((p - box * np.floor(p / box)) / box * nc).astype(int) % nc
        return tuple(c)

    for s in chosen:
        centre = sites[s] + rng.normal(scale=jitter, size=3)
        best, best_d = None, -1.0
        near = []
        kc = key(centre)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    near += grid.get(((kc[0] + dx) % nc[0], (kc[1] + dy) % nc[1], (kc[2] + dz) % nc[2]), [])
        near = np.array(near) if near else np.zeros((0, 3))
        for _ in range(n_orient):
            R = _random_rotation(rng)
            xyz = centre + geo @ R.T
            if len(near):
                dd = _min_image_dist(xyz[1:], near, box).min()
            else:
                dd = 1.0
            if dd > best_d:
                best, best_d = xyz, dd
        B.add_water(best)
        for h in best[1:]:
            grid.setdefault(key(h), []).append(h)
            placed_h.append(h)
    return chosen


def _add_rigid_solute(B, xyz, mass, rng, frozen):
    n = len(xyz)
    q = _random_charges(rng, n)
    sig = rng.uniform(0.25, 0.35, size=n)
    eps = rng.uniform(0.1, 0.5, size=n)
    m = np.zeros(n) if frozen else mass
    b = B.add_atoms(xyz, q, sig, eps, m, True)
    # rigid: every intramolecular pair is excluded (its energy is constant)
    for i in range(n):
        for j in range(i + 1, n):
            B.excl.append((b + i, b + j))
    return b


COMMON = dict(order=4, skin=0.1, temperature=298.0, friction=10.0, k_e=138.935458)


def make_c0(seed=2608, lam=None):
    """Plain FP64 single-lambda case: 12-atom rigid solute + 216 rigid waters,
    1.86 nm box, cutoff 0.9 nm, alpha 3.12 nm^-1, PME 16^3 order 4."""
    rng = np.random.default_rng(seed)
    box = f32([1.86, 1.86, 1.86])
    B = _Builder(box)
    xyz, mass = solute_ring12(rng)
    R = _random_rotation(rng)
    xyz = box / 2 + xyz @ R.T
    _add_rigid_solute(B, xyz, mass, rng, frozen=True)
    sites = _lattice_sites(box, 7)
    _place_waters(B, rng, sites, 216, xyz, 0.30, 0.02)
    lam = float(rng.uniform(0.0, 1.0)) if lam is None else lam
    return B.finish(r_cut=0.9, r_switch=0.8, alpha=3.12, grid=[16, 16, 16], lam=lam,
                    dt=0.002, name="c0_ring12_water216", **COMMON)


def make_water_box(seed=2610, n_waters=4000, box_len=4.93, solute="rigid20", n_side=16,
                   frozen_solute=True, phi_psi_chi=None, lam=None, r_cut=1.0, grid=48):
    """Solute in rigid 3-site waters on a jittered lattice (configs with 4,000
    waters in a 4.93 nm box; smaller variants for tests)."""
    rng = np.random.default_rng(seed)
    box = f32([box_len] * 3)
    B = _Builder(box)
    avoid = np.zeros((0, 3))
    if solute == "rigid20":
        xyz, mass = solute_rigid20(rng)
        xyz = box / 2 + xyz @ _random_rotation(rng).T
        _add_rigid_solute(B, xyz, mass, rng, frozen=frozen_solute)
        avoid = xyz
    elif solute == "ring12":
        xyz, mass = solute_ring12(rng)
        xyz = box / 2 + xyz @ _random_rotation(rng).T
        _add_rigid_solute(B, xyz, mass, rng, frozen=frozen_solute)
        avoid = xyz
    elif solute == "dipeptide22":
        if phi_psi_chi is None:
            phi_psi_chi = rng.uniform(-180.0, 180.0, size=3)
        xyz = solute_dipeptide22(*phi_psi_chi)
        xyz = box / 2 + xyz @ _random_rotation(rng).T
        _add_flexible_dipeptide(B, xyz, rng)
        avoid = xyz
    elif solute is None:
        pass
    else:
        raise ValueError(solute)
    sites = _lattice_sites(box, n_side)
    _place_waters(B, rng, sites, n_waters, avoid, 0.30, 0.02)
    lam = float(rng.uniform(0.0, 1.0)) if lam is None else lam
    return B.finish(r_cut=r_cut, r_switch=r_cut - 0.1, alpha=3.12, grid=[grid] * 3, lam=lam,
                    dt=0.002, name=f"water{n_waters}_{solute}", **COMMON)


def make_c2(seed=2610, lam=None):
    """Water box of the lambda-dynamics loop: 4,000 waters + 20-atom solute
    (12,020 atoms), 4.93 nm box, PME 48^3."""
    d = make_water_box(seed=seed, lam=lam)
    d.update(lambda_mass=20.0, lambda_friction=25.0, opes_stride=500,
             opes_dE_std=30.0 * 4.184, opes_dE_exp=5.0 * 4.184, opes_sigma=0.10,
             name="c2_water4000_rigid20")
    return d


def make_c4_frame(seed=2612, frame=0):
    """One of the 64 differentiation frames: flexible 22-atom solute with
    phi, psi, chi ~ U(-180, 180] deg in 4,000 waters, lambda ~ U[0, 1]."""
    rng = np.random.default_rng([seed, frame])
    ang = rng.uniform(-180.0, 180.0, size=3)
    lam = float(rng.uniform(0.0, 1.0))
    d = make_water_box(seed=seed * 1000 + frame, solute="dipeptide22", phi_psi_chi=ang, lam=lam)
    d["name"] = f"c4_dipeptide22_frame{frame}"
    d["phi_psi_chi"] = ang
    return d


# synthetic dipeptide force field: element -> (sigma nm, eps kJ/mol)
_DP_LJ = {"C": (0.34, 0.36), "H": (0.25, 0.07), "O": (0.30, 0.88), "N": (0.325, 0.71)}
_DP_Q = {"C": 0.1, "H": 0.1, "O": -0.55, "N": -0.45}


def _add_flexible_dipeptide(B, xyz, rng):
    elem = DIPEPTIDE_ELEM
    n = len(elem)
    q = np.array([_DP_Q[e] for e in elem]) + rng.uniform(-0.05, 0.05, size=n)
    q -= q.mean()
    sig = np.array([_DP_LJ[e][0] for e in elem])
    eps = np.array([_DP_LJ[e][1] for e in elem]) * rng.uniform(0.9, 1.1, size=n)
    mass = np.array([{"C": M_C, "H": M_H, "O": M_O, "N": M_N}[e] for e in elem])
    b = B.add_atoms(xyz, q, sig, eps, mass, True)
    _add_molecule_topology(B, b, xyz, DIPEPTIDE_BONDS, elem, constrain_h=False)


def _add_molecule_topology(B, b, xyz, bonds, elem, constrain_h):
    """Bonds, angles, torsions, exclusions (1-2, 1-3), scaled 1-4 pairs
    (s_LJ 0.5, s_C 1/1.2) of one flexible molecule starting at atom b, with
    equilibrium values taken from the built geometry."""
    n = len(elem)
    p12, p13, p14, angles, tors = _graph_lists(n, bonds)
    for i, j in bonds:
        r0 = float(np.linalg.norm(xyz[j] - xyz[i]))
        is_h = elem[i].startswith("H") or elem[j].startswith("H")
        if constrain_h and is_h:
            B.cons.append((b + i, b + j))
            B.cons_len.append(r0)
        else:
            B.bonds.append((b + i, b + j))
            B.bond_par.append((2.5e5 if not is_h else 3.0e5, r0))
    for i, j, k in angles:
        u, v = xyz[i] - xyz[j], xyz[k] - xyz[j]
        th0 = math.acos(np.clip(u @ v / (np.linalg.norm(u) * np.linalg.norm(v)), -1, 1))
        B.angles.append((b + i, b + j, b + k))
        B.angle_par.append((400.0, th0))
    for i, j, k, l in tors:
        heavy = not (elem[i].startswith("H") or elem[l].startswith("H"))
        if heavy or elem[l] == "HO" or elem[i] == "HO":
            B.tors.append((b + i, b + j, b + k, b + l))
            B.tors_par.append((0.6, 3.0, 0.0))
    for i, j in p12 + p13 + p14:
        B.excl.append((b + i, b + j))
    for i, j in p14:
        B.p14.append((b + i, b + j))
        B.s14.append((0.5, 1.0 / 1.2))


# octanol-like chain: C1..C8, O, HO, then 17 H (3 on C1, 2 on C2..C8)
OCT_ELEM = ["C"] * 8 + ["O", "HO"] + ["H"] * 17
OCT_LJ = {"C": (0.34, 0.45), "H": (0.26, 0.07), "O": (0.30, 0.88), "HO": (0.0, 0.0)}
OCT_Q = {"C": -0.18, "H": 0.06, "O": -0.68, "HO": 0.42}


def octanol_chain(rng, dihedral_sd=8.0):
    """Near-trans octanol-like chain along +z (heavy-atom dihedrals drawn
    N(180, dihedral_sd) deg); returns xyz (27, 3) and the bond list."""
    zm = []
    dih = lambda: 180.0 + rng.normal(scale=dihedral_sd)
    # heavy atoms 0..7 carbons, 8 O, 9 HO
    zm.append((0, None, 0, None, 0, None))
    zm.append((0, 0.153, 0, None, 0, None))
    zm.append((1, 0.153, 0, 111.0, 0, None))
    for k in range(3, 8):
        zm.append((k - 1, 0.153, k - 2, 111.0, k - 3, dih()))
    zm.append((7, 0.143, 6, 109.5, 5, dih()))
    zm.append((8, 0.096, 7, 108.5, 6, dih()))
    # hydrogens: C1 methyl (3), C2..C8 two each
    hs = []
    for t in (60.0, 180.0, -60.0):
        hs.append((0, 0.109, 1, 109.5, 2, t))
    for k in range(1, 8):
        nxt = k + 1  # carbon k+1 or O (index 8) for k = 7
        hs.append((k, 0.109, nxt, 109.5, k - 1, 120.0))
        hs.append((k, 0.109, nxt, 109.5, k - 1, -120.0))
    rows = [(r[0], r[1], r[2], r[3], r[4], r[5]) for r in zm + hs]
    xyz = _build_zmatrix([(i, rr, j, a if a is not None else 0.0, l, d if d is not None else 0.0)
                          for (i, rr, j, a, l, d) in rows])
    bonds = [(k, k + 1) for k in range(8)] + [(8, 9)]
    bonds += [(0, 10), (0, 11), (0, 12)]
    h = 13
    for k in range(1, 8):
        bonds += [(k, h), (k, h + 1)]
        h += 2
    # orient: chain axis (C1 -> O) along +z, zigzag plane = xz
    ax = xyz[8] - xyz[0]
    ax /= np.linalg.norm(ax)
    zig = xyz[1] - 0.5 * (xyz[0] + xyz[2])
    zig -= (zig @ ax) * ax
    zig /= np.linalg.norm(zig)
    R = np.stack([zig, np.cross(ax, zig), ax])  # rows: new x, y, z
    xyz = (xyz - xyz[:9].mean(axis=0)) @ R.T
    return xyz, bonds


def _separate_chains(seed, xyzs, centres, fixed_xyz, box, r_min=0.13, rounds=20):
    """Chains (list of (27, 3) arrays around their slot centres) redrawn
    until no atom of one comes within r_min of an atom of another or of
    fixed_xyz: each round, every chain in such a contact (the later one of
    a chain-chain pair) gets a new conformation and flip at its slot, from
    a generator of its own (seeded by seed), so that starts without such
    contacts are left as drawn."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng([seed, 1])
    xyzs = [np.asarray(x, dtype=np.float64) for x in xyzs]
    n_f = len(fixed_xyz)
    for _ in range(rounds):
        allx = np.concatenate([fixed_xyz] + xyzs)
        owner = np.concatenate([np.full(n_f, -1)] + [np.full(len(x), c) for c, x in enumerate(xyzs)])
        tree = cKDTree(np.mod(allx, box), boxsize=np.asarray(box, dtype=np.float64))
        pr = tree.query_pairs(r_min, output_type="ndarray")
        a, b = owner[pr[:, 0]], owner[pr[:, 1]]
        hit = np.unique(np.maximum(a[a != b], b[a != b]))
        if hit.size == 0:
            break
        for c in hit:
            xyz, _ = octanol_chain(rng)
            if rng.random() < 0.5:
                xyz = xyz * np.array([1.0, -1.0, -1.0])
            xyzs[c] = centres[c] + xyz
    return xyzs


def make_octanol_box(seed=2609, n_chains=500, box_len=4.8, nx=12, ny=11, nz=4, lam=None,
                     mass_scale=0.1, r_cut=1.0, grid=48):
    """Octanol-like solvation box: n_chains 27-atom chains packed in nz layers
    on an nx x ny grid (alternate layers offset by half a cell), a rigid
    20-atom solute at the centre, solvent masses scaled by mass_scale."""
    rng = np.random.default_rng(seed)
    box = f32([box_len] * 3)
    B = _Builder(box)
    sxyz, smass = solute_rigid20(rng)
    sxyz = box / 2 + sxyz @ _random_rotation(rng).T
    _add_rigid_solute(B, sxyz, smass, rng, frozen=True)
    slots = []
    for iz in range(nz):
        off = 0.5 * (iz % 2)
        for ix in range(nx):
            for iy in range(ny):
                slots.append(((ix + 0.5 + off) * box[0] / nx, (iy + 0.5 + off) * box[1] / ny,
                              (iz + 0.5) * box[2] / nz))
    slots = np.array(slots)

    chains = []
    for s in slots:
        xyz, bonds = octanol_chain(rng)
        if rng.random() < 0.5:   # head/tail flip keeps the zigzag plane
            xyz = xyz * np.array([1.0, -1.0, -1.0])
        chains.append((s + xyz, bonds))
    # drop every chain that comes within 0.3 nm of the solute, then thin to n_chains
    keep = [k for k, (xyz, _) in enumerate(chains)
            if _min_image_dist(xyz, sxyz, box).min() >= 0.30]
    if len(keep) < n_chains:
        raise ValueError("not enough chain slots")
    keep = np.sort(rng.choice(keep, size=n_chains, replace=False))
    placed = _separate_chains(seed, [chains[k][0] for k in keep], slots[keep], sxyz, box)
    for k, xyz in zip(keep, placed):
        bonds = chains[k][1]
        q = np.array([OCT_Q[e] for e in OCT_ELEM])
        q[7] = -0.18 + 0.68     # neutralise: the carbon bonded to O carries +0.50 e
        sig = np.array([OCT_LJ[e][0] for e in OCT_ELEM])
        eps = np.array([OCT_LJ[e][1] for e in OCT_ELEM])
        mass = np.array([{"C": M_C, "H": M_H, "O": M_O, "HO": M_H}[e] for e in OCT_ELEM]) * mass_scale
        b = B.add_atoms(xyz, q, sig, eps, mass, False)
        _add_molecule_topology(B, b, xyz, bonds, OCT_ELEM, constrain_h=True)
    lam = float(rng.uniform(0.0, 1.0)) if lam is None else lam
    return B.finish(r_cut=r_cut, r_switch=r_cut - 0.1, alpha=3.12, grid=[grid] * 3, lam=lam,
                    dt=0.002, lambda_mass=20.0, lambda_friction=25.0, opes_stride=500,
                    opes_dE_std=30.0 * 4.184, opes_dE_exp=5.0 * 4.184, opes_sigma=0.10,
                    name=f"octanol{n_chains}_rigid20", **COMMON)


def make_c1(seed=2609, lam=None):
    """Octanol solvation box: 500 chains + 20-atom solute (13,520 atoms), 4.8 nm,
    cutoff 1.0 nm, PME 48^3, octanol masses x 0.1.  Time step 1 fs: with the
    hydrogen masses scaled to 0.1 amu the H-C-H bending period is ~7 fs and
    the constrained leapfrog diverges at 2 fs (the paper runs 1 fs).  The
    lattice start is denser than liquid octanol and has close H-H contacts:
    runs begin with a short small-step, high-friction equilibration."""
    d = make_octanol_box(seed=seed, lam=lam)
    d["name"] = "c1_octanol500_rigid20"
    d["dt"] = 0.001
    return d


def batch_lambdas(n=32):
    """lambda_r = r / (n - 1), r = 0..n-1."""
    return [r / (n - 1) for r in range(n)]


def subsystem(d, keep):
    """Copy of system d restricted to the atoms in `keep` (sorted index array),
    with topology lists remapped and pairs touching removed atoms dropped."""
    keep = np.asarray(keep)
    remap = -np.ones(len(d["charge"]), dtype=np.int64)
    remap[keep] = np.arange(len(keep))
    out = dict(d)
    for k in ("pos",):
        out[k] = d[k][keep]
    for k in ("charge", "sigma", "epsilon", "solute", "mass"):
        out[k] = d[k][keep]

    def remap_list(a, par=None):
        if a.size == 0:
            return a, par
        m = remap[a]
        ok = (m >= 0).all(axis=1)
        return m[ok].astype(np.int32), (par[ok] if par is not None else None)

    out["excl"], _ = remap_list(d["excl"])
    out["pairs14"], out["scale14"] = remap_list(d["pairs14"], d["scale14"])
    out["waters"], _ = remap_list(d["waters"])
    out["bonds"], out["bond_par"] = remap_list(d["bonds"], d["bond_par"])
    out["angles"], out["angle_par"] = remap_list(d["angles"], d["angle_par"])
    out["torsions"], out["torsion_par"] = remap_list(d["torsions"], d["torsion_par"])
    out["constraints"], out["constraint_len"] = remap_list(d["constraints"], d["constraint_len"])
    return out
