"""Oracle for the Monte Carlo barostat of the paper's isothermal-isobaric runs
(Section 2.6: isotropic volume moves attempted every 50 fs at 298 K and 1 atm,
after Aqvist et al. 2004).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy float64.
The paper names the method without equations; this module states the
standard Metropolis volume move it refers to:

  propose   V' = V + dV,  dV uniform in [-dV_max, dV_max]  (rejected if V' <= 0)
  scale     every box edge by s = (V'/V)^(1/3) and every molecule's centre
            of mass by s, its atoms moved rigidly with the centre
  accept    with probability min(1, exp(-beta (U' - U + P (V' - V))
                                        + N_mol ln(V'/V)))

The N_mol ln(V'/V) term is the Jacobian of the scaled molecular centres; with
it the chain samples p(V) proportional to V^N_mol exp(-beta (U + P V)).
Reading: the centre that is scaled is the centre of mass (the published
method allows any fixed molecular reference point; the Jacobian is the same);
a molecule whose atoms are all massless (the frozen rigid solutes of the
dynamics workloads) is scaled about its geometric centre, so that it keeps its
shape and moves with the box.
"""
import math

import numpy as np

KB = 0.0083144626           # kJ mol^-1 K^-1
BAR = 0.0602214076          # 1 bar in kJ mol^-1 nm^-3 (1e5 J m^-3 x N_A / 1e3 / 1e27)
ATM = 1.01325 * BAR         # 1 atm


def molecule_ids(n_atoms, bonded_pairs):
    """Molecule index of every atom: connected components of the graph whose
    edges are the given atom pairs (bonds, constraints or exclusions), numbered
    in order of their lowest atom."""
    parent = list(range(n_atoms))

    def root(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i

    for i, j in np.asarray(bonded_pairs, dtype=np.int64).reshape(-1, 2):
        a, b = root(int(i)), root(int(j))
        if a != b:
            parent[max(a, b)] = min(a, b)
    roots = [root(i) for i in range(n_atoms)]
    number = {}
    return np.array([number.setdefault(r, len(number)) for r in roots], dtype=np.int64)


def scale_molecules(pos, mass, mol, box, s):
    """Positions and box after scaling every molecule's centre of mass by s.

    Molecules are kept whole: each atom's offset from its molecule's first
    atom is taken under the minimum image, so a molecule split by the
    periodic boundary scales as one body.  Returns (pos', box')."""
    pos = np.asarray(pos, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    out = np.empty_like(pos)
    for m in np.unique(mol):
        idx = np.flatnonzero(mol == m)
        d = pos[idx] - pos[idx[0]]
        d -= box * np.round(d / box)                 # whole molecule
        mt = mass[idx].sum()
        w = mass[idx] / mt if mt > 0.0 else np.full(idx.size, 1.0 / idx.size)
        com = pos[idx[0]] + (w[:, None] * d).sum(axis=0)
        out[idx] = s * com + (d - (w[:, None] * d).sum(axis=0))
    return out, s * box


def accept_probability(dU, P, V, V_new, n_mol, kT):
    """Metropolis probability of the volume move V -> V_new with energy change
    dU (kJ/mol) at pressure P (kJ mol^-1 nm^-3)."""
    if V_new <= 0.0:
        return 0.0
    x = -(dU + P * (V_new - V)) / kT + n_mol * math.log(V_new / V)
    return 1.0 if x >= 0.0 else math.exp(x)


def volume_move(pos, box, mass, mol, energy, U, P, kT, dV_max, u_propose, u_accept):
    """One Monte Carlo volume move.

    energy(pos, box) -> U is the potential energy; U is its value at the
    current state; u_propose and u_accept are uniforms in [0, 1) supplied by
    the caller.  Returns (pos, box, U, accepted)."""
    V = float(np.prod(box))
    V_new = V + dV_max * (2.0 * u_propose - 1.0)
    if V_new <= 0.0:
        return pos, box, U, False
    n_mol = int(np.unique(mol).size)
    pos_new, box_new = scale_molecules(pos, mass, mol, box, (V_new / V) ** (1.0 / 3.0))
    U_new = energy(pos_new, box_new)
    if u_accept < accept_probability(U_new - U, P, V, V_new, n_mol, kT):
        return pos_new, box_new, U_new, True
    return pos, box, U, False
