"""ctypes front end of the C oracle plus the lambda assembly of Eq. 4.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Level 1 = real-space pairs + direct Ewald k-sum (the definition).
Level 2 = real-space pairs + smooth PME with a naive DFT on the same grid as
the CUDA path (Essmann 1995).  Level 0 = real space only (no reciprocal,
self or background term).
"""
import ctypes
import math
import os

import numpy as np

from .build import build

E_NAMES = [
    "U_vv", "U_uu", "U_uv", "U_soft",
    "coul_real_vv", "coul_real_uu", "coul_real_uv",
    "rec_vv", "rec_uu", "rec_uv",
    "self_vv", "self_uu",
    "bg_vv", "bg_uu", "bg_uv",
    "lj_vv", "lj_uu", "lj_uv",
    "excl_vv", "excl_uu", "excl_uv",
    "p14_vv", "p14_uu",
    "n_pairs", "dUsc_dl",
]
NE = len(E_NAMES)


class _Params(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("r_cut", ctypes.c_double),
        ("r_switch", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("level", ctypes.c_int),
        ("kmax", ctypes.c_int * 3),
        ("grid", ctypes.c_int * 3),
        ("order", ctypes.c_int),
        ("sc_alpha", ctypes.c_double),
        ("sc_power", ctypes.c_double),
        ("sc_lambda", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.orc_ucap.restype = d
        _lib.orc_ucap.argtypes = [d, dp]
        _lib.orc_S22.restype = d
        _lib.orc_S22.argtypes = [d, dp]
        _lib.orc_S32.restype = d
        _lib.orc_S32.argtypes = [d, dp]
        _lib.orc_switch.restype = d
        _lib.orc_switch.argtypes = [d, d, d, dp]
        _lib.orc_switching.restype = None
        _lib.orc_switching.argtypes = [d, dp, dp, dp, dp]
        _lib.orc_bspline.restype = d
        _lib.orc_bspline.argtypes = [ctypes.c_int, d]
        _lib.orc_bmod2.restype = d
        _lib.orc_bmod2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib.orc_dihedral.restype = d
        _lib.orc_dihedral.argtypes = [dp, dp, dp, dp, dp]
        _lib.orc_dihedral_grad.restype = d
        _lib.orc_dihedral_grad.argtypes = [dp, dp, dp, dp, dp, dp]
        _lib.orc_bonded.restype = d
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def _ptr(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ------------------------------------------------------------ scalar pieces

def ucap(x):
    """u_cap(x) and du/dx (Eq. 6)."""
    du = ctypes.c_double()
    u = lib().orc_ucap(float(x), ctypes.byref(du))
    return u, du.value


def S22(x):
    d = ctypes.c_double()
    v = lib().orc_S22(float(x), ctypes.byref(d))
    return v, d.value


def S32(x):
    d = ctypes.c_double()
    v = lib().orc_S32(float(x), ctypes.byref(d))
    return v, d.value


def lj_switch(r, rc, rs):
    d = ctypes.c_double()
    v = lib().orc_switch(float(r), float(rc), float(rs), ctypes.byref(d))
    return v, d.value


def switching(lam):
    """(h_A, h_B, dh_A/dlambda, dh_B/dlambda) of Eq. 7-8."""
    a, b, da, db = (ctypes.c_double() for _ in range(4))
    lib().orc_switching(float(lam), ctypes.byref(a), ctypes.byref(b), ctypes.byref(da), ctypes.byref(db))
    return a.value, b.value, da.value, db.value


def bspline(n, u):
    return lib().orc_bspline(int(n), float(u))


def bmod2(n, K, m):
    return lib().orc_bmod2(int(n), int(K), int(m))


def dihedral(a, b, c, d, box):
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (a, b, c, d, box)]
    return lib().orc_dihedral(*[_ptr(x) for x in arrs])


def dihedral_grad(a, b, c, d, box):
    """(phi, dphi/dr [4, 3]) in the convention of the torsion terms."""
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (a, b, c, d, box)]
    g = np.zeros(12)
    phi = lib().orc_dihedral_grad(*[_ptr(x) for x in arrs], _ptr(g))
    return phi, g.reshape(4, 3)


# --------------------------------------------------------- nonbonded energy

def kmax_for(box, alpha, tol=1e-17):
    """Smallest |m| per axis with exp(-pi^2 m^2 / (L^2 alpha^2)) < tol."""
    f = math.sqrt(-math.log(tol)) / math.pi
    return [int(math.ceil(L * alpha * f)) for L in box]


def nonbonded(sysd, level=2, alpha=None, kmax=None, grid=None, order=None,
              r_cut=None, r_switch=None, solute=None, pos=None, forces=True, sc_lambda=None):
    """Basis energies and basis forces of the nonbonded part of Eq. 4.

    Returns (E dict, F0, Fuv, Fsoft) with F0 = -grad(U_vv + U_uu),
    Fuv = -grad U_uv, Fsoft = -grad U_soft, each (N, 3) or None.
    With sysd["sc_alpha"] > 0 (soft-core coupling) the soft slot holds the
    soft-core solute-solvent LJ at sc_lambda and E["dUsc_dl"] its lambda
    derivative (see lfe_oracle.c).
    """
    L = lib()
    box = np.asarray(sysd["box"], dtype=np.float64)
    pos = np.ascontiguousarray(sysd["pos"] if pos is None else pos, dtype=np.float64)
    n = pos.shape[0]
    q = np.ascontiguousarray(sysd["charge"], dtype=np.float64)
    sig = np.ascontiguousarray(sysd["sigma"], dtype=np.float64)
    eps = np.ascontiguousarray(sysd["epsilon"], dtype=np.float64)
    sol = np.ascontiguousarray(sysd["solute"] if solute is None else solute, dtype=np.uint8)
    excl = np.ascontiguousarray(sysd["excl"], dtype=np.int32).reshape(-1, 2)
    p14 = np.ascontiguousarray(sysd["pairs14"], dtype=np.int32).reshape(-1, 2)
    s14 = np.ascontiguousarray(sysd["scale14"], dtype=np.float64).reshape(-1, 2)
    p = _Params()
    for k in range(3):
        p.box[k] = box[k]
    p.r_cut = sysd["r_cut"] if r_cut is None else r_cut
    p.r_switch = sysd["r_switch"] if r_switch is None else r_switch
    p.alpha = sysd["alpha"] if alpha is None else alpha
    p.level = int(level)
    km = kmax if kmax is not None else kmax_for(box, p.alpha)
    g = grid if grid is not None else sysd["grid"]
    for k in range(3):
        p.kmax[k] = int(km[k])
        p.grid[k] = int(g[k])
    p.order = int(sysd["order"] if order is None else order)
    p.sc_alpha = float(sysd.get("sc_alpha", 0.0) or 0.0)
    p.sc_power = float(sysd.get("sc_power", 1.0) or 1.0)
    if p.sc_alpha > 0.0:
        if sc_lambda is None:
            raise ValueError("soft-core coupling needs sc_lambda")
        p.sc_lambda = float(sc_lambda)
    E = np.zeros(NE)
    F = [np.zeros((n, 3)) if forces else None for _ in range(3)]
    rc = L.orc_nonbonded(
        ctypes.byref(p), ctypes.c_int(n), _ptr(pos), _ptr(q), _ptr(sig), _ptr(eps),
        _ptr(sol, ctypes.c_ubyte), ctypes.c_int(excl.shape[0]), _ptr(excl, ctypes.c_int),
        ctypes.c_int(p14.shape[0]), _ptr(p14, ctypes.c_int), _ptr(s14), _ptr(E),
        _ptr(F[0]), _ptr(F[1]), _ptr(F[2]))
    if rc != 0:
        raise ValueError(f"oracle rejected the input (code {rc})")
    return dict(zip(E_NAMES, E)), F[0], F[1], F[2]


def bonded(sysd, pos=None, forces=True):
    """Bonded energy (bonds, angles, torsions) and its force."""
    L = lib()
    box = np.ascontiguousarray(sysd["box"], dtype=np.float64)
    pos = np.ascontiguousarray(sysd["pos"] if pos is None else pos, dtype=np.float64)
    n = pos.shape[0]
    arrs = {}
    for name, w, dt in (("bonds", 2, np.int32), ("bond_par", 2, np.float64),
                        ("angles", 3, np.int32), ("angle_par", 2, np.float64),
                        ("torsions", 4, np.int32), ("torsion_par", 3, np.float64)):
        a = sysd.get(name)
        arrs[name] = np.ascontiguousarray(np.zeros((0, w)) if a is None else a, dtype=dt).reshape(-1, w)
    F = np.zeros((n, 3)) if forces else None
    ci = ctypes.c_int
    U = L.orc_bonded(
        _ptr(box), ci(n), _ptr(pos),
        ci(arrs["bonds"].shape[0]), _ptr(arrs["bonds"], ci), _ptr(arrs["bond_par"]),
        ci(arrs["angles"].shape[0]), _ptr(arrs["angles"], ci), _ptr(arrs["angle_par"]),
        ci(arrs["torsions"].shape[0]), _ptr(arrs["torsions"], ci), _ptr(arrs["torsion_par"]),
        _ptr(F))
    return U, F


def evaluate(sysd, lam, level=2, with_bonded=True, **kw):
    """U(lambda), dU/dlambda and F(lambda) of Eq. 4 (plus bonded terms).

    dU/dlambda = h_A'(lambda) U_uv + h_B'(lambda) U_soft (the lambda
    dependence enters only through h_A and h_B, Section 2.2).
    """
    sc = float(sysd.get("sc_alpha", 0.0) or 0.0) > 0.0
    E, F0, Fuv, Fs = nonbonded(sysd, level=level, sc_lambda=lam if sc else None, **kw)
    hA, hB, dhA, dhB = switching(lam)
    Ub, Fb = (0.0, None)
    if with_bonded:
        Ub, Fb = bonded(sysd, pos=kw.get("pos"))
    # linear-basis coupling: h_B weights the capped soft basis; soft-core
    # coupling: the soft slot is already the soft-core term at lambda
    wS, dS = (1.0, E["dUsc_dl"]) if sc else (hB, dhB * E["U_soft"])
    U = E["U_vv"] + E["U_uu"] + hA * E["U_uv"] + wS * E["U_soft"] + Ub
    dU = dhA * E["U_uv"] + dS
    F = None
    if F0 is not None:
        F = F0 + hA * Fuv + wS * Fs
        if Fb is not None:
            F = F + Fb
    return {"U": U, "dUdl": dU, "F": F, "E": E, "U_bonded": Ub,
            "hA": hA, "hB": hB, "dhA": dhA, "dhB": dhB}


def num_threads():
    return lib().orc_num_threads()


def param_grad(sysd, level=2, pos=None, charge=None, sigma=None, epsilon=None, **kw):
    """Class-resolved parameter gradients G[n, 3 (q, sigma, eps), 3 (own, uv, soft)]."""
    L = lib()
    box = np.asarray(sysd["box"], dtype=np.float64)
    pos = np.ascontiguousarray(sysd["pos"] if pos is None else pos, dtype=np.float64)
    n = pos.shape[0]
    q = np.ascontiguousarray(sysd["charge"] if charge is None else charge, dtype=np.float64)
    sig = np.ascontiguousarray(sysd["sigma"] if sigma is None else sigma, dtype=np.float64)
    eps = np.ascontiguousarray(sysd["epsilon"] if epsilon is None else epsilon, dtype=np.float64)
    sol = np.ascontiguousarray(sysd["solute"], dtype=np.uint8)
    excl = np.ascontiguousarray(sysd["excl"], dtype=np.int32).reshape(-1, 2)
    p14 = np.ascontiguousarray(sysd["pairs14"], dtype=np.int32).reshape(-1, 2)
    s14 = np.ascontiguousarray(sysd["scale14"], dtype=np.float64).reshape(-1, 2)
    p = _Params()
    for k in range(3):
        p.box[k] = box[k]
    p.r_cut = kw.get("r_cut", sysd["r_cut"])
    p.r_switch = kw.get("r_switch", sysd["r_switch"])
    p.alpha = kw.get("alpha", sysd["alpha"])
    p.level = int(level)
    km = kw.get("kmax") or kmax_for(box, p.alpha)
    g = kw.get("grid") or sysd["grid"]
    for k in range(3):
        p.kmax[k] = int(km[k])
        p.grid[k] = int(g[k])
    p.order = int(sysd["order"])
    G = np.zeros((n, 9))
    ci = ctypes.c_int
    rc = L.orc_param_grad(ctypes.byref(p), ci(n), _ptr(pos), _ptr(q), _ptr(sig), _ptr(eps),
                          _ptr(sol, ctypes.c_ubyte), ci(excl.shape[0]), _ptr(excl, ci),
                          ci(p14.shape[0]), _ptr(p14, ci), _ptr(s14), _ptr(G))
    if rc != 0:
        raise ValueError("oracle rejected the input")
    return G.reshape(n, 3, 3)


def assemble_param_grad(G, lam):
    """dU/dp and d2U/dlambda dp from the class-resolved gradients (Eq. 4)."""
    hA, hB, dA, dB = switching(lam)
    dU = G[:, :, 0] + hA * G[:, :, 1] + hB * G[:, :, 2]
    d2 = dA * G[:, :, 1] + dB * G[:, :, 2]
    return dU, d2
