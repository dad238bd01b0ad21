"""Oracle for the extended-variable loop: mirror map, OPES bias, Langevin
middle-scheme steps with constraints, and the Philox counter RNG.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy float64,
written from the paper's equations and the published definitions cited on
each function.
"""
import math

import numpy as np

KB = 0.0083144626  # kJ mol^-1 K^-1

# ------------------------------------------------------------------ Philox
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
# as 1, 2, 3", SC 2011): 10 rounds of two 32x32->64 multiplies with the
# published multipliers and Weyl key increments.
_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    c = [int(x) & _MASK for x in ctr]
    k0, k1 = int(key[0]) & _MASK, int(key[1]) & _MASK
    for _ in range(10):
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> 32, p0 & _MASK
        hi1, lo1 = p1 >> 32, p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c


def uniforms(ctr, key):
    """Four uniforms in (0, 1): (x + 0.5) / 2^32."""
    return [(x + 0.5) / 4294967296.0 for x in philox4x32_10(ctr, key)]


def normals3(ctr, key):
    """Three standard normals by the Box-Muller transform of the four uniforms
    (u0, u1) -> (n0, n1), (u2, u3) -> n2."""
    u = uniforms(ctr, key)
    r0 = math.sqrt(-2.0 * math.log(u[0]))
    r1 = math.sqrt(-2.0 * math.log(u[2]))
    return (r0 * math.cos(2 * math.pi * u[1]), r0 * math.sin(2 * math.pi * u[1]),
            r1 * math.cos(2 * math.pi * u[3]))


def seed_key(seed):
    return (seed & _MASK, (seed >> 32) & _MASK)


def atom_normals(n, step, seed):
    """Normals for atoms 0..n-1 at a step: counter (i, step_lo, step_hi, 0)."""
    key = seed_key(seed)
    out = np.empty((n, 3))
    for i in range(n):
        out[i] = normals3((i, step & _MASK, step >> 32, 0), key)
    return out


def theta_normal(step, seed):
    """Normal for the alchemical variable: counter (0, step_lo, step_hi, 1)."""
    return normals3((0, step & _MASK, step >> 32, 1), seed_key(seed))[0]


# -------------------------------------------------------------- mirror map

def theta_to_lambda(theta):
    """Eq. 3: lambda = theta on [0, 1], 2 - theta on (1, 2]; theta is wrapped
    into [0, 2) first.  Returns (lambda, dlambda/dtheta)."""
    th = theta - 2.0 * math.floor(theta / 2.0)
    if th <= 1.0:
        return th, 1.0
    return 2.0 - th, -1.0


# -------------------------------------------------------------------- OPES

class Opes:
    """One OPES bias on theta (Eq. 11-13).

    kind = "std" (OPES-Standard: nu = 1 - 1/gamma, kernel weight exp(beta V))
    or "exp" (OPES-Explore: nu = gamma - 1, unit weights).
    rho_hat(theta) = sum_k w_k G_k(theta) / sum_k w_k with periodic Gaussian
    kernels of width sigma on theta (period 2); rho_bar is the mean of rho_hat
    over the kernel centres; V = (nu/beta) ln(rho_hat/rho_bar + eps), and V = 0
    before the first deposit.
    """

    def __init__(self, kind, dE, sigma, T):
        self.kind = kind
        self.beta = 1.0 / (KB * T)
        self.gamma = self.beta * dE
        self.nu = (1.0 - 1.0 / self.gamma) if kind == "std" else (self.gamma - 1.0)
        self.eps = math.exp(-self.beta * dE / self.nu)
        self.sigma = sigma
        self.c = []
        self.w = []
        self.rho_bar = 0.0

    @staticmethod
    def _pdiff(a, b):
        d = a - b
        return d - 2.0 * math.floor((d + 1.0) / 2.0)

    def _rho(self, th):
        if not self.c:
            return 0.0, 0.0
        s = ds = 0.0
        for ck, wk in zip(self.c, self.w):
            d = self._pdiff(th, ck)
            g = math.exp(-0.5 * d * d / (self.sigma * self.sigma))
            s += wk * g
            ds += wk * g * (-d / (self.sigma * self.sigma))
        W = sum(self.w)
        return s / W, ds / W

    def bias(self, th):
        """(V(theta), dV/dtheta)."""
        if not self.c:
            return 0.0, 0.0
        r, dr = self._rho(th)
        a = r / self.rho_bar + self.eps
        return self.nu / self.beta * math.log(a), self.nu / self.beta * (dr / self.rho_bar) / a

    def deposit(self, th, v_other=0.0):
        """Append a kernel at th.  A Standard kernel's weight undoes the whole
        bias the trajectory feels at th: exp(beta (V(th) + v_other)), with
        v_other the other bias of the dual protocol at th (0 for a single
        bias); both are taken before this deposit.  Explore weights are 1."""
        w = math.exp(self.beta * (self.bias(th)[0] + v_other)) if self.kind == "std" else 1.0
        self.c.append(th - 2.0 * math.floor(th / 2.0))
        self.w.append(w)
        self.rho_bar = sum(self._rho(ck)[0] for ck in self.c) / len(self.c)


def opes_dual_deposit(std, exp, th):
    """Deposit at th into the biases of Eq. 14 (either may be None): each is
    updated separately, the Standard weight uses the total bias at th, and
    both biases are evaluated before either deposit."""
    Vs = std.bias(th)[0] if std is not None else 0.0
    Ve = exp.bias(th)[0] if exp is not None else 0.0
    if std is not None:
        std.deposit(th, v_other=Ve)
    if exp is not None:
        exp.deposit(th, v_other=Vs)


# -------------------------------------------------------------- constraints

def shake(x_new, x_ref, pairs, lengths, w, box, tol=1e-13, max_iter=100000):
    """Iterate SHAKE to convergence: move x_new along the reference bond
    vectors (inverse-mass weighted) until every |r_ij| equals its length."""
    x = x_new.copy()
    for _ in range(max_iter):
        worst = 0.0
        for (i, j), d0 in zip(pairs, lengths):
            r = x[j] - x[i]
            r -= box * np.round(r / box)
            r0 = x_ref[j] - x_ref[i]
            r0 -= box * np.round(r0 / box)
            diff = r @ r - d0 * d0
            worst = max(worst, abs(diff) / (d0 * d0))
            wsum = w[i] + w[j]
            if wsum == 0.0:
                continue
            g = diff / (2.0 * wsum * (r @ r0))
            x[i] += g * w[i] * r0
            x[j] -= g * w[j] * r0
        if worst < tol:
            return x
    raise RuntimeError("SHAKE did not converge")


def constraint_list(sysd):
    """All distance constraints: the three of each rigid water and the X-H list."""
    pairs, lens = [], []
    from_geo = {}
    r_oh = 0.09572
    ang = math.radians(104.52)
    r_hh = 2.0 * r_oh * math.sin(ang / 2.0)
    for o, h1, h2 in np.asarray(sysd.get("waters", np.zeros((0, 3), int))):
        pairs += [(o, h1), (o, h2), (h1, h2)]
        lens += [r_oh, r_oh, r_hh]
    for (i, j), d0 in zip(np.asarray(sysd.get("constraints", np.zeros((0, 2), int))),
                          np.asarray(sysd.get("constraint_len", np.zeros(0)))):
        pairs.append((int(i), int(j)))
        lens.append(float(d0))
    return pairs, lens


# ---------------------------------------------------------------- stepping

def langevin_middle_step(x, v, F, mass, dt, gamma, T, normals, box, pairs, lengths):
    """One step of the Langevin middle scheme (Zhang et al. 2019, cited in
    Section 2.6): kick v += dt F/m; half drift; Ornstein-Uhlenbeck
    v = a v + sqrt(kT (1 - a^2)/m) R, a = exp(-gamma dt); half drift;
    constrain the new positions.  The velocity carried to the next step is
    the post-noise one plus the constraint displacement over dt,
    v = v_OU + (x_constrained - x_unconstrained)/dt (for an unconstrained
    atom simply v_OU).  Atoms of mass 0 stay fixed."""
    w = np.where(mass > 0, 1.0 / np.where(mass > 0, mass, 1.0), 0.0)
    a = math.exp(-gamma * dt)
    v = v + dt * w[:, None] * F
    xn = x + 0.5 * dt * v
    sd = np.sqrt(KB * T * (1.0 - a * a) * w)
    v = a * v + sd[:, None] * normals
    xn = xn + 0.5 * dt * v
    if pairs:
        xc = shake(xn, x, pairs, lengths, w, box)
        v = v + (xc - xn) / dt
        xn = xc
    v[w == 0.0] = 0.0
    xn[w == 0.0] = x[w == 0.0]
    return xn, v


def theta_step(theta, p_theta, dUdl, dlam_dtheta, dV, m, dt, gamma, T, normal):
    """The same middle scheme for theta with momentum p_theta = m dtheta/dt and
    generalized force -(dlambda/dtheta) dU/dlambda - dV_OPES/dtheta."""
    f = -dlam_dtheta * dUdl - dV
    vt = p_theta / m + dt * f / m
    th = theta + 0.5 * dt * vt
    a = math.exp(-gamma * dt)
    vt = a * vt + math.sqrt(KB * T * (1.0 - a * a) / m) * normal
    th = th + 0.5 * dt * vt
    return th - 2.0 * math.floor(th / 2.0), m * vt


# ----------------------------------- regulated Nose-Hoover-Langevin (RNHL)
# Section 2.6 couples the extended variables to the regulated Nose-Hoover-
# Langevin thermostat of Abreu and Tuckerman (time constant 40 fs, friction
# 25 ps^-1, regulation parameter 1) without restating it.  Written here from
# that method's definition, for one variable of mass m at temperature T:
#   kinetic function  K(p) = n kT ln cosh(p / sqrt(n m kT)),
#   dx/dt   = K'(p) = sqrt(n kT / m) tanh(p / sqrt(n m kT))   (regulated velocity,
#             bounded by sqrt(n kT / m); p / m as n -> infinity)
#   dp/dt   = f - v_eta p                                       (Nose-Hoover friction)
#   dv_eta  = (p K'(p) - kT) / Q dt - gamma v_eta dt + sqrt(2 gamma kT / Q) dW,
#   Q = kT tau^2.
# Its invariant density is exp(-(U(x) + K(p) + Q v_eta^2 / 2) / kT): the
# position marginal is Boltzmann, <p K'(p)> = kT, <v_eta^2> = kT / Q.
# Reading: the step keeps the leapfrog middle layout of the atoms (full
# kick, half drift, thermostat, half drift) with the thermostat part split
# symmetrically as NH(dt/2) OU(dt) NH(dt/2), where NH(h) is
#   v_eta += h/2 G(p); p *= exp(-v_eta h); v_eta += h/2 G(p), with
# G(p) = (p K'(p) - kT) / Q, and OU(dt) the exact Ornstein-Uhlenbeck step of
# v_eta with the variable's standard normal.

def regulated_velocity(p, m, kT, n):
    """K'(p) = sqrt(n kT / m) tanh(p / sqrt(n m kT))."""
    return np.sqrt(n * kT / m) * np.tanh(p / np.sqrt(n * m * kT))


def nhl_thermostat(p, v_eta, m, kT, Q, gamma, n, dt, normal):
    """The thermostat part of one RNHL step: NH(dt/2), OU(dt), NH(dt/2)."""
    def nh(p, v_eta, h):
        v_eta = v_eta + 0.5 * h * (p * regulated_velocity(p, m, kT, n) - kT) / Q
        p = p * np.exp(-v_eta * h)
        v_eta = v_eta + 0.5 * h * (p * regulated_velocity(p, m, kT, n) - kT) / Q
        return p, v_eta
    p, v_eta = nh(p, v_eta, 0.5 * dt)
    a = math.exp(-gamma * dt)
    v_eta = a * v_eta + np.sqrt(kT * (1.0 - a * a) / Q) * normal
    p, v_eta = nh(p, v_eta, 0.5 * dt)
    return p, v_eta


def rnhl_step(x, p, v_eta, f, m, dt, gamma, T, tau, n, normal):
    """One RNHL step of a variable at x with momentum p under force f:
    p += dt f; x += dt/2 K'(p); thermostat; x += dt/2 K'(p).  Works on
    scalars and on numpy arrays of independent variables."""
    kT = KB * T
    Q = kT * tau * tau
    p = p + dt * f
    x = x + 0.5 * dt * regulated_velocity(p, m, kT, n)
    p, v_eta = nhl_thermostat(p, v_eta, m, kT, Q, gamma, n, dt, normal)
    x = x + 0.5 * dt * regulated_velocity(p, m, kT, n)
    return x, p, v_eta


def theta_step_rnhl(theta, p_theta, v_eta, dUdl, dlam_dtheta, dV, m, dt, gamma, T, tau, n, normal):
    """theta_step under RNHL: the same generalized force, theta wrapped
    into [0, 2).  Returns (theta, p_theta, v_eta)."""
    f = -dlam_dtheta * dUdl - dV
    th, p, v_eta = rnhl_step(theta, p_theta, v_eta, f, m, dt, gamma, T, tau, n, normal)
    return th - 2.0 * math.floor(th / 2.0), p, v_eta


def dafed_step_rnhl(s, p, v_eta, Fs, m, dt, gamma, T, tau, n, normal):
    """dafed_step under RNHL at the auxiliary temperature T; s wrapped into
    [-pi, pi).  Returns (s, p, v_eta)."""
    x, p, v_eta = rnhl_step(s, p, v_eta, Fs, m, dt, gamma, T, tau, n, normal)
    return wrap_angle(x), p, v_eta


# ------------------------------------------------ thermodynamic integration
# Eq. 2: Delta G = integral over lambda in [0, 1] of <dU/dlambda>_lambda.  The
# conditional mean is accumulated in TI_BINS equal bins of lambda (bin b holds
# lambda in [b/n, (b+1)/n), lambda = 1 in the last bin) and the profile of the
# bin means, placed at the bin centres, is integrated by the trapezoid rule;
# on [0, first centre] and [last centre, 1] the line through the two nearest
# occupied centres is extended (a constant if only one bin is occupied).
TI_BINS = 100


class TIAccumulator:
    def __init__(self, n=TI_BINS):
        self.n = n
        self.sum = np.zeros(n)
        self.count = np.zeros(n, dtype=np.int64)

    def add(self, lam, dUdl):
        b = min(self.n - 1, int(math.floor(lam * self.n)))
        self.sum[b] += dUdl
        self.count[b] += 1

    def means(self):
        m = np.full(self.n, np.nan)
        occ = self.count > 0
        m[occ] = self.sum[occ] / self.count[occ]
        return m

    def delta_g(self):
        occ = np.flatnonzero(self.count > 0)
        if occ.size == 0:
            return float("nan")
        x = (occ + 0.5) / self.n
        y = self.sum[occ] / self.count[occ]
        if occ.size == 1:
            return float(y[0])
        total = 0.0
        for k in range(occ.size - 1):
            total += 0.5 * (y[k] + y[k + 1]) * (x[k + 1] - x[k])
        # linear extension to lambda = 0 and lambda = 1
        s0 = (y[1] - y[0]) / (x[1] - x[0])
        y0 = y[0] - s0 * x[0]
        total += 0.5 * (y0 + y[0]) * x[0]
        s1 = (y[-1] - y[-2]) / (x[-1] - x[-2])
        y1 = y[-1] + s1 * (1.0 - x[-1])
        total += 0.5 * (y[-1] + y1) * (1.0 - x[-1])
        return total


# ------------------------------------------------------------------ d-AFED
# Eq. 15: U = sum_k kappa_k / 2 (xi_k(r) - s_k)^2, the difference taken as a
# periodic angle in [-pi, pi).  xi_k is the dihedral of four atoms, with the
# oracle's torsion convention and gradient (reference.dihedral_grad, pinned
# by central differences in the bonded tests).

def wrap_angle(x):
    """x in [-pi, pi)."""
    return x - 2.0 * math.pi * math.floor((x + math.pi) / (2.0 * math.pi))


def dihedral_grad(pos, idx, box):
    """(xi, dxi/dr[4, 3]) of the dihedral of atoms idx = (a, b, c, d)."""
    from . import reference as R
    return R.dihedral_grad(*(pos[i] for i in idx), box)


def dafed_energy_forces(pos, cvs, s, kappa, box):
    """(U, forces on atoms [N, 3], forces on s [K]) of Eq. 15."""
    F = np.zeros_like(np.asarray(pos, dtype=np.float64))
    Fs = np.zeros(len(cvs))
    U = 0.0
    for k, idx in enumerate(cvs):
        xi, g = dihedral_grad(pos, idx, box)
        dlt = wrap_angle(xi - s[k])
        U += 0.5 * kappa[k] * dlt * dlt
        for j, atom in enumerate(idx):
            F[atom] -= kappa[k] * dlt * g[j]
        Fs[k] = kappa[k] * dlt
    return U, F, Fs


def dafed_masses(pos, cvs, mass, c, box):
    """Eq. 16: m_s = c [sum_i ||d xi / d r_i||^2 / m_i]^-1 (massless = fixed atoms skipped)."""
    out = np.zeros(len(cvs))
    for k, idx in enumerate(cvs):
        _, g = dihedral_grad(pos, idx, box)
        tot = 0.0
        for j, atom in enumerate(idx):
            if mass[atom] > 0.0:
                tot += np.dot(g[j], g[j]) / mass[atom]
        out[k] = c / tot
    return out


def dafed_normal(k, step, seed):
    """Normal of auxiliary variable k at a step: counter (k, step_lo, step_hi, 2)."""
    return normals3((k, step & _MASK, step >> 32, 2), seed_key(seed))[0]


def dafed_step(s, p, Fs, m, dt, gamma, T, normal):
    """Middle scheme for one auxiliary variable at its own temperature T:
    kick, half drift, Ornstein-Uhlenbeck, half drift; s wrapped into [-pi, pi)."""
    v = p / m + dt * Fs / m
    x = s + 0.5 * dt * v
    a = math.exp(-gamma * dt)
    v = a * v + math.sqrt(KB * T * (1.0 - a * a) / m) * normal
    x = x + 0.5 * dt * v
    return wrap_angle(x), m * v


# ------------------------------------------------- lambda replica exchange

def hrex_delta(lam_a, lam_b, uuv_i, usoft_i, uuv_j, usoft_j):
    """Energy change of swapping lambda between replica i (at lam_a) and
    replica j (at lam_b).  With the potential linear in the two basis
    energies (Eq. 4), U(x; lam) = U_0(x) + h_A(lam) U_uv(x) + h_B(lam) U_soft(x),
    so  [U(x_i; b) + U(x_j; a)] - [U(x_i; a) + U(x_j; b)]
      = (h_A(b) - h_A(a)) (U_uv,i - U_uv,j) + (h_B(b) - h_B(a)) (U_soft,i - U_soft,j)."""
    from oracle.reference import switching
    ha, hb = switching(lam_a)[:2], switching(lam_b)[:2]
    return (hb[0] - ha[0]) * (uuv_i - uuv_j) + (hb[1] - ha[1]) * (usoft_i - usoft_j)


def hrex_attempt(lams, uuv, usoft, T, seed, attempt):
    """One exchange attempt over a ladder (replicas listed in lambda order,
    lams[k] the lambda of the k-th): the pairs (k, k+1) with k of the
    attempt's parity are tried; pair k is accepted with probability
    min(1, exp(-beta Delta_k)), using the uniform (x + 0.5)/2^32 of the first
    Philox4x32-10 word at counter (k, attempt_lo, attempt_hi, 3).  Returns
    (accepted flags [n-1], new lambda of each replica)."""
    n = len(lams)
    beta = 1.0 / (KB * T)
    acc = [0] * max(n - 1, 0)
    new = list(lams)
    key = seed_key(seed)
    for k in range(attempt % 2, n - 1, 2):
        d = hrex_delta(lams[k], lams[k + 1], uuv[k], usoft[k], uuv[k + 1], usoft[k + 1])
        u = uniforms((k, attempt & _MASK, attempt >> 32, 3), key)[0]
        if d <= 0.0 or u < math.exp(-beta * d):
            acc[k] = 1
            new[k], new[k + 1] = lams[k + 1], lams[k]
    return acc, new
