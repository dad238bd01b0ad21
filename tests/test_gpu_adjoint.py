"""GPU parity of the parameter-gradient kernel (differentiation workload).

The flexible 22-atom solute in 4,000 waters (a seeded differentiation frame):
dU/dp, d2U/(dlambda dp) and the class derivatives of every solute atom's
charge, sigma and epsilon against the FP64 oracle on the same PME grid, against
central finite differences (h = 1e-4) of the library's own U and dU/dlambda,
and through the torch.autograd.Function.  The kernel is FP64 in both
precision modes; its inputs (float positions, fixed-point charge grid) are
exact or rounded far below the bar, so the oracle bar is 1e-8 of the
gradient's scale.
"""
import functools

import numpy as np
import pytest

from oracle import reference as R
from paper_2608_12691_b300 import lfe
from paper_2608_12691_b300 import systems as S

pytestmark = pytest.mark.gpu

FRAMES = (3, 17)


@functools.lru_cache(maxsize=None)
def frame(k):
    d = S.make_c4_frame(frame=k)
    G = R.param_grad(d, level=2)
    return d, G


_sys = {}


def gpu(k, precision):
    key = (k, precision)
    if key not in _sys:
        _sys[key] = lfe.System(frame(k)[0], precision=precision)
    return _sys[key]


def _scale(x):
    return np.maximum(1.0, np.abs(x))


@pytest.mark.parametrize("precision", [lfe.LFE_FP64, lfe.LFE_FP32_MIXED])
@pytest.mark.parametrize("k", FRAMES)
def test_param_grad_matches_oracle(k, precision):
    d, G = frame(k)
    sol = np.flatnonzero(d["solute"])
    lam = d["lam"]
    g = gpu(k, precision)
    dU, d2, basis = g.param_grad(lam)
    Go = G[sol]                                 # [n_u, 3, 3]
    err = np.abs(basis - Go) / _scale(Go)
    assert err.max() <= 1e-8, f"class derivatives: max rel err {err.max():.3e} at {np.unravel_index(err.argmax(), err.shape)}"
    dUo, d2o = R.assemble_param_grad(Go, lam)
    assert np.all(np.abs(dU - dUo) <= 1e-8 * _scale(dUo))
    assert np.all(np.abs(d2 - d2o) <= 1e-8 * _scale(d2o))


def test_param_grad_is_reproducible_and_keeps_lambda_state():
    g = gpu(FRAMES[0], lfe.LFE_FP32_MIXED)
    _, _, ext0 = g.get_state()
    a = g.param_grad(0.4)
    b = g.param_grad(0.4)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    _, _, ext1 = g.get_state()
    assert ext1["lambda"] == ext0["lambda"] and ext1["theta"] == ext0["theta"]


def test_param_grad_matches_fd_of_the_library():
    # central differences (h = 1e-4) of the library's own FP64 U and dU/dlambda
    d, _ = frame(FRAMES[1])
    g = lfe.System(d, precision=lfe.LFE_FP64)
    sol = np.flatnonzero(d["solute"])
    lam = 0.71
    dU, d2, _ = g.param_grad(lam)
    base = {k: d[k][sol].copy() for k in ("charge", "sigma", "epsilon")}
    h = 1e-4
    for b in (0, 4, 11, 20):
        for p, key in enumerate(("charge", "sigma", "epsilon")):
            vals = []
            for sgn in (+1, -1):
                v = dict(base)
                v[key] = base[key].copy()
                v[key][b] += sgn * h
                g.set_solute_params(v["charge"], v["sigma"], v["epsilon"])
                t, _ = g.eval(lam, forces=False)
                vals.append((t["U"], t["dUdl"]))
            fdU = (vals[0][0] - vals[1][0]) / (2 * h)
            fdd = (vals[0][1] - vals[1][1]) / (2 * h)
            # bar: truncation (h/p)^2 < 1e-5 relative for sigma and epsilon, plus
            # the rounding of U: ~1e5 fixed-point energy terms of 2^-36 kJ/mol
            # each give ~1e-8 kJ/mol, i.e. ~1e-4 absolute after dividing by 2h
            assert abs(dU[b, p] - fdU) <= 1e-5 * abs(fdU) + 1e-4, (b, key, dU[b, p], fdU)
            assert abs(d2[b, p] - fdd) <= 1e-5 * abs(fdd) + 1e-4, (b, key, d2[b, p], fdd)
    g.set_solute_params(base["charge"], base["sigma"], base["epsilon"])
    g.close()


@pytest.mark.parametrize("precision", [lfe.LFE_FP64, lfe.LFE_FP32_MIXED])
def test_set_solute_params_changes_the_evaluated_system(precision):
    # new solute parameters (charges still summing to 0): the library's
    # energies, forces and dU/dlambda must follow the oracle of the new system
    d0, _ = frame(FRAMES[0])
    rng = np.random.default_rng(5)
    sol = np.flatnonzero(d0["solute"])
    d = dict(d0)
    q = d0["charge"].copy()
    dq = S.f32(rng.uniform(-0.05, 0.05, size=sol.size))
    dq -= dq.mean()
    q[sol] = S.f32(q[sol] + dq)
    sig = d0["sigma"].copy()
    sig[sol] = S.f32(sig[sol] * 1.03)
    eps = d0["epsilon"].copy()
    eps[sol] = S.f32(eps[sol] * 0.9)
    d.update(charge=q, sigma=sig, epsilon=eps)
    g = lfe.System(d0, precision=precision)
    g.set_solute_params(q[sol], sig[sol], eps[sol])
    lam = 0.55
    t, F = g.eval(lam)
    o = R.evaluate(d, lam, level=2)
    tolF = 1e-5 if precision == lfe.LFE_FP32_MIXED else 1e-9
    tolE = 1e-6 if precision == lfe.LFE_FP32_MIXED else 1e-9
    E = o["E"]
    hA, hB, dA, dB = R.switching(lam)
    # U is a sum of large terms of both signs (self energies, exclusion
    # corrections, real and reciprocal parts): its error is measured against
    # the sum of their magnitudes
    parts = [f"{p}_{c}" for p in ("coul_real", "rec", "bg", "lj", "excl") for c in ("vv", "uu", "uv")]
    parts += ["self_vv", "self_uu", "p14_vv", "p14_uu", "U_soft"]
    scaleU = sum(abs(E[k]) for k in parts) + abs(o["U_bonded"])
    scale_dU = abs(dA * E["U_uv"]) + abs(dB * E["U_soft"])
    assert np.linalg.norm(F - o["F"]) / np.linalg.norm(o["F"]) <= tolF
    assert abs(t["U"] - o["U"]) <= tolE * scaleU
    assert abs(t["dUdl"] - o["dUdl"]) <= 1e-6 * scale_dU
    g.close()


def _qu_scale(q, sol):
    sv, su = np.sum(q[~sol] ** 2), np.sum(q[sol] ** 2)
    sc = np.sqrt(sv / su) if su > 0 and sv > 0 else 1.0
    return 2.0 ** np.round(np.log2(max(1.0, sc)))


@pytest.mark.parametrize("precision", [lfe.LFE_FP64, lfe.LFE_FP32_MIXED])
def test_set_solute_params_equals_creating_with_them(precision):
    # replacing the parameters of a live system is the same as creating the
    # system with them (identical evaluation), and the step graph captured
    # before the change is recaptured with the new constant energies
    d0 = S.make_c0(seed=31, lam=0.6)
    sol = d0["solute"].astype(bool)
    rng = np.random.default_rng(8)
    q = d0["charge"].copy()
    dq = S.f32(rng.uniform(-0.04, 0.04, size=sol.sum()))
    q[sol] = S.f32(q[sol] + dq - dq.mean())
    sig = d0["sigma"].copy()
    sig[sol] = S.f32(sig[sol] * 0.97)
    eps = d0["epsilon"].copy()
    eps[sol] = S.f32(eps[sol] * 1.1)
    assert _qu_scale(q, sol) == _qu_scale(d0["charge"], sol)
    d1 = dict(d0, charge=q, sigma=sig, epsilon=eps)
    a = lfe.System(d0, precision=precision)
    a.step(2)                       # a captured graph exists before the change
    a.set_positions(d0["pos"])
    a.build_neighbors()             # the same list as a fresh build at these positions
    a.set_velocities(np.zeros_like(d0["pos"]))
    a.set_solute_params(q[sol], sig[sol], eps[sol])
    b = lfe.System(d1, precision=precision)
    ta, Fa = a.eval(0.6)
    tb, Fb = b.eval(0.6)
    assert np.array_equal(Fa, Fb)
    for k in ("U", "dUdl", "U_vv", "U_uu", "U_uv", "U_soft"):
        assert ta[k] == tb[k], k
    a.step(3)
    _, _, ext = a.get_state()
    assert ext["step"] == 5 and np.isfinite(ext["U"])
    a.close()
    b.close()


def test_autograd_function_on_device():
    torch = pytest.importorskip("torch")
    from paper_2608_12691_b300.autograd import lambda_nonbonded

    d, G = frame(FRAMES[0])
    sol = np.flatnonzero(d["solute"])
    g = gpu(FRAMES[0], lfe.LFE_FP32_MIXED)
    dev = torch.device("cuda:0")
    q = torch.tensor(d["charge"][sol], dtype=torch.float64, device=dev, requires_grad=True)
    s = torch.tensor(d["sigma"][sol], dtype=torch.float64, device=dev, requires_grad=True)
    e = torch.tensor(d["epsilon"][sol], dtype=torch.float64, device=dev, requires_grad=True)
    lam = 0.37
    U, dUdl = lambda_nonbonded(g, lam, q, s, e)
    loss = 0.5 * U + 2.0 * dUdl
    loss.backward()
    dUo, d2o = R.assemble_param_grad(G[sol], lam)
    want = 0.5 * dUo + 2.0 * d2o
    got = torch.stack([q.grad, s.grad, e.grad], dim=1).cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-8 * _scale(want))
    t, _ = g.eval(lam, forces=False)
    assert U.item() == t["U"] and dUdl.item() == t["dUdl"]
