"""Thin ctypes binding of the C-ABI in include/lfe.h (argument marshalling only).

Every computation runs in the CUDA library ``liblfe.so`` built in-tree by
``paper_2608_12691_b300.build``.  There is no fallback: if the library is
missing or cannot be loaded, ``load()`` raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblfe.so")

LFE_OK = 0
LFE_ERR_ARG = -1
LFE_ERR_CUDA = -2
LFE_ERR_OVERFLOW = -3
LFE_ERR_NONFINITE = -4
LFE_ERR_TIMEOUT = -5
LFE_ERR_STATE = -6
LFE_FP32_MIXED = 0
LFE_FP64 = 1
LFE_EXT_LANGEVIN = 0
LFE_EXT_RNHL = 1
NTERMS = 10
NEXT = 13
TI_BINS = 100
TERM_NAMES = ["U", "dUdl", "U_vv", "U_uu", "U_uv", "U_soft", "U_bonded", "n_pairs", "hA", "hB"]

EXPORTED = [
    "lfe_create", "lfe_set_positions", "lfe_set_velocities", "lfe_set_integrator",
    "lfe_build_neighbors", "lfe_eval",
    "lfe_param_grad", "lfe_set_solute_params", "lfe_ti", "lfe_set_dafed", "lfe_dafed_state",
    "lfe_set_ext_thermostat", "lfe_ext_thermostat_state",
    "lfe_dafed_masses", "lfe_step", "lfe_get_state", "lfe_checkpoint", "lfe_restore",
    "lfe_time_stages", "lfe_autotune", "lfe_alu_peak", "lfe_set_theta", "lfe_set_list_capacity", "lfe_step_io", "lfe_step_io_f32", "lfe_set_list_prune", "lfe_mc_volume_move", "lfe_batch_create", "lfe_batch_eval", "lfe_batch_step", "lfe_batch_time_pairs", "lfe_batch_set_exchange",
    "lfe_batch_exchange_state",
    "lfe_batch_exchange", "lfe_batch_destroy", "lfe_batch_last_error", "lfe_last_error", "lfe_destroy", "lfe_pme_noalloc",
]
NOALLOC_MAX_GRID = 110592


def alu_peak():
    """Measured FP32 and FP64 FMA throughput of the current device, TFLOP/s
    (lfe_alu_peak)."""
    lib = load()
    f32 = ctypes.c_double()
    f64 = ctypes.c_double()
    rc = lib.lfe_alu_peak(ctypes.byref(f32), ctypes.byref(f64))
    if rc != 0:
        raise LfeError(rc, "lfe_alu_peak failed")
    return f32.value, f64.value


class LfeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lfe error {code}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("r_cut", ctypes.c_double),
        ("r_switch", ctypes.c_double),
        ("ewald_alpha", ctypes.c_double),
        ("pme_grid", ctypes.c_int * 3),
        ("pme_order", ctypes.c_int),
        ("skin", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("temperature", ctypes.c_double),
        ("friction", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("lambda_mass", ctypes.c_double),
        ("lambda_friction", ctypes.c_double),
        ("theta0", ctypes.c_double),
        ("opes_stride", ctypes.c_int),
        ("opes_dE_std", ctypes.c_double),
        ("opes_dE_exp", ctypes.c_double),
        ("opes_sigma", ctypes.c_double),
        ("opes_max_kernels", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("lambda_temperature", ctypes.c_double),
        ("sc_alpha", ctypes.c_double),
        ("sc_power", ctypes.c_double),
    ]


_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)


class Topology(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int),
        ("pos", _dp), ("charge", _dp), ("sigma", _dp), ("epsilon", _dp),
        ("solute", ctypes.POINTER(ctypes.c_ubyte)), ("mass", _dp),
        ("n_excl", ctypes.c_int), ("excl", _ip),
        ("n_14", ctypes.c_int), ("pairs14", _ip), ("scale14", _dp),
        ("n_waters", ctypes.c_int), ("water_OHH", _ip), ("water_rOH", ctypes.c_double),
        ("water_rHH", ctypes.c_double),
        ("n_constraints", ctypes.c_int), ("constraints", _ip), ("constraint_len", _dp),
        ("n_bonds", ctypes.c_int), ("bonds", _ip), ("bond_par", _dp),
        ("n_angles", ctypes.c_int), ("angles", _ip), ("angle_par", _dp),
        ("n_torsions", ctypes.c_int), ("torsions", _ip), ("torsion_par", _dp),
    ]


_lib = None


def load():
    """Load liblfe.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FileNotFoundError(f"{LIB_PATH} is missing: run paper_2608_12691_b300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    lib.lfe_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Topology), ctypes.POINTER(vp)]
    lib.lfe_set_positions.argtypes = [vp, vp, ctypes.c_int, vp]
    lib.lfe_set_velocities.argtypes = [vp, vp]
    lib.lfe_set_integrator.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.lfe_build_neighbors.argtypes = [vp, vp]
    lib.lfe_eval.argtypes = [vp, ctypes.c_double, vp, vp, ctypes.c_int, vp]
    lib.lfe_param_grad.argtypes = [vp, ctypes.c_double, vp, vp, vp, ctypes.c_int, vp]
    lib.lfe_set_solute_params.argtypes = [vp, vp, vp, vp, ctypes.c_int, vp]
    lib.lfe_step.argtypes = [vp, ctypes.c_int, vp]
    lib.lfe_ti.argtypes = [vp, vp, vp, vp, ctypes.c_int]
    lib.lfe_set_dafed.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_double, ctypes.c_double, vp]
    lib.lfe_dafed_state.argtypes = [vp, vp, vp, vp]
    lib.lfe_dafed_masses.argtypes = [vp, ctypes.c_int, vp, ctypes.c_double, vp]
    lib.lfe_set_ext_thermostat.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.lfe_ext_thermostat_state.argtypes = [vp, vp, vp]
    lib.lfe_get_state.argtypes = [vp, vp, vp, vp]
    lib.lfe_checkpoint.argtypes = [vp, ctypes.c_char_p]
    lib.lfe_restore.argtypes = [vp, ctypes.c_char_p]
    lib.lfe_set_theta.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    lib.lfe_set_theta.restype = ctypes.c_int
    lib.lfe_set_list_capacity.argtypes = [vp, ctypes.c_int]
    lib.lfe_set_list_capacity.restype = ctypes.c_int
    lib.lfe_step_io.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.lfe_step_io.restype = ctypes.c_int
    lib.lfe_step_io_f32.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.lfe_step_io_f32.restype = ctypes.c_int
    lib.lfe_set_list_prune.argtypes = [vp, ctypes.c_double]
    lib.lfe_set_list_prune.restype = ctypes.c_int
    lib.lfe_mc_volume_move.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_ulonglong, ctypes.c_ulonglong,
                                       vp, vp, vp]
    lib.lfe_mc_volume_move.restype = ctypes.c_int
    lib.lfe_batch_exchange.argtypes = [vp, ctypes.c_int, vp, ctypes.c_double, ctypes.c_ulonglong,
                                       ctypes.c_ulonglong, vp, vp]
    lib.lfe_batch_exchange.restype = ctypes.c_int
    lib.lfe_alu_peak.argtypes = [vp, vp]
    lib.lfe_alu_peak.restype = ctypes.c_int
    lib.lfe_autotune.argtypes = [vp, ctypes.c_int, ctypes.c_char_p, vp, vp]
    lib.lfe_autotune.restype = ctypes.c_int
    lib.lfe_time_stages.argtypes = [vp, ctypes.c_double, ctypes.c_int, vp,
                                    ctypes.POINTER(ctypes.c_char_p), _dp, ctypes.c_int]
    lib.lfe_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp)]
    lib.lfe_batch_eval.argtypes = [vp, vp, vp, vp]
    lib.lfe_batch_step.argtypes = [vp, ctypes.c_int, vp]
    lib.lfe_batch_time_pairs.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.lfe_batch_time_pairs.restype = ctypes.c_int
    lib.lfe_batch_set_exchange.argtypes = [vp, ctypes.c_int, vp, ctypes.c_double, ctypes.c_ulonglong, ctypes.c_int]
    lib.lfe_batch_set_exchange.restype = ctypes.c_int
    lib.lfe_batch_exchange_state.argtypes = [vp, vp, vp, vp]
    lib.lfe_batch_exchange_state.restype = ctypes.c_int
    lib.lfe_batch_destroy.argtypes = [vp]
    lib.lfe_batch_destroy.restype = None
    lib.lfe_batch_last_error.argtypes = [vp]
    lib.lfe_batch_last_error.restype = ctypes.c_char_p
    lib.lfe_last_error.argtypes = [vp]
    lib.lfe_last_error.restype = ctypes.c_char_p
    lib.lfe_destroy.argtypes = [vp]
    lib.lfe_destroy.restype = None
    lib.lfe_pme_noalloc.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                    ctypes.POINTER(ctypes.c_int), ctypes.c_double, vp, vp, vp]
    _lib = lib
    return lib


def _arr(a, dtype, width=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if width is not None:
        a = a.reshape(-1, width)
    return a


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def pme_noalloc(n, pos_ptr, charge_ptr, solute_ptr, box, alpha, grid, lam, forces_ptr, energies_ptr,
                stream=None):
    """Reciprocal-space class energies and forces without device allocation
    (all pointers are device memory; see lfe_pme_noalloc in include/lfe.h)."""
    lib = load()
    b = (ctypes.c_double * 3)(*[float(x) for x in box])
    g = (ctypes.c_int * 3)(*[int(x) for x in grid])
    rc = lib.lfe_pme_noalloc(int(n), pos_ptr, charge_ptr, solute_ptr, b, float(alpha), g, float(lam),
                             forces_ptr, energies_ptr, _stream_ptr(stream))
    if rc != LFE_OK:
        raise LfeError(rc, lib.lfe_last_error(None).decode())


class System:
    """A system on the current CUDA device, created from a dict of the shape
    produced by ``paper_2608_12691_b300.systems``."""

    def __init__(self, d, precision=LFE_FP32_MIXED, skin=0.1, seed=2608, theta0=None, **over):
        lib = load()
        self._lib = lib
        self.n = len(d["charge"])
        pr = Params()
        box = np.asarray(d["box"], dtype=np.float64)
        for k in range(3):
            pr.box[k] = box[k]
            pr.pme_grid[k] = int(d["grid"][k])
        pr.r_cut = float(d["r_cut"])
        pr.r_switch = float(d["r_switch"])
        pr.ewald_alpha = float(d["alpha"])
        pr.pme_order = int(d.get("order", 4))
        pr.skin = float(skin)
        pr.precision = int(precision)
        pr.temperature = float(d.get("temperature", 298.0))
        pr.friction = float(d.get("friction", 10.0))
        pr.dt = float(d.get("dt", 0.002))
        pr.lambda_mass = float(d.get("lambda_mass", 0.0))
        pr.lambda_friction = float(d.get("lambda_friction", 25.0))
        pr.theta0 = float(d.get("lam", 0.5) if theta0 is None else theta0)
        pr.opes_stride = int(d.get("opes_stride", 0))
        pr.opes_dE_std = float(d.get("opes_dE_std", 0.0))
        pr.opes_dE_exp = float(d.get("opes_dE_exp", 0.0))
        pr.opes_sigma = float(d.get("opes_sigma", 0.1))
        pr.opes_max_kernels = int(d.get("opes_max_kernels", 1024))
        pr.seed = int(seed)
        pr.lambda_temperature = float(d.get("lambda_temperature", 0.0))
        pr.sc_alpha = float(d.get("sc_alpha", 0.0) or 0.0)
        pr.sc_power = float(d.get("sc_power", 1.0) or 1.0)
        for k, v in over.items():
            setattr(pr, k, v)
        self.params = pr
        self._n_u = int(np.count_nonzero(np.asarray(d["solute"])))
        keep = {}

        def K(name, dtype, width=None):
            a = d.get(name)
            if a is None:
                a = np.zeros((0,) if width is None else (0, width))
            a = _arr(a, dtype, width)
            keep[name] = a
            return a

        t = Topology()
        t.n_atoms = self.n
        t.pos = _p(K("pos", np.float64, 3), ctypes.c_double)
        t.charge = _p(K("charge", np.float64), ctypes.c_double)
        t.sigma = _p(K("sigma", np.float64), ctypes.c_double)
        t.epsilon = _p(K("epsilon", np.float64), ctypes.c_double)
        t.solute = _p(K("solute", np.uint8), ctypes.c_ubyte)
        t.mass = _p(K("mass", np.float64), ctypes.c_double)
        ex = K("excl", np.int32, 2)
        t.n_excl, t.excl = ex.shape[0], _p(ex, ctypes.c_int)
        p14 = K("pairs14", np.int32, 2)
        t.n_14, t.pairs14 = p14.shape[0], _p(p14, ctypes.c_int)
        t.scale14 = _p(K("scale14", np.float64, 2), ctypes.c_double)
        w = K("waters", np.int32, 3)
        t.n_waters, t.water_OHH = w.shape[0], _p(w, ctypes.c_int)
        t.water_rOH = 0.09572
        t.water_rHH = 2 * 0.09572 * np.sin(np.radians(104.52) / 2)
        c = K("constraints", np.int32, 2)
        t.n_constraints, t.constraints = c.shape[0], _p(c, ctypes.c_int)
        t.constraint_len = _p(K("constraint_len", np.float64), ctypes.c_double)
        b = K("bonds", np.int32, 2)
        t.n_bonds, t.bonds = b.shape[0], _p(b, ctypes.c_int)
        t.bond_par = _p(K("bond_par", np.float64, 2), ctypes.c_double)
        a = K("angles", np.int32, 3)
        t.n_angles, t.angles = a.shape[0], _p(a, ctypes.c_int)
        t.angle_par = _p(K("angle_par", np.float64, 2), ctypes.c_double)
        to = K("torsions", np.int32, 4)
        t.n_torsions, t.torsions = to.shape[0], _p(to, ctypes.c_int)
        t.torsion_par = _p(K("torsion_par", np.float64, 3), ctypes.c_double)
        h = ctypes.c_void_p()
        rc = lib.lfe_create(ctypes.byref(pr), ctypes.byref(t), ctypes.byref(h))
        if rc != LFE_OK:
            raise LfeError(rc, lib.lfe_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != LFE_OK:
            raise LfeError(rc, self._lib.lfe_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self._lib.lfe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- calls
    def eval(self, lam, forces=True):
        """Host outputs: (terms dict, forces (N, 3) float64 or None)."""
        terms = np.zeros(NTERMS)
        F = np.zeros((self.n, 3)) if forces else None
        self._check(self._lib.lfe_eval(self.h, float(lam), F.ctypes.data if F is not None else None,
                                       terms.ctypes.data, 0, None))
        return dict(zip(TERM_NAMES, terms)), F

    def eval_device(self, lam, forces_ptr, terms_ptr, stream=None):
        """Device outputs: pointers to float64 device buffers ([3N] and [NTERMS])."""
        self._check(self._lib.lfe_eval(self.h, float(lam), forces_ptr, terms_ptr, 1, _stream_ptr(stream)))

    def set_positions(self, pos, stream=None):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        self._check(self._lib.lfe_set_positions(self.h, pos.ctypes.data, 0, _stream_ptr(stream)))

    def set_positions_ptr(self, ptr, on_device, stream=None):
        self._check(self._lib.lfe_set_positions(self.h, ptr, int(on_device), _stream_ptr(stream)))

    def set_velocities(self, vel):
        vel = np.ascontiguousarray(vel, dtype=np.float64)
        self._check(self._lib.lfe_set_velocities(self.h, vel.ctypes.data))

    def set_integrator(self, dt, friction, temperature):
        self._check(self._lib.lfe_set_integrator(self.h, float(dt), float(friction), float(temperature)))

    def build_neighbors(self, stream=None):
        self._check(self._lib.lfe_build_neighbors(self.h, _stream_ptr(stream)))

    def step(self, n, stream=None):
        self._check(self._lib.lfe_step(self.h, int(n), _stream_ptr(stream)))

    def get_state(self):
        pos = np.zeros((self.n, 3))
        vel = np.zeros((self.n, 3))
        ext = np.zeros(NEXT)
        self._check(self._lib.lfe_get_state(self.h, pos.ctypes.data, vel.ctypes.data, ext.ctypes.data))
        keys = ["theta", "p_theta", "lambda", "dUdl", "U", "n_kernels_std", "n_kernels_exp", "step",
                "n_rebuilds", "n_tiles", "n_pairs_step", "n_tiles_pruned", "n_prunes"]
        return pos, vel, dict(zip(keys, ext))

    def mc_volume_move(self, pressure_bar, dv_max, seed, attempt):
        """One Monte Carlo volume move (lfe_mc_volume_move).  Returns
        (accepted, box [3], (U before, U proposed))."""
        acc = ctypes.c_int()
        box = np.zeros(3)
        en = np.zeros(2)
        self._check(self._lib.lfe_mc_volume_move(self.h, float(pressure_bar), float(dv_max), int(seed), int(attempt),
                                                 ctypes.byref(acc), box.ctypes.data, en.ctypes.data))
        return bool(acc.value), box, (float(en[0]), float(en[1]))

    def step_io(self, pos_in_ptr, pos_out_ptr, vel_out_ptr, ext_out_ptr, stream=None):
        """One step with host input/output in one captured graph (lfe_step_io);
        the pointers are page-locked host buffers (0/None for NULL)."""
        self._check(self._lib.lfe_step_io(self.h, pos_in_ptr or None, pos_out_ptr or None, vel_out_ptr or None,
                                          ext_out_ptr or None, _stream_ptr(stream)))

    def set_list_prune(self, inner_buffer):
        """Dynamic pruning of the neighbour list between rebuilds
        (lfe_set_list_prune); inner buffer in nm, 0 switches it off."""
        self._check(self._lib.lfe_set_list_prune(self.h, float(inner_buffer)))

    def step_io_f32(self, pos_in_ptr, pos_out_ptr, vel_out_ptr, ext_out_ptr, stream=None):
        """lfe_step_io with float positions and velocities (lfe_step_io_f32);
        the pointers are page-locked host buffers (0/None for NULL)."""
        self._check(self._lib.lfe_step_io_f32(self.h, pos_in_ptr or None, pos_out_ptr or None, vel_out_ptr or None,
                                              ext_out_ptr or None, _stream_ptr(stream)))

    def get_state_into(self, pos_ptr, vel_ptr, ext_ptr):
        self._check(self._lib.lfe_get_state(self.h, pos_ptr, vel_ptr, ext_ptr))

    def checkpoint(self, path):
        self._check(self._lib.lfe_checkpoint(self.h, str(path).encode()))

    def restore(self, path):
        self._check(self._lib.lfe_restore(self.h, str(path).encode()))

    @property
    def n_solute(self):
        return self._n_u

    def param_grad(self, lam):
        """Host outputs (dU/dp [n_u, 3], d2U/dlambda dp [n_u, 3], class
        derivatives [n_u, 3 (q, sigma, eps), 3 (uu, uv, soft)]), float64."""
        n_u = self._n_u
        dU = np.zeros((n_u, 3))
        d2 = np.zeros((n_u, 3))
        basis = np.zeros((n_u, 3, 3))
        self._check(self._lib.lfe_param_grad(self.h, float(lam), dU.ctypes.data, d2.ctypes.data,
                                             basis.ctypes.data, 0, None))
        return dU, d2, basis

    def param_grad_device(self, lam, dU_ptr, d2_ptr, basis_ptr=None, stream=None):
        """Device outputs: float64 device buffers [3 n_u], [3 n_u], [9 n_u] (any may be None)."""
        self._check(self._lib.lfe_param_grad(self.h, float(lam), dU_ptr, d2_ptr, basis_ptr, 1,
                                             _stream_ptr(stream)))

    def set_solute_params(self, charge=None, sigma=None, epsilon=None):
        """New solute charges / sigma / epsilon ([n_u] float64 host arrays; None = unchanged)."""
        keep = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
                for a in (charge, sigma, epsilon)]
        for a in keep:
            if a is not None and a.shape[0] != self._n_u:
                raise ValueError(f"expected {self._n_u} solute values, got {a.shape[0]}")
        ptrs = [None if a is None else a.ctypes.data for a in keep]
        self._check(self._lib.lfe_set_solute_params(self.h, *ptrs, 0, None))

    def set_solute_params_device(self, charge_ptr=None, sigma_ptr=None, epsilon_ptr=None, stream=None):
        """Same, from float64 device buffers of n_u entries (None = unchanged)."""
        self._check(self._lib.lfe_set_solute_params(self.h, charge_ptr, sigma_ptr, epsilon_ptr, 1,
                                                    _stream_ptr(stream)))

    def ti(self, reset=False):
        """Eq. 2 estimator: (bin means [TI_BINS] with NaN for empty bins,
        sample counts [TI_BINS], Delta G)."""
        mean = np.zeros(TI_BINS)
        count = np.zeros(TI_BINS)
        dg = np.zeros(1)
        self._check(self._lib.lfe_ti(self.h, mean.ctypes.data, count.ctypes.data, dg.ctypes.data, int(reset)))
        return mean, count, float(dg[0])

    def set_dafed(self, atoms, kappa, mass, temperature=1000.0, friction=25.0, s0=None):
        """Couple torsions (rows of 4 atom indices) to auxiliary angles (Eq. 15)."""
        atoms = np.ascontiguousarray(atoms, dtype=np.int32).reshape(-1, 4)
        k = atoms.shape[0]
        kappa = np.ascontiguousarray(np.broadcast_to(kappa, (k,)), dtype=np.float64)
        mass = np.ascontiguousarray(np.broadcast_to(mass, (k,)), dtype=np.float64)
        s0a = None if s0 is None else np.ascontiguousarray(s0, dtype=np.float64).reshape(k)
        self._dafed_n = k
        self._check(self._lib.lfe_set_dafed(self.h, k, atoms.ctypes.data, kappa.ctypes.data, mass.ctypes.data,
                                            float(temperature), float(friction),
                                            None if s0a is None else s0a.ctypes.data))

    def set_ext_thermostat(self, kind, tau=0.04, n_reg=1.0):
        """Thermostat of theta and the d-AFED auxiliary angles
        (lfe_set_ext_thermostat): LFE_EXT_LANGEVIN or LFE_EXT_RNHL."""
        self._check(self._lib.lfe_set_ext_thermostat(self.h, int(kind), float(tau), float(n_reg)))

    def ext_thermostat_state(self):
        """(v_eta of theta, v_eta of the auxiliary angles [n_cv])."""
        vt = ctypes.c_double()
        va = np.zeros(max(getattr(self, "_dafed_n", 0), 1))
        self._check(self._lib.lfe_ext_thermostat_state(self.h, ctypes.byref(vt), va.ctypes.data))
        return vt.value, va[:getattr(self, "_dafed_n", 0)]

    def dafed_state(self):
        """(s, p_s, xi at the current positions), each [n_cv]."""
        k = getattr(self, "_dafed_n", 0)
        s = np.zeros(k)
        p = np.zeros(k)
        xi = np.zeros(k)
        if k:
            self._check(self._lib.lfe_dafed_state(self.h, s.ctypes.data, p.ctypes.data, xi.ctypes.data))
        return s, p, xi

    def dafed_masses(self, atoms, c=300.0):
        """Eq. 16 auxiliary masses at the current positions."""
        atoms = np.ascontiguousarray(atoms, dtype=np.int32).reshape(-1, 4)
        out = np.zeros(atoms.shape[0])
        self._check(self._lib.lfe_dafed_masses(self.h, atoms.shape[0], atoms.ctypes.data, float(c),
                                               out.ctypes.data))
        return out

    def set_theta(self, theta, p_theta=0.0):
        """Set theta and its momentum (lambda follows Eq. 3; lfe_set_theta)."""
        self._check(self._lib.lfe_set_theta(self.h, float(theta), float(p_theta)))

    def set_list_capacity(self, tiles):
        """Shrink or grow the neighbour-list tile capacity; the list is
        rebuilt by the next step or evaluation (lfe_set_list_capacity)."""
        self._check(self._lib.lfe_set_list_capacity(self.h, int(tiles)))

    def autotune(self, reps=20, cache_path=None):
        """Choose the evaluation's launch shapes (and, for skin <= 0, the list
        buffer) by timing (lfe_autotune).  Returns (objective ms,
        {pair_blocks_per_sm, uv_blocks, df64_lines, from_cache, skin_pm})."""
        best = ctypes.c_double()
        params = (ctypes.c_int * 5)()
        path = None if cache_path is None else str(cache_path).encode()
        self._check(self._lib.lfe_autotune(self.h, int(reps), path, ctypes.byref(best), params))
        return best.value, dict(zip(["pair_blocks_per_sm", "uv_blocks", "df64_lines", "from_cache", "skin_pm"],
                                    list(params)))

    def time_stages(self, lam, reps=10, stream=None, max_n=32):
        names = (ctypes.c_char_p * max_n)()
        ms = np.zeros(max_n)
        r = self._lib.lfe_time_stages(self.h, float(lam), int(reps), _stream_ptr(stream), names,
                                      ms.ctypes.data_as(_dp), max_n)
        if r < 0:
            self._check(r)
        return {names[k].decode(): float(ms[k]) for k in range(r)}


class Batch:
    """Replicas advanced together by one graph launch per step (lfe_batch_*)."""

    def __init__(self, systems):
        lib = load()
        self._lib = lib
        self.systems = list(systems)
        arr = (ctypes.c_void_p * len(self.systems))(*[s.h.value for s in self.systems])
        h = ctypes.c_void_p()
        rc = lib.lfe_batch_create(arr, len(self.systems), ctypes.byref(h))
        if rc != LFE_OK:
            raise LfeError(rc, lib.lfe_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != LFE_OK:
            raise LfeError(rc, self._lib.lfe_batch_last_error(self.h).decode())

    def step(self, n, stream=None):
        self._check(self._lib.lfe_batch_step(self.h, int(n), _stream_ptr(stream)))

    def set_exchange(self, ladder, temperature, seed, stride):
        """Device-side lambda exchange every `stride` batch steps
        (lfe_batch_set_exchange; stride <= 0 switches it off)."""
        lad = np.ascontiguousarray(ladder, dtype=np.int32)
        self._check(self._lib.lfe_batch_set_exchange(self.h, len(lad), lad.ctypes.data, float(temperature), int(seed),
                                                     int(stride)))

    def exchange_state(self):
        """(ladder, attempts, accepted per ladder position) of the device-side
        exchange (lfe_batch_exchange_state)."""
        n = len(self.systems)
        lad = np.zeros(n, dtype=np.int32)
        att = ctypes.c_ulonglong()
        acc = np.zeros(max(n - 1, 1), dtype=np.uint64)
        self._check(self._lib.lfe_batch_exchange_state(self.h, lad.ctypes.data, ctypes.byref(att), acc.ctypes.data))
        return lad, int(att.value), acc

    def time_pairs(self, reps=20, stream=None):
        """Mean device time (ms) of the FP32 replicas' shared pair-kernel launch
        (lfe_batch_time_pairs); call between steps."""
        ms = ctypes.c_double()
        self._check(self._lib.lfe_batch_time_pairs(self.h, int(reps), ctypes.byref(ms), _stream_ptr(stream)))
        return ms.value

    def exchange(self, ladder, temperature, seed, attempt, stream=None):
        """One lambda-exchange attempt over `ladder` (replica indices in lambda
        order; lfe_batch_exchange).  Returns (new ladder, accepted flags)."""
        lad = np.ascontiguousarray(ladder, dtype=np.int32).copy()
        acc = np.zeros(max(len(lad) - 1, 0), dtype=np.int32)
        self._check(self._lib.lfe_batch_exchange(self.h, len(lad), lad.ctypes.data, float(temperature), int(seed),
                                                 int(attempt), acc.ctypes.data, _stream_ptr(stream)))
        return lad, acc

    def eval(self, lambdas):
        lam = np.ascontiguousarray(lambdas, dtype=np.float64)
        terms = np.zeros((len(self.systems), NTERMS))
        self._check(self._lib.lfe_batch_eval(self.h, lam.ctypes.data, terms.ctypes.data, None))
        return [dict(zip(TERM_NAMES, t)) for t in terms]

    def close(self):
        if getattr(self, "h", None):
            self._lib.lfe_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
