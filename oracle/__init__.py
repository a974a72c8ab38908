"""ctypes front end of the plain FP64 CPU oracle (oracle/sl_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by the CPU-baseline leg of bench.py.  The library path never imports it.

Every function follows the paper's definitions (arXiv 1801.10233): see the
header of sl_oracle.c for the equation each part implements.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB, build

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int_p = ctypes.POINTER(ctypes.c_int)

ORC_OK, ORC_ERR_ARG, ORC_ERR_BOX, ORC_ERR_SPIN_NORM, ORC_ERR_SKIN, ORC_ERR_OOM = 0, -1, -3, -4, -5, -8

# Learned model layout (sl_learned.c): float params W1[64][48], b1[64],
# W2[64][64], b2[64], w3[64], b3; float norm mean[48], inv_std[48], lo[48], hi[48].
ML_NF, ML_NH, ML_RC = 48, 64, 6.0
ML_OFF_W1 = 0
ML_OFF_B1 = ML_OFF_W1 + ML_NH * ML_NF
ML_OFF_W2 = ML_OFF_B1 + ML_NH
ML_OFF_B2 = ML_OFF_W2 + ML_NH * ML_NH
ML_OFF_W3 = ML_OFF_B2 + ML_NH
ML_OFF_B3 = ML_OFF_W3 + ML_NH
ML_NPARAM = ML_OFF_B3 + 1
ML_NNORM = 4 * ML_NF
HBAR = 6.582119569e-4


class _Params(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int32), ("rotation", ctypes.c_int32), ("fix_lattice", ctypes.c_int32),
        ("rebuild_every", ctypes.c_int32), ("morse_shift", ctypes.c_int32), ("brute_force", ctypes.c_int32),
        ("box", ctypes.c_double * 3), ("mass", ctypes.c_double), ("mu_s", ctypes.c_double),
        ("H", ctypes.c_double * 3), ("dt", ctypes.c_double),
        ("ex_alpha", ctypes.c_double), ("ex_gamma", ctypes.c_double), ("ex_delta", ctypes.c_double),
        ("ex_rc", ctypes.c_double),
        ("m_D0", ctypes.c_double), ("m_alpha", ctypes.c_double), ("m_r0", ctypes.c_double),
        ("m_rc", ctypes.c_double), ("skin", ctypes.c_double),
        ("lam", ctypes.c_double), ("temperature", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("replica", ctypes.c_int32), ("hamiltonian", ctypes.c_int32),
        ("lat_gamma", ctypes.c_double), ("lat_temperature", ctypes.c_double),
        ("an_K", ctypes.c_double), ("an_axis", ctypes.c_double * 3),
        ("neel_alpha", ctypes.c_double), ("neel_gamma", ctypes.c_double), ("neel_delta", ctypes.c_double),
        ("dmi_alpha", ctypes.c_double), ("dmi_gamma", ctypes.c_double), ("dmi_delta", ctypes.c_double),
        ("eam_A", ctypes.c_double), ("eam_d", ctypes.c_double), ("eam_beta", ctypes.c_double),
        ("ground_sub", ctypes.c_int32), ("eam_tab", ctypes.c_int32),
    ]


_lib = None
# observation point inside a step: (user, event, arg); event 0 after a colour's
# pass (arg = colour), 1 after the drift
HOOK = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(_Params), _c_double_p, _c_double_p, _c_double_p, _c_int_p]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_step.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.orc_get_state.argtypes = [ctypes.c_void_p, _c_double_p, _c_double_p, _c_double_p]
        L.orc_get_forces.argtypes = [ctypes.c_void_p, _c_double_p]
        L.orc_get_omega.argtypes = [ctypes.c_void_p, _c_double_p]
        L.orc_get_order.argtypes = [ctypes.c_void_p, _c_int_p, _c_int_p, _c_int_p, _c_int_p, _c_int_p]
        L.orc_get_step.restype = ctypes.c_long
        L.orc_get_step.argtypes = [ctypes.c_void_p]
        L.orc_get_rebuilds.restype = ctypes.c_int
        L.orc_get_rebuilds.argtypes = [ctypes.c_void_p]
        L.orc_get_error.restype = ctypes.c_int
        L.orc_get_error.argtypes = [ctypes.c_void_p]
        L.orc_create_threads.restype = ctypes.c_void_p
        L.orc_create_threads.argtypes = [ctypes.POINTER(_Params), _c_double_p, _c_double_p, _c_double_p, ctypes.c_int,
                                         _c_int_p]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_count_pairs.restype = ctypes.c_int
        L.orc_count_pairs.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_energy.argtypes = [ctypes.c_void_p, _c_double_p]
        L.orc_magnetization.argtypes = [ctypes.c_void_p, _c_double_p]
        L.orc_potential_energy.restype = ctypes.c_int
        L.orc_potential_energy.argtypes = [ctypes.POINTER(_Params), _c_double_p, _c_double_p, _c_double_p]
        L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32 * 4), ctypes.POINTER(ctypes.c_uint32 * 2),
                                        ctypes.POINTER(ctypes.c_uint32 * 4)]
        L.orc_gauss3.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                 _c_double_p]
        _f_p = ctypes.POINTER(ctypes.c_float)
        L.orc_ml_set_model.restype = ctypes.c_int
        L.orc_ml_set_model.argtypes = [ctypes.c_void_p, _f_p, _f_p]
        L.orc_ml_gate.argtypes = [ctypes.c_void_p, _c_int_p]
        L.orc_ml_eval.restype = ctypes.c_int
        L.orc_ml_eval.argtypes = [ctypes.c_int, _c_double_p, _c_double_p, _c_double_p, _f_p, _f_p,
                                  _c_double_p, _c_double_p, _c_double_p, _c_double_p, _c_double_p]
        L.orc_ml_vjp.restype = ctypes.c_int
        L.orc_ml_vjp.argtypes = [ctypes.c_int, _c_double_p, _c_double_p, _c_double_p, _f_p, _f_p,
                                 ctypes.c_double, _c_double_p, _c_double_p, _c_double_p]
        L.orc_ml_loss.restype = ctypes.c_int
        L.orc_ml_loss.argtypes = [ctypes.c_int, _c_int_p, _c_double_p, _c_double_p, _c_double_p, _c_double_p,
                                  _c_double_p, _c_double_p, _c_double_p, ctypes.c_double, _f_p, _f_p,
                                  _c_double_p, _c_double_p]
        L.orc_ml_adam.argtypes = [ctypes.c_int, _f_p, _c_double_p, _c_double_p, _c_double_p, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_ml_eval_sample.restype = ctypes.c_int
        L.orc_ml_eval_sample.argtypes = [ctypes.c_int, _c_double_p, _c_double_p, _c_double_p, _f_p, _f_p,
                                         ctypes.c_int, _c_int_p, _c_double_p, _c_double_p, _c_double_p,
                                         _c_double_p]
        L.orc_set_eam_tables.restype = ctypes.c_int
        L.orc_set_eam_tables.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, _c_double_p, ctypes.c_int,
                                         ctypes.c_double, _c_double_p, _c_double_p]
        L.orc_potential_energy_state.restype = ctypes.c_int
        L.orc_potential_energy_state.argtypes = [ctypes.c_void_p, _c_double_p, _c_double_p, _c_double_p]
        L.orc_spline_eval.restype = ctypes.c_int
        L.orc_spline_eval.argtypes = [ctypes.c_int, ctypes.c_double, _c_double_p, ctypes.c_int, _c_double_p,
                                      _c_double_p, _c_double_p]
        L.orc_set_hook.argtypes = [ctypes.c_void_p, HOOK, ctypes.c_void_p]
        L.orc_set_atoms.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_int_p, _c_double_p, _c_double_p]
        L.orc_bf16_value.restype = ctypes.c_double
        L.orc_bf16_value.argtypes = [ctypes.c_float]
        L.orc_params_size.restype = ctypes.c_int
        if L.orc_params_size() != ctypes.sizeof(_Params):
            raise RuntimeError("oracle parameter struct layout mismatch")
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_c_double_p)


def _ip(a):
    return a.ctypes.data_as(_c_int_p)


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _f32(a, n):
    a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
    if a.size != n:
        raise ValueError(f"expected {n} floats, got {a.size}")
    return a


def _opt(a):
    return None if a is None else _dp(a)


def make_params(p: dict, brute_force=False, lam=0.0, temperature=0.0, seed=0, replica=0) -> _Params:
    q = _Params()
    q.n_atoms = int(p["n_atoms"])
    q.rotation = int(p.get("rotation", 0))
    q.fix_lattice = int(p.get("fix_lattice", 0))
    q.rebuild_every = int(p.get("rebuild_every", 0))
    q.morse_shift = int(p.get("morse_shift_energy", 1))
    q.brute_force = int(bool(brute_force))
    for a in range(3):
        q.box[a] = float(p["box"][a])
        q.H[a] = float(p["H_tesla"][a])
    q.mass = float(p["mass_amu"])
    q.mu_s = float(p["mu_s_muB"])
    q.dt = float(p["dt_ps"])
    q.ex_alpha, q.ex_gamma = float(p["ex_alpha_eV"]), float(p["ex_gamma"])
    q.ex_delta, q.ex_rc = float(p["ex_delta_A"]), float(p["ex_rc_A"])
    q.m_D0, q.m_alpha = float(p["morse_D0_eV"]), float(p["morse_alpha_invA"])
    q.m_r0, q.m_rc = float(p["morse_r0_A"]), float(p["morse_rc_A"])
    q.skin = float(p["skin_A"])
    q.lam = float(lam)
    q.temperature = float(temperature)
    q.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    q.replica = int(replica)
    q.hamiltonian = int(p.get("hamiltonian", 0))
    q.lat_gamma = float(p.get("lattice_gamma_ps", 0.0))
    q.lat_temperature = float(p.get("lattice_temperature_K", 0.0))
    q.an_K = float(p.get("aniso_K_eV", 0.0))
    for a, x in enumerate(p.get("aniso_axis", (0.0, 0.0, 1.0))):
        q.an_axis[a] = float(x)
    q.neel_alpha, q.neel_gamma = float(p.get("neel_alpha_eV", 0.0)), float(p.get("neel_gamma", 0.0))
    q.neel_delta = float(p.get("neel_delta_A", 1.0))
    q.dmi_alpha, q.dmi_gamma = float(p.get("dmi_alpha_eV", 0.0)), float(p.get("dmi_gamma", 0.0))
    q.dmi_delta = float(p.get("dmi_delta_A", 1.0))
    q.eam_A, q.eam_d = float(p.get("eam_A_eV", 0.0)), float(p.get("eam_d_A", 1.0))
    q.eam_beta = float(p.get("eam_beta", 0.0))
    q.ground_sub = int(p.get("subtract_ground_exchange", 0))
    q.eam_tab = int(p.get("eam_tabulated", 0))
    return q


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle error {code}")
        self.code = code


class Oracle:
    """Plain FP64 reference of one coupled spin-lattice system."""

    def __init__(self, params: dict, r, v, s, brute_force=False, lam=0.0, temperature=0.0, seed=0, replica=0,
                 threads=1):
        self._L = lib()
        self.params = dict(params)
        self.n = int(params["n_atoms"])
        self._p = make_params(params, brute_force, lam, temperature, seed, replica)
        r = np.ascontiguousarray(r, dtype=np.float64).reshape(self.n, 3)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(self.n, 3)
        s = np.ascontiguousarray(s, dtype=np.float64).reshape(self.n, 3)
        err = ctypes.c_int(0)
        h = self._L.orc_create_threads(ctypes.byref(self._p), _dp(r), _dp(v), _dp(s), int(threads), ctypes.byref(err))
        if not h:
            raise OracleError(err.value)
        self._h = ctypes.c_void_p(h)
        self.threads = self.set_threads(threads)

    def set_threads(self, threads):
        """Threads for later steps (1 = serial); returns the number used.
        Any number gives results bit-identical to one thread."""
        self.threads = int(self._L.orc_set_threads(self._h, int(threads)))
        return self.threads

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and self._L is not None:
            self._L.orc_destroy(h)
            self._h = None

    def step(self, n=1):
        return int(self._L.orc_step(self._h, int(n)))

    def set_dt(self, dt):
        self._L.orc_set_dt(self._h, float(dt))

    def state(self):
        r = np.empty((self.n, 3)); v = np.empty((self.n, 3)); s = np.empty((self.n, 3))
        self._L.orc_get_state(self._h, _dp(r), _dp(v), _dp(s))
        return r, v, s

    def forces(self):
        F = np.empty((self.n, 3))
        self._L.orc_get_forces(self._h, _dp(F))
        return F

    def omega(self):
        w = np.empty((self.n, 3))
        self._L.orc_get_omega(self._h, _dp(w))
        return w

    def order(self):
        order = np.empty(self.n, dtype=np.int32)
        cs = np.empty(9, dtype=np.int32)
        sec = np.empty(self.n, dtype=np.int32)
        col = np.empty(self.n, dtype=np.int32)
        ns = np.empty(3, dtype=np.int32)
        self._L.orc_get_order(self._h, _ip(order), _ip(cs), _ip(sec), _ip(col), _ip(ns))
        return dict(order=order, colour_start=cs, sector=sec, colour=col, nsec=ns)

    @property
    def steps_done(self):
        return int(self._L.orc_get_step(self._h))

    @property
    def rebuilds(self):
        return int(self._L.orc_get_rebuilds(self._h))

    @property
    def error(self):
        return int(self._L.orc_get_error(self._h))

    def pair_count(self, which="exchange"):
        return int(self._L.orc_count_pairs(self._h, 0 if which == "exchange" else 1))

    def energy(self):
        out = np.empty(8)
        self._L.orc_energy(self._h, _dp(out))
        return out

    def magnetization(self):
        out = np.empty(4)
        self._L.orc_magnetization(self._h, _dp(out))
        return out

    def set_model(self, params, norm):
        """Install the learned model (hamiltonian = 1 only) and recompute forces."""
        self._ml = (_f32(params, ML_NPARAM), _f32(norm, ML_NNORM))
        e = int(self._L.orc_ml_set_model(self._h, _fp(self._ml[0]), _fp(self._ml[1])))
        if e:
            raise OracleError(e)

    def set_eam_tables(self, F, drho, rho, phi, dr):
        """Tables of the tabulated embedded-atom potential (params
        eam_tabulated = 1): F on rho = k drho, rho(r) and phi(r) on r = k dr."""
        F = np.ascontiguousarray(F, dtype=np.float64)
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        if rho.shape != phi.shape:
            raise ValueError("rho and phi tables differ in length")
        e = self._L.orc_set_eam_tables(self._h, len(F), float(drho), _dp(F), len(rho), float(dr), _dp(rho), _dp(phi))
        if e:
            raise OracleError(e)

    def potential_energy(self, r, s):
        """(E_mech, E_exch, E_zeeman, sum, E_spin_orbit) of arbitrary positions
        and spins with this system's parameters and tables (brute-force pairs)."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.float64)
        out = np.empty(5)
        e = self._L.orc_potential_energy_state(self._h, _dp(r), _dp(s), _dp(out))
        if e:
            raise OracleError(e)
        return out

    def set_hook(self, fn):
        """Call fn(event, arg) at the step's observation points (None: off)."""
        self._hook = None if fn is None else HOOK(lambda user, ev, arg: fn(int(ev), int(arg)))
        self._L.orc_set_hook(self._h, self._hook if self._hook is not None else HOOK(), None)

    def set_atoms(self, ids, r=None, s=None):
        """Overwrite the positions and/or spins of the atoms `ids`."""
        ids = np.ascontiguousarray(ids, dtype=np.int32)
        r = None if r is None else np.ascontiguousarray(r, dtype=np.float64).reshape(len(ids), 3)
        s = None if s is None else np.ascontiguousarray(s, dtype=np.float64).reshape(len(ids), 3)
        self._L.orc_set_atoms(self._h, len(ids), _ip(ids), _opt(r), _opt(s))

    def gate(self):
        """(out-of-range atoms at the last learned evaluation point, points handed to the analytic H)."""
        out = np.zeros(2, dtype=np.int32)
        self._L.orc_ml_gate(self._h, _ip(out))
        return int(out[0]), int(out[1])


def potential_energy(params: dict, r, s):
    """(E_morse, E_exch, E_zeeman, sum, E_spin_orbit) of arbitrary positions
    and spin vectors (spins need not be unit length), brute-force pairs; the
    sum includes the spin-orbit part."""
    L = lib()
    p = make_params(params)
    r = np.ascontiguousarray(r, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.empty(5)
    L.orc_potential_energy(ctypes.byref(p), _dp(r), _dp(s), _dp(out))
    return out


def spline_eval(y, h, x):
    """Natural cubic spline through (k h, y_k), evaluated at the points x:
    (values, derivatives)."""
    L = lib()
    y = np.ascontiguousarray(y, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    v = np.empty_like(x)
    dv = np.empty_like(x)
    e = L.orc_spline_eval(len(y), float(h), _dp(y), len(x), _dp(x), _dp(v), _dp(dv))
    if e:
        raise OracleError(e)
    return v, dv


def philox4x32_10(ctr, key):
    L = lib()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    L.orc_philox4x32_10(ctypes.byref(c), ctypes.byref(k), ctypes.byref(o))
    return [int(x) for x in o]


def gauss3(seed, replica, step, subpass, atom):
    L = lib()
    g = np.empty(3)
    L.orc_gauss3(int(seed) & 0xFFFFFFFFFFFFFFFF, int(replica), int(step), int(subpass), int(atom), _dp(g))
    return g


# ---------------------------------------------------------------------------
# Learned model (sl_learned.c)
# ---------------------------------------------------------------------------
def bf16_value(x: float) -> float:
    """x rounded to bfloat16 (nearest, ties to even), as the model uses its weights."""
    return float(lib().orc_bf16_value(float(x)))


def ml_eval(r, s, box, params, norm):
    """Learned energy and gradients of one periodic frame (brute-force pairs).
    Returns dict(e_atom, D, G, F, B, out_of_range)."""
    L = lib()
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    s = np.ascontiguousarray(s, dtype=np.float64).reshape(-1, 3)
    n = r.shape[0]
    box = np.ascontiguousarray(box, dtype=np.float64).reshape(3)
    pa, no = _f32(params, ML_NPARAM), _f32(norm, ML_NNORM)
    e = np.empty(n); D = np.empty((n, ML_NF)); G = np.empty((n, ML_NF))
    F = np.empty((n, 3)); B = np.empty((n, 3))
    bad = L.orc_ml_eval(n, _dp(r), _dp(s), _dp(box), _fp(pa), _fp(no), _dp(e), _dp(D), _dp(G), _dp(F), _dp(B))
    if bad < 0:
        raise OracleError(bad)
    return dict(e_atom=e, D=D, G=G, F=F, B=B, out_of_range=int(bad))


def ml_vjp(r, s, box, params, norm, gE=0.0, gF=None, gB=None):
    """d/dparams of gE E + sum gF.F + sum gB.B (F = -dE/dr, B = -dE/ds)."""
    L = lib()
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    s = np.ascontiguousarray(s, dtype=np.float64).reshape(-1, 3)
    n = r.shape[0]
    box = np.ascontiguousarray(box, dtype=np.float64).reshape(3)
    pa, no = _f32(params, ML_NPARAM), _f32(norm, ML_NNORM)
    gF = None if gF is None else np.ascontiguousarray(gF, dtype=np.float64).reshape(n, 3)
    gB = None if gB is None else np.ascontiguousarray(gB, dtype=np.float64).reshape(n, 3)
    grad = np.empty(ML_NPARAM)
    e = L.orc_ml_vjp(n, _dp(r), _dp(s), _dp(box), _fp(pa), _fp(no), float(gE), _opt(gF), _opt(gB), _dp(grad))
    if e:
        raise OracleError(e)
    return grad


def ml_loss(frames, E_ref, F_ref, B_ref, w, params, norm, want_grad=True):
    """Training loss over frames [(r, s, box), ...] and its parameter gradient.
    Returns (out[4] = L, L_E, L_F, L_omega; grad or None)."""
    L = lib()
    n_of = np.array([np.asarray(f[0]).reshape(-1, 3).shape[0] for f in frames], dtype=np.int32)
    r = np.ascontiguousarray(np.concatenate([np.asarray(f[0], dtype=np.float64).reshape(-1, 3) for f in frames]))
    s = np.ascontiguousarray(np.concatenate([np.asarray(f[1], dtype=np.float64).reshape(-1, 3) for f in frames]))
    boxes = np.ascontiguousarray(np.array([f[2] for f in frames], dtype=np.float64).reshape(-1))
    E_ref = np.ascontiguousarray(E_ref, dtype=np.float64)
    F_ref = np.ascontiguousarray(F_ref, dtype=np.float64).reshape(-1, 3)
    B_ref = np.ascontiguousarray(B_ref, dtype=np.float64).reshape(-1, 3)
    wv = np.ascontiguousarray(w, dtype=np.float64)
    pa, no = _f32(params, ML_NPARAM), _f32(norm, ML_NNORM)
    out = np.empty(4)
    grad = np.empty(ML_NPARAM) if want_grad else None
    e = L.orc_ml_loss(len(frames), _ip(n_of), _dp(r), _dp(s), _dp(boxes), _dp(E_ref), _dp(F_ref), _dp(B_ref),
                      _dp(wv), HBAR, _fp(pa), _fp(no), _dp(out), _opt(grad))
    if e:
        raise OracleError(e)
    return out, grad


def ml_adam(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step on float32 params (in place); m, v float64 moments (in place)."""
    L = lib()
    assert params.dtype == np.float32 and params.flags.c_contiguous
    g = np.ascontiguousarray(grad, dtype=np.float64)
    L.orc_ml_adam(params.size, _fp(params), _dp(g), _dp(m), _dp(v), int(t), float(lr), float(beta1),
                  float(beta2), float(eps))


def ml_eval_sample(r, s, box, params, norm, idx):
    """E_i, F_i, B_i, D_i of the sampled atoms idx of a (large) frame, each from
    scratch by scans over all atoms.  Returns dict(e_atom, F, B, D)."""
    L = lib()
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1, 3)
    s = np.ascontiguousarray(s, dtype=np.float64).reshape(-1, 3)
    box = np.ascontiguousarray(box, dtype=np.float64).reshape(3)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    m = len(idx)
    pa, no = _f32(params, ML_NPARAM), _f32(norm, ML_NNORM)
    e = np.empty(m); F = np.empty((m, 3)); B = np.empty((m, 3)); D = np.empty((m, ML_NF))
    rc = L.orc_ml_eval_sample(r.shape[0], _dp(r), _dp(s), _dp(box), _fp(pa), _fp(no), m, _ip(idx), _dp(e), _dp(F),
                              _dp(B), _dp(D))
    if rc:
        raise OracleError(rc)
    return dict(e_atom=e, F=F, B=B, D=D)
