"""ctypes binding of libsl (include/sl.h): argument marshalling only.

Every step of the method runs in the CUDA kernels of libsl.so; this module
allocates device buffers with PyTorch, passes their pointers and raises on
error codes.  There is no fallback: if libsl.so is missing or cannot load,
`load()` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsl.so")

SL_OK = 0
SL_ERR_ARG, SL_ERR_CUDA, SL_ERR_BOX, SL_ERR_SPIN_NORM = -1, -2, -3, -4
SL_ERR_SKIN, SL_ERR_TIMEOUT, SL_ERR_NONFINITE, SL_ERR_WORKSPACE, SL_ERR_NBR_OVERFLOW = -5, -6, -7, -8, -9
SL_ROT_RODRIGUES, SL_ROT_CAYLEY = 0, 1
SL_HAM_ANALYTIC, SL_HAM_LEARNED = 0, 1

# Learned model layout (include/sl.h)
SL_ML_NF, SL_ML_NH, SL_ML_RC = 48, 64, 6.0
SL_ML_OFF_W1, SL_ML_OFF_B1, SL_ML_OFF_W2, SL_ML_OFF_B2, SL_ML_OFF_W3, SL_ML_OFF_B3 = 0, 3072, 3136, 7232, 7296, 7360
SL_ML_NPARAM, SL_ML_NNORM = 7361, 192

# Every exported symbol of include/sl.h.
EXPORTS = (
    "sl_workspace_bytes", "sl_sector_grid", "sl_init", "sl_build_neighbors", "sl_step", "sl_set_dt", "sl_set_field",
    "sl_energy", "sl_magnetization", "sl_get_state", "sl_set_state", "sl_get_state_host",
    "sl_set_state_host", "sl_get_forces", "sl_get_omega", "sl_get_order", "sl_counters", "sl_set_timing",
    "sl_get_timing", "sl_magnetization_static", "sl_df_fma_rate", "sl_df_eval", "sl_check_bounded_wait", "sl_set_eam_tables", "sl_status", "sl_strerror", "sl_destroy",
    "sl_workspace_bytes_batch", "sl_init_batch", "sl_batch_size", "sl_energy_batch", "sl_magnetization_batch",
    "sl_ml_set_model", "sl_ml_get_model", "sl_ml_eval", "sl_ml_descriptor_stats", "sl_ml_gate", "sl_ml_vjp",
    "sl_ml_train_step", "sl_autotune", "sl_set_launch_shape",
)
PHASES = ("kick", "spin_half_op_1", "drift_rebuild", "exchange_table", "spin_half_op_2", "force_kick")


class sl_eam_tables(ctypes.Structure):
    _fields_ = [("nrho", ctypes.c_int32), ("nr", ctypes.c_int32), ("drho", ctypes.c_double),
                ("dr", ctypes.c_double), ("F", ctypes.POINTER(ctypes.c_double)),
                ("rho", ctypes.POINTER(ctypes.c_double)), ("phi", ctypes.POINTER(ctypes.c_double))]


class sl_params(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int32), ("rotation", ctypes.c_int32), ("fix_lattice", ctypes.c_int32),
        ("rebuild_every", ctypes.c_int32), ("morse_shift_energy", ctypes.c_int32),
        ("max_ex_neighbors", ctypes.c_int32), ("max_morse_neighbors", ctypes.c_int32),
        ("hamiltonian", ctypes.c_int32),
        ("box", ctypes.c_double * 3), ("mass_amu", ctypes.c_double), ("mu_s_muB", ctypes.c_double),
        ("H_tesla", ctypes.c_double * 3), ("dt_ps", ctypes.c_double),
        ("ex_alpha_eV", ctypes.c_double), ("ex_gamma", ctypes.c_double), ("ex_delta_A", ctypes.c_double),
        ("ex_rc_A", ctypes.c_double),
        ("morse_D0_eV", ctypes.c_double), ("morse_alpha_invA", ctypes.c_double), ("morse_r0_A", ctypes.c_double),
        ("morse_rc_A", ctypes.c_double), ("skin_A", ctypes.c_double),
        ("lambda_", ctypes.c_double), ("temperature_K", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("replica", ctypes.c_int32), ("reserved1", ctypes.c_int32),
        ("lattice_gamma_ps", ctypes.c_double), ("lattice_temperature_K", ctypes.c_double),
        ("aniso_K_eV", ctypes.c_double), ("aniso_axis", ctypes.c_double * 3),
        ("neel_alpha_eV", ctypes.c_double), ("neel_gamma", ctypes.c_double), ("neel_delta_A", ctypes.c_double),
        ("dmi_alpha_eV", ctypes.c_double), ("dmi_gamma", ctypes.c_double), ("dmi_delta_A", ctypes.c_double),
        ("eam_A_eV", ctypes.c_double), ("eam_d_A", ctypes.c_double), ("eam_beta", ctypes.c_double),
        ("subtract_ground_exchange", ctypes.c_int32), ("eam_tabulated", ctypes.c_int32),
    ]


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_lib = None


def load():
    """Load libsl.so (built in-tree by build.py).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1801_10233_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER(sl_params)
    sig = {
        "sl_workspace_bytes": ([P, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "sl_sector_grid": ([P, ctypes.POINTER(ctypes.c_int32), _dp], ctypes.c_int),
        "sl_init": ([P, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
        "sl_build_neighbors": ([_vp], ctypes.c_int),
        "sl_step": ([_vp, ctypes.c_int32], ctypes.c_int),
        "sl_set_dt": ([_vp, ctypes.c_double], ctypes.c_int),
        "sl_set_field": ([_vp, _dp], ctypes.c_int),
        "sl_energy": ([_vp, _dp], ctypes.c_int),
        "sl_magnetization": ([_vp, _dp], ctypes.c_int),
        "sl_get_state": ([_vp, _vp, _vp, _vp], ctypes.c_int),
        "sl_set_state": ([_vp, _vp, _vp, _vp], ctypes.c_int),
        "sl_get_state_host": ([_vp, _vp, _vp, _vp], ctypes.c_int),
        "sl_set_state_host": ([_vp, _vp, _vp, _vp], ctypes.c_int),
        "sl_get_forces": ([_vp, _vp], ctypes.c_int),
        "sl_get_omega": ([_vp, _vp], ctypes.c_int),
        "sl_get_order": ([_vp, _vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "sl_counters": ([_vp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "sl_set_timing": ([_vp, ctypes.c_int32], ctypes.c_int),
        "sl_get_timing": ([_vp, _dp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "sl_magnetization_static": ([_vp, ctypes.c_int32, _vp, _vp], ctypes.c_int),
        "sl_df_fma_rate": ([ctypes.c_int32, _dp, _dp], ctypes.c_int),
        "sl_df_eval": ([ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
        "sl_check_bounded_wait": ([ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
        "sl_set_eam_tables": ([_vp, ctypes.POINTER(sl_eam_tables)], ctypes.c_int),
        "sl_status": ([_vp], ctypes.c_int),
        "sl_workspace_bytes_batch": ([P, ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
        "sl_init_batch": ([P, ctypes.c_int32, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)],
                          ctypes.c_int),
        "sl_batch_size": ([_vp], ctypes.c_int),
        "sl_energy_batch": ([_vp, _dp], ctypes.c_int),
        "sl_magnetization_batch": ([_vp, _dp], ctypes.c_int),
        "sl_ml_set_model": ([_vp, _vp, _vp], ctypes.c_int),
        "sl_ml_get_model": ([_vp, _vp], ctypes.c_int),
        "sl_ml_eval": ([_vp, _dp, _vp, _vp, _vp], ctypes.c_int),
        "sl_ml_descriptor_stats": ([_vp, _dp], ctypes.c_int),
        "sl_ml_gate": ([_vp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "sl_ml_vjp": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
        "sl_ml_train_step": ([_vp, _vp, _vp, _vp, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, _dp], ctypes.c_int),
        "sl_autotune": ([_vp, _vp, ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "sl_set_launch_shape": ([_vp, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
        "sl_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "sl_destroy": ([_vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


class SlError(RuntimeError):
    def __init__(self, code, what=""):
        msg = load().sl_strerror(int(code)).decode()
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")
        self.code = int(code)


def check(code, what=""):
    if code != SL_OK:
        raise SlError(code, what)


def make_params(p: dict) -> sl_params:
    q = sl_params()
    q.n_atoms = int(p["n_atoms"])
    q.rotation = int(p.get("rotation", 0))
    q.fix_lattice = int(p.get("fix_lattice", 0))
    q.rebuild_every = int(p.get("rebuild_every", 0))
    q.morse_shift_energy = int(p.get("morse_shift_energy", 1))
    q.max_ex_neighbors = int(p.get("max_ex_neighbors", 0))
    q.max_morse_neighbors = int(p.get("max_morse_neighbors", 0))
    for a in range(3):
        q.box[a] = float(p["box"][a])
        q.H_tesla[a] = float(p["H_tesla"][a])
    q.mass_amu = float(p["mass_amu"])
    q.mu_s_muB = float(p["mu_s_muB"])
    q.dt_ps = float(p["dt_ps"])
    q.ex_alpha_eV, q.ex_gamma = float(p["ex_alpha_eV"]), float(p["ex_gamma"])
    q.ex_delta_A, q.ex_rc_A = float(p["ex_delta_A"]), float(p["ex_rc_A"])
    q.morse_D0_eV, q.morse_alpha_invA = float(p["morse_D0_eV"]), float(p["morse_alpha_invA"])
    q.morse_r0_A, q.morse_rc_A = float(p["morse_r0_A"]), float(p["morse_rc_A"])
    q.skin_A = float(p["skin_A"])
    q.lambda_ = float(p.get("lambda", 0.0))
    q.temperature_K = float(p.get("temperature_K", 0.0))
    q.seed = int(p.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    q.replica = int(p.get("replica", 0))
    q.hamiltonian = int(p.get("hamiltonian", 0))
    q.lattice_gamma_ps = float(p.get("lattice_gamma_ps", 0.0))
    q.lattice_temperature_K = float(p.get("lattice_temperature_K", 0.0))
    q.aniso_K_eV = float(p.get("aniso_K_eV", 0.0))
    axis = p.get("aniso_axis", (0.0, 0.0, 1.0))
    for a in range(3):
        q.aniso_axis[a] = float(axis[a])
    q.neel_alpha_eV = float(p.get("neel_alpha_eV", 0.0))
    q.neel_gamma = float(p.get("neel_gamma", 0.0))
    q.neel_delta_A = float(p.get("neel_delta_A", 1.0))
    q.dmi_alpha_eV = float(p.get("dmi_alpha_eV", 0.0))
    q.dmi_gamma = float(p.get("dmi_gamma", 0.0))
    q.dmi_delta_A = float(p.get("dmi_delta_A", 1.0))
    q.eam_A_eV = float(p.get("eam_A_eV", 0.0))
    q.eam_d_A = float(p.get("eam_d_A", 1.0))
    q.eam_beta = float(p.get("eam_beta", 0.0))
    q.subtract_ground_exchange = int(p.get("subtract_ground_exchange", 0))
    q.eam_tabulated = int(p.get("eam_tabulated", 0))
    return q


def params_array(ps) -> ctypes.Array:
    """ctypes array of sl_params for one dict or a list of dicts (a batch)."""
    ps = [ps] if isinstance(ps, dict) else list(ps)
    arr = (sl_params * len(ps))()
    for k, p in enumerate(ps):
        arr[k] = make_params(p)
    return arr


def workspace_bytes(p) -> int:
    """Workspace bytes for one system (dict) or a batch (list of dicts)."""
    L = load()
    arr = params_array(p)
    b = ctypes.c_size_t(0)
    check(L.sl_workspace_bytes_batch(arr, len(arr), ctypes.byref(b)), "sl_workspace_bytes_batch")
    return int(b.value)


def sector_grid(p):
    """(sectors per edge, sector edges in A) of the sectored sweep for the
    parameter dict p, computed on the host."""
    n = (ctypes.c_int32 * 3)()
    e = (ctypes.c_double * 3)()
    check(load().sl_sector_grid(ctypes.byref(make_params(p)), n, e), "sl_sector_grid")
    return [int(x) for x in n], [float(x) for x in e]


def df_fma_rate(iters=4096):
    """(flop/s, ms) of the double-float multiply-add on the current device
    (2 flop per multiply-add), measured by the library."""
    f = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    check(load().sl_df_fma_rate(int(iters), ctypes.byref(f), ctypes.byref(ms)), "sl_df_fma_rate")
    return f.value, ms.value


SL_DF_EXP, SL_DF_RSQRT, SL_DF_SQRT = 0, 1, 2


def df_eval(fn: int, x_ptr: int, y_ptr: int, n: int, stream: int = 0):
    """y = f(x) in the library's double-float arithmetic (device pointers to
    n doubles, stream-ordered on `stream`)."""
    check(load().sl_df_eval(int(fn), x_ptr, y_ptr, int(n), stream), "sl_df_eval")


def strerror(code: int) -> str:
    return load().sl_strerror(int(code)).decode()


def _arr_ptr(a):
    return a.ctypes.data_as(_dp)
