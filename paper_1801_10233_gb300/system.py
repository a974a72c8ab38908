"""`System`: one coupled spin-lattice system driven through libsl's C ABI.

PyTorch provides the device memory (state tensors and the workspace) and the
CUDA stream; every computation runs in libsl's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import check


def _cuda_f64(x, device):
    if isinstance(x, torch.Tensor):
        t = x.to(device=device, dtype=torch.float64)
    else:
        t = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device=device)
    return t.reshape(-1, 3).contiguous()


class System:
    """A system of `params["n_atoms"]` atoms with positions r, velocities v and
    unit spins s ([N, 3] float64; numpy arrays or tensors, caller order).

    `params` may also be a list of parameter dicts: a batch of independent
    replicas (sl_init_batch), whose atoms are given back to back in r, v, s."""

    def __init__(self, params, r, v, s, device=None, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libsl needs a CUDA GPU")
        self._L = _lib.load()
        plist = [params] if isinstance(params, dict) else list(params)
        self.params = dict(plist[0])
        self.replica_params = [dict(p) for p in plist]
        self.nrep = len(plist)
        self.n = int(sum(int(p["n_atoms"]) for p in plist))
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._p = _lib.params_array(plist)
        nbytes = _lib.workspace_bytes(plist)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self._ws_bytes = nbytes
        r, v, s = (_cuda_f64(a, self.device) for a in (r, v, s))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            torch.cuda.current_stream(self.device).synchronize()
            rc = self._L.sl_init_batch(self._p, self.nrep, r.data_ptr(), v.data_ptr(), s.data_ptr(),
                                       self._ws_ptr, self._ws_bytes, self.stream.cuda_stream, ctypes.byref(h))
        check(rc, "sl_init_batch")
        self._h = h

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.sl_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- dynamics ----------------------------------------------------------
    def step(self, n: int = 1):
        check(self._L.sl_step(self._h, int(n)), "sl_step")

    def build_neighbors(self):
        check(self._L.sl_build_neighbors(self._h), "sl_build_neighbors")

    def set_dt(self, dt: float):
        check(self._L.sl_set_dt(self._h, float(dt)), "sl_set_dt")

    def set_field(self, H):
        h = np.ascontiguousarray(H, dtype=np.float64)
        check(self._L.sl_set_field(self._h, _lib._arr_ptr(h)), "sl_set_field")

    def set_eam_tables(self, F, drho, rho, phi, dr):
        """Tables of the tabulated embedded-atom potential (eam_tabulated = 1):
        F on rho = k drho, rho(r) and phi(r) on r = k dr (host arrays)."""
        F = np.ascontiguousarray(F, dtype=np.float64)
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        if rho.shape != phi.shape:
            raise ValueError("rho and phi tables differ in length")
        t = _lib.sl_eam_tables(len(F), len(rho), float(drho), float(dr), _lib._arr_ptr(F), _lib._arr_ptr(rho),
                               _lib._arr_ptr(phi))
        check(self._L.sl_set_eam_tables(self._h, ctypes.byref(t)), "sl_set_eam_tables")

    # -- observables -------------------------------------------------------
    def energy(self) -> np.ndarray:
        """E_kin, E_morse, E_exch, E_zeeman, E_total (eV), T_L, T_S (K), 0."""
        out = np.empty(8)
        check(self._L.sl_energy(self._h, _lib._arr_ptr(out)), "sl_energy")
        return out

    def magnetization(self) -> np.ndarray:
        out = np.empty(4)
        check(self._L.sl_magnetization(self._h, _lib._arr_ptr(out)), "sl_magnetization")
        return out

    def energy_per_replica(self) -> np.ndarray:
        """[n_replicas, 8] as energy() for each replica."""
        out = np.empty((self.nrep, 8))
        check(self._L.sl_energy_batch(self._h, _lib._arr_ptr(out)), "sl_energy_batch")
        return out

    def magnetization_per_replica(self) -> np.ndarray:
        out = np.empty((self.nrep, 4))
        check(self._L.sl_magnetization_batch(self._h, _lib._arr_ptr(out)), "sl_magnetization_batch")
        return out

    def status(self) -> int:
        return int(self._L.sl_status(self._h))

    def counters(self):
        out = (ctypes.c_int64 * 8)()
        check(self._L.sl_counters(self._h, out), "sl_counters")
        return dict(steps=out[0], rebuilds=out[1], max_ex_seen=out[2], max_morse_seen=out[3],
                    kernels_per_step=out[4], graph=bool(out[5]))

    def set_timing(self, enable: bool):
        """Per-phase CUDA-event timing of each step (direct launches)."""
        check(self._L.sl_set_timing(self._h, int(bool(enable))), "sl_set_timing")

    def timing(self):
        """{phase: (total ms, launches)} since timing was enabled."""
        ms = np.zeros(8)
        cnt = (ctypes.c_int64 * 8)()
        check(self._L.sl_get_timing(self._h, _lib._arr_ptr(ms), cnt), "sl_get_timing")
        return {name: (float(ms[k]), int(cnt[k])) for k, name in enumerate(_lib.PHASES)}

    # -- state transfer ----------------------------------------------------
    def _empty3(self):
        return torch.empty((self.n, 3), dtype=torch.float64, device=self.device)

    def state(self):
        """(r, v, s) as new [N, 3] float64 CUDA tensors in caller order."""
        r, v, s = self._empty3(), self._empty3(), self._empty3()
        check(self._L.sl_get_state(self._h, r.data_ptr(), v.data_ptr(), s.data_ptr()), "sl_get_state")
        self.stream.synchronize()
        return r, v, s

    def set_state(self, r, v, s):
        r, v, s = (_cuda_f64(a, self.device) for a in (r, v, s))
        self.stream.synchronize()
        check(self._L.sl_set_state(self._h, r.data_ptr(), v.data_ptr(), s.data_ptr()), "sl_set_state")
        self.stream.synchronize()

    def state_host(self, r: torch.Tensor, v: torch.Tensor, s: torch.Tensor):
        """Copy the state into host tensors (pinned for speed) [N, 3] float64."""
        check(self._L.sl_get_state_host(self._h, r.data_ptr(), v.data_ptr(), s.data_ptr()), "sl_get_state_host")

    def set_state_host(self, r: torch.Tensor, v: torch.Tensor, s: torch.Tensor):
        """Replace the state from host tensors (pinned for speed) [N, 3] float64."""
        check(self._L.sl_set_state_host(self._h, r.data_ptr(), v.data_ptr(), s.data_ptr()), "sl_set_state_host")

    def forces(self):
        F = self._empty3()
        check(self._L.sl_get_forces(self._h, F.data_ptr()), "sl_get_forces")
        self.stream.synchronize()
        return F

    def omega(self):
        w = self._empty3()
        check(self._L.sl_get_omega(self._h, w.data_ptr()), "sl_get_omega")
        self.stream.synchronize()
        return w

    def order(self):
        o = torch.empty(self.n, dtype=torch.int32, device=self.device)
        cs = (ctypes.c_int32 * 9)()
        ns = (ctypes.c_int32 * 3)()
        check(self._L.sl_get_order(self._h, o.data_ptr(), cs, ns), "sl_get_order")
        return dict(order=o.cpu().numpy(), colour_start=np.array(cs[:], dtype=np.int32),
                    nsec=np.array(ns[:], dtype=np.int32))

    # -- launch shapes -------------------------------------------------------
    def autotune(self, steps: int = 3):
        """Time every launch shape on this system's own state (restored
        afterwards) and keep the fastest.  Returns dict(variant, block,
        ns_per_step, default_ns_per_step, candidates, sectors_per_block)."""
        scratch = torch.empty(self._ws_bytes, dtype=torch.uint8, device=self.device)
        out = (ctypes.c_int64 * 8)()
        self.stream.synchronize()
        check(self._L.sl_autotune(self._h, scratch.data_ptr(), self._ws_bytes, int(steps), out), "sl_autotune")
        del scratch
        return dict(variant=int(out[0]), block=int(out[1]), ns_per_step=int(out[2]),
                    default_ns_per_step=int(out[3]), candidates=int(out[4]), sectors_per_block=int(out[5]))

    def set_launch_shape(self, variant: int, block: int):
        check(self._L.sl_set_launch_shape(self._h, int(variant), int(block)), "sl_set_launch_shape")

    # -- learned Hamiltonian -----------------------------------------------
    def ml_set_model(self, params, norm):
        """Install the network (float32 params [SL_ML_NPARAM], norm [SL_ML_NNORM])."""
        p = torch.as_tensor(params, dtype=torch.float32).to(self.device).contiguous()
        q = torch.as_tensor(norm, dtype=torch.float32).to(self.device).contiguous()
        self.stream.synchronize()
        check(self._L.sl_ml_set_model(self._h, p.data_ptr(), q.data_ptr()), "sl_ml_set_model")
        self.stream.synchronize()

    def ml_get_model(self) -> torch.Tensor:
        p = torch.empty(_lib.SL_ML_NPARAM, dtype=torch.float32, device=self.device)
        check(self._L.sl_ml_get_model(self._h, p.data_ptr()), "sl_ml_get_model")
        self.stream.synchronize()
        return p

    def ml_eval(self, want_D=False):
        """Network at the current state (gate ignored): (E per replica [nrep]
        numpy, F [N,3], B = -dE/ds [N,3], D [N,48] or None) in caller order."""
        e = np.empty(self.nrep)
        F, B = self._empty3(), self._empty3()
        D = torch.empty((self.n, _lib.SL_ML_NF), dtype=torch.float64, device=self.device) if want_D else None
        check(self._L.sl_ml_eval(self._h, _lib._arr_ptr(e), F.data_ptr(), B.data_ptr(),
                                 D.data_ptr() if D is not None else None), "sl_ml_eval")
        return e, F, B, D

    def ml_descriptor_stats(self) -> np.ndarray:
        """[4, 48]: mean, std, min, max of the raw descriptors over all atoms."""
        out = np.empty((4, _lib.SL_ML_NF))
        check(self._L.sl_ml_descriptor_stats(self._h, _lib._arr_ptr(out)), "sl_ml_descriptor_stats")
        return out

    def ml_gate(self):
        """(atoms out of range at the last evaluation point, network in use there, points handed back)."""
        out = (ctypes.c_int64 * 4)()
        check(self._L.sl_ml_gate(self._h, out), "sl_ml_gate")
        return int(out[0]), int(out[1]), int(out[2])

    def ml_vjp(self, gE=None, gF=None, gB=None) -> torch.Tensor:
        """d/dparams of sum gE.E_rep + sum gF.F + sum gB.B (float64 [SL_ML_NPARAM])."""
        def dev(x, shape):
            if x is None:
                return None
            return torch.as_tensor(x, dtype=torch.float64).to(self.device).reshape(shape).contiguous()
        gE_, gF_, gB_ = dev(gE, (self.nrep,)), dev(gF, (self.n, 3)), dev(gB, (self.n, 3))
        grad = torch.empty(_lib.SL_ML_NPARAM, dtype=torch.float64, device=self.device)
        self.stream.synchronize()
        check(self._L.sl_ml_vjp(self._h, gE_.data_ptr() if gE_ is not None else None,
                                gF_.data_ptr() if gF_ is not None else None,
                                gB_.data_ptr() if gB_ is not None else None, grad.data_ptr()), "sl_ml_vjp")
        self.stream.synchronize()
        return grad

    def ml_train_step(self, E_ref, F_ref, B_ref, w, lr, beta1=0.9, beta2=0.999, eps=1e-8, want_loss=True):
        """One Adam step on the frames currently loaded; returns the loss terms
        (L, L_E, L_F, L_omega) before the update, or None."""
        E_ref = torch.as_tensor(E_ref, dtype=torch.float64).to(self.device).contiguous()
        F_ref = torch.as_tensor(F_ref, dtype=torch.float64).to(self.device).reshape(-1, 3).contiguous()
        B_ref = torch.as_tensor(B_ref, dtype=torch.float64).to(self.device).reshape(-1, 3).contiguous()
        wv = np.ascontiguousarray(w, dtype=np.float64)
        loss = np.empty(4) if want_loss else None
        check(self._L.sl_ml_train_step(self._h, E_ref.data_ptr(), F_ref.data_ptr(), B_ref.data_ptr(),
                                       _lib._arr_ptr(wv), float(lr), float(beta1), float(beta2), float(eps),
                                       _lib._arr_ptr(loss) if loss is not None else None), "sl_ml_train_step")
        if loss is None:
            self.stream.synchronize()
        return loss
