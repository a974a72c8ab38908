"""Learned per-atom Hamiltonian: PyTorch autograd front ends, training data
and training loop around libsl's kernels (include/sl.h, "Learned per-atom
Hamiltonian").

Every number here comes from libsl: the descriptors, the network, its
backward pass (forces -dE/dr and fields -dE/ds), the parameter gradients and
the Adam update all run in CUDA kernels; this module only moves tensors.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import _lib, inputs
from .system import System

HBAR = 6.582119569e-4        # eV ps / rad
MU_B = 5.7883818060e-5       # eV / T


def zeeman_field(params) -> np.ndarray:
    """mu_s mu_B H (eV): the Zeeman part of -dH/ds, which the network does not model."""
    return float(params["mu_s_muB"]) * MU_B * np.asarray(params["H_tesla"], dtype=np.float64)


class LearnedEnergy(torch.autograd.Function):
    """E_r(r, s) = sum of the network's E_i over replica r.

    forward(r, s, params, system) -> E [n_replicas]; backward gives
    dE/dr = -F and dE/ds = -B from the hand-written backward kernel, and
    dE/dparams from the parameter vector-Jacobian product kernel.  `system`
    is a System created with hamiltonian = SL_HAM_LEARNED; its state is
    replaced by (r, s) (velocities zero)."""

    @staticmethod
    def forward(ctx, r, s, params, system: System):
        system.ml_set_model(params.detach(), system._ml_norm)
        system.set_state(r.detach(), torch.zeros_like(r, dtype=torch.float64), s.detach())
        e, F, B, _ = system.ml_eval()
        ctx.system = system
        ctx.save_for_backward(F, B)
        return torch.as_tensor(e, dtype=torch.float64, device=r.device)

    @staticmethod
    def backward(ctx, gE):
        F, B = ctx.saved_tensors
        system = ctx.system
        rep = system._atom_replica.to(gE.device)
        g_atom = gE.to(torch.float64)[rep].unsqueeze(1)
        grad_r = -g_atom * F if ctx.needs_input_grad[0] else None
        grad_s = -g_atom * B if ctx.needs_input_grad[1] else None
        grad_p = None
        if ctx.needs_input_grad[2]:
            grad_p = system.ml_vjp(gE=gE).to(torch.float32)
        return grad_r, grad_s, grad_p, None


class LearnedForces(torch.autograd.Function):
    """(E [n_replicas], F [N,3], B [N,3]) of the network as functions of its
    parameters; backward is the forward-over-reverse vector-Jacobian product
    kernel, so a loss on forces and fields can be differentiated with respect
    to the parameters."""

    @staticmethod
    def forward(ctx, params, system: System):
        system.ml_set_model(params.detach(), system._ml_norm)
        e, F, B, _ = system.ml_eval()
        ctx.system = system
        return torch.as_tensor(e, dtype=torch.float64, device=F.device), F, B

    @staticmethod
    def backward(ctx, gE, gF, gB):
        g = ctx.system.ml_vjp(gE=gE, gF=gF, gB=gB)
        return g.to(torch.float32), None


def learned_system(params_list, r, v, s, norm, model, device=None) -> System:
    """A System with the learned Hamiltonian and a model installed."""
    plist = [params_list] if isinstance(params_list, dict) else list(params_list)
    plist = [dict(p, hamiltonian=_lib.SL_HAM_LEARNED) for p in plist]
    sysm = System(plist, r, v, s, device=device)
    sysm._ml_norm = torch.as_tensor(norm, dtype=torch.float32)
    counts = [int(p["n_atoms"]) for p in plist]
    sysm._atom_replica = torch.repeat_interleave(torch.arange(len(counts)), torch.tensor(counts))
    sysm.ml_set_model(model, norm)
    return sysm


def normalisation(stats: np.ndarray, gate_margin: float = 0.5) -> np.ndarray:
    """Normalisation vector from descriptor statistics [4, 48] (mean, std,
    min, max): inv_std = 1/(std + 1e-3); the gate accepts [min - m (max - min),
    max + m (max - min)]."""
    mean, std, lo, hi = stats
    span = np.maximum(hi - lo, 1e-6)
    out = np.concatenate([mean, 1.0 / (std + 1e-3), lo - gate_margin * span, hi + gate_margin * span])
    return out.astype(np.float32)


# ---------------------------------------------------------------------------
# Training data: snapshots of analytic trajectories
# ---------------------------------------------------------------------------
def snapshots(plist, r, v, s, n_snap, every, device=None, warm=0):
    """Run the analytic Hamiltonian on the replicas of `plist` and take n_snap
    snapshots, `every` steps apart.  Returns a dict of device tensors:
    r, s [n_snap, N, 3], E [n_snap, n_replicas] (Morse + exchange energy),
    F [n_snap, N, 3], B [n_snap, N, 3] (-dE/ds without the Zeeman part)."""
    sysa = System(plist, r, v, s, device=device)
    if warm:
        sysa.step(warm)
    zee = torch.as_tensor(np.stack([zeeman_field(p) for p in plist]), device=sysa.device)
    counts = [int(p["n_atoms"]) for p in plist]
    rep = torch.repeat_interleave(torch.arange(len(counts)), torch.tensor(counts)).to(sysa.device)
    out = {k: [] for k in ("r", "s", "E", "F", "B")}
    for k in range(n_snap):
        if k:
            sysa.step(every)
        rr, _, ss = sysa.state()
        e = sysa.energy_per_replica()
        out["r"].append(rr)
        out["s"].append(ss)
        out["E"].append(torch.as_tensor(e[:, 1] + e[:, 2], device=sysa.device))
        out["F"].append(sysa.forces())
        out["B"].append(sysa.omega() * HBAR - zee[rep])
    sysa.close()
    return {k: torch.stack(v) for k, v in out.items()}


def train(sysm: System, data, epochs, lr, w=(1.0, 1.0, 1e-6), batch_frames=None, lr_min=None, log=None):
    """Adam on the network of `sysm`, whose replicas are the frames of one
    batch: data["r"], data["s"] [n_frames, N, 3] (N = sysm.n) with labels
    data["E"] [n_frames, nrep], data["F"], data["B"].  Cosine learning-rate
    decay to lr_min.  Returns the list of per-step losses."""
    n_frames = data["r"].shape[0]
    zeros = torch.zeros_like(data["r"][0])
    losses = []
    total = epochs * n_frames
    lr_min = lr if lr_min is None else lr_min
    step = 0
    for ep in range(epochs):
        for f in range(n_frames):
            cur = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * step / max(1, total - 1)))
            sysm.set_state(data["r"][f], zeros, data["s"][f])
            loss = sysm.ml_train_step(data["E"][f], data["F"][f], data["B"][f], w, cur)
            losses.append(loss.copy())
            if log is not None and (step % log == 0):
                print(f"train step {step} lr {cur:.2e} loss {loss}")
            step += 1
    return losses


def learned_params(p):
    """The parameter dict of a system run with the learned Hamiltonian (no spin bath)."""
    return dict(p, hamiltonian=_lib.SL_HAM_LEARNED, temperature_K=0.0, **{"lambda": 0.0})


def training_set(n_frames=20000, n_replicas=64, every=10, warm=100, seed=18015, device=None):
    """Snapshots of bath-coupled analytic trajectories of 10^3-cell replicas
    at 50..1200 K (inputs.training_replicas): n_frames frames, n_replicas per
    snapshot.  Returns (plist, data) with data as snapshots()."""
    plist, r, v, s = inputs.training_replicas(n_replicas, seed)
    n_snap = max(1, -(-n_frames // n_replicas))
    return plist, snapshots(plist, r, v, s, n_snap, every, device=device, warm=warm)


def fit_normalisation(sysm: System, data, picks=(0,), gate_margin=0.5):
    """Descriptor statistics of a few training snapshots -> normalisation vector."""
    zeros = torch.zeros_like(data["r"][0])
    stats = []
    for k in picks:
        sysm.set_state(data["r"][k], zeros, data["s"][k])
        stats.append(sysm.ml_descriptor_stats())
    st = np.stack(stats)
    comb = np.stack([st[:, 0].mean(0), np.sqrt((st[:, 1] ** 2).mean(0)), st[:, 2].min(0), st[:, 3].max(0)])
    return normalisation(comb, gate_margin)


def train_model(plist, data, epochs=8, lr=2e-3, lr_min=2e-5, w=(1.0, 1.0, 1e-4), seed=3, log=None, device=None):
    """Fit the network to the snapshots (one Adam step per snapshot of all
    replicas).  Returns (params float32 numpy, norm, per-step losses, seconds)."""
    import time
    lp = [learned_params(p) for p in plist]
    r0 = data["r"][0]
    e0 = float(data["E"][0].sum().item() / r0.shape[0])
    init = inputs.ml_init_params(seed, e0=e0)
    sysm = System(lp, r0, torch.zeros_like(r0), data["s"][0], device=device)
    counts = [int(p["n_atoms"]) for p in lp]
    sysm._atom_replica = torch.repeat_interleave(torch.arange(len(counts)), torch.tensor(counts))
    n = data["r"].shape[0]
    open_gate = np.concatenate([np.zeros(48), np.ones(48), np.full(48, -3e38), np.full(48, 3e38)]).astype(np.float32)
    sysm.ml_set_model(init, open_gate)
    norm = fit_normalisation(sysm, data, picks=sorted({0, n // 2, n - 1}))
    sysm.ml_set_model(init, norm)
    sysm._ml_norm = torch.as_tensor(norm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = train(sysm, data, epochs, lr, w=w, lr_min=lr_min, log=log)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    params = sysm.ml_get_model().cpu().numpy()
    sysm.close()
    return params, norm, np.array(losses), secs


def _drift(ts, es):
    """Least-squares slope of es against ts."""
    t = np.asarray(ts, dtype=np.float64)
    e = np.asarray(es, dtype=np.float64)
    if len(t) < 2:
        return 0.0
    A = np.stack([t, np.ones_like(t)], 1)
    return float(np.linalg.lstsq(A, e, rcond=None)[0][0])


def judge(params, norm, p, r, v, s, steps, every, device=None):
    """Run the learned and the analytic Hamiltonian side by side from the same
    state and report the learned model's errors (energy per atom, forces,
    precession vector normal to s) against the analytic Hamiltonian at the
    learned trajectory's states, the energy drift of both runs (eV/atom/ps),
    the largest |M| difference between the runs, and the gate counters."""
    n = int(p["n_atoms"])
    pa = dict(p, hamiltonian=_lib.SL_HAM_ANALYTIC)
    plain = System(pa, r, v, s, device=device)
    probe = System(pa, r, v, s, device=device)
    lsys = System(learned_params(p), r, v, s, device=device)
    lsys._ml_norm = torch.as_tensor(norm)
    lsys._atom_replica = torch.zeros(n, dtype=torch.long)
    lsys.ml_set_model(params, norm)
    zee = torch.as_tensor(zeeman_field(p), device=lsys.device)
    dt = float(p["dt_ps"])
    ts, e_plain, e_learn, dM = [], [], [], []
    errE, errF, errW = [], [], []
    for k in range(0, steps + 1, every):
        if k:
            plain.step(every)
            lsys.step(every)
        ts.append(k * dt)
        e_plain.append(plain.energy()[4] / n)
        e_learn.append(lsys.energy()[4] / n)
        dM.append(abs(plain.magnetization()[3] - lsys.magnetization()[3]))
        rl, vl, sl = lsys.state()
        probe.set_state(rl, vl, sl)
        ea = probe.energy()
        el, Fl, Bl, _ = lsys.ml_eval()
        errE.append(abs(el[0] - (ea[1] + ea[2])) / n)
        dF = Fl - probe.forces()
        errF.append(float(torch.sqrt((dF ** 2).sum(1).mean()).item()))
        dB = (Bl + zee) / HBAR - probe.omega()
        dB = dB - (dB * sl).sum(1, keepdim=True) * sl
        errW.append(float(torch.sqrt((dB ** 2).sum(1).mean()).item()))
    gate = lsys.ml_gate()
    out = dict(steps=steps, atoms=n, drift_plain_eV_per_atom_ps=_drift(ts, e_plain),
               drift_learned_eV_per_atom_ps=_drift(ts, e_learn), max_dM=float(max(dM)),
               err_E_eV_per_atom=float(max(errE)), rmse_F_eV_per_A=float(max(errF)),
               rmse_omega_perp_rad_per_ps=float(max(errW)), gate_points_handed_back=gate[2])
    for x in (plain, probe, lsys):
        x.close()
    return out


def main(argv=None):
    """Train the network on snapshots and run the learned Hamiltonian beside
    the analytic one on a workload:
        python -m paper_1801_10233_gb300.learned --frames 640 --epochs 1 \\
            --workload fe_bcc_40x40x40_nve --steps 20
    Prints one JSON line (training, rates, judge)."""
    import argparse
    import json
    import time
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--frames", type=int, default=2560)
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--workload", default="fe_bcc_40x40x40_nve", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--judge-steps", type=int, default=0)
    ap.add_argument("--save-model", default=None, help="write params and norm to this .npz")
    ap.add_argument("--load-model", default=None, help="skip training: params and norm from this .npz")
    args = ap.parse_args(argv)
    from . import build
    build.build()
    if args.load_model:
        m = np.load(args.load_model)
        params, norm, secs, losses = m["params"], m["norm"], 0.0, [np.full(4, np.nan)]
    else:
        plist, data = training_set(n_frames=args.frames)
        params, norm, losses, secs = train_model(plist, data, epochs=args.epochs)
        del data
        if args.save_model:
            np.savez(args.save_model, params=params, norm=norm)
    p, r, v, s = inputs.workload(args.workload)
    sysm = learned_system(learned_params(p), r, v, s, norm, params)
    sysm.step(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sysm.step(args.steps)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / max(1, args.steps)
    out = {"workload": args.workload, "n_atoms": p["n_atoms"], "learned_ms_per_step": ms,
           "train_seconds": secs, "loss_last": [float(x) for x in losses[-1]], "gate": sysm.ml_gate()}
    sysm.close()
    if args.judge_steps:
        out["judge"] = judge(params, norm, p, r, v, s, args.judge_steps, max(1, args.judge_steps // 10))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
