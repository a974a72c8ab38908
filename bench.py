#!/usr/bin/env python
"""Benchmark of the coupled spin-lattice timestep (arXiv 1801.10233) on GB300.

Default workload: bcc Fe, 100x100x100 cells (2,000,000 atoms), Morse
lattice potential + Bethe-Slater exchange + 1 T Zeeman field, 300 K, random
spins, FP64 state with double-float pair and rotation arithmetic, dt = 0.1
fs, seeded synthetic inputs.  One bench step = one full timestep of
Eq. general_ST_decomposition (half-kick, 16 colour passes, drift + rebuild
check + exchange table, 16 colour passes, forces + half-kick).  The other
workloads (64^3 cells, 10^3 cells, the replica batch, the spin-orbit and
embedding terms, the learned Hamiltonian) are reported as forms.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.  With torchrun (N > 1) every rank
runs its own replica of the workload (replicas only: no collective on the
data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spin-lattice atom-steps/s on 1 GB300 (plain vs learned/batched) + HBM roofline %"
UNIT = "atom-steps/s"
# The largest single-GPU workload: 100^3 cells, 2,000,000 atoms, 300 K,
# random spins (the 64^3-cell workload is one of the forms).
DEFAULT_WORKLOAD = "fe_bcc_100x100x100_nve"
DEFAULT_STEPS = 1000
# Oracle sample: the same recipe on a 16x16x16-cell box (8,192 atoms); the
# oracle's cost per atom-step does not depend on the box size.
SAMPLE_CELLS = 16

# Algorithmic FP64-equivalent arithmetic per atom-step of each kernel family,
# with the scope table's per-unit estimates (an exponential ~20 ops, a square
# root or division ~10, a sine or cosine ~40, a multiply-add 1; each
# unordered pair once): Morse 32 pairs x ~45, exchange table 7 pairs x ~40,
# spin rotations 4 per atom-step x (14 x 3 multiply-adds + ~60).
KERNEL_OPS_PER_ATOM_STEP = {
    "k_sweep_pass": 4 * (14 * 3 + 60),
    "k_force": 32 * 45,
    "k_jtable": 7 * 40,
    "k_drift": 6,
    "k_kick": 6,
}
# Kernel family of each timed phase; launches per step of each family.
PHASE_KERNEL = {"kick": "k_kick", "spin_half_op_1": "k_sweep_pass", "drift_rebuild": "k_drift",
                "exchange_table": "k_jtable", "spin_half_op_2": "k_sweep_pass", "force_kick": "k_force"}
KERNEL_LAUNCHES_PER_STEP = {"k_sweep_pass": 30, "k_force": 1, "k_jtable": 1, "k_drift": 1, "k_kick": 1}
# What the path computes in: the bench line's dtype is "df64".
ARITH = ("FP64 state (r, v, s, F), FP64 per-atom updates and energy sums; pair and rotation arithmetic "
         "in double-float (unevaluated float pairs, ~48-bit significand, error-free transformations) on the "
         "FP32 pipes, exp to <7e-14 and rsqrt to <5e-14 relative; positions also in 64-bit fixed point for exact "
         "separations")
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 pipe, nominal at 2070 MHz (context only)
# Compulsory state traffic: r, v, s read and written once per step.
STATE_BYTES_PER_ATOM_STEP = 144.0
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of a
# kernel on a workload, from one ncu capture, with a hash of the kernel
# sources it was taken on: a profile whose sources have changed since is
# reported as null (stale), never reused.
PROFILED_DRAM = {
    ("fe_bcc_100x100x100_nve", "k_sweep_pass"): {
        "dram_bytes_per_launch": 172.7e6, "sources_sha": "0258bccf97492cd8",
        "profile": "ncu dram__bytes_read.sum + dram__bytes_write.sum, --cache-control none, mean of 2 launches "
                   "of k_sweep_pass<16, 128, 0, 1024> (launch shape 3,128) inside 3-step runs"},
    ("fe_bcc_100x100x100_nve", "k_force"): {
        "dram_bytes_per_launch": 2415.1e6, "sources_sha": "0258bccf97492cd8",
        "profile": "ncu dram__bytes_read.sum + dram__bytes_write.sum, --cache-control none, mean of 2 launches "
                   "of k_force<0, 0> (launch shape 3,128) inside 3-step runs"},
}
PROFILED_SOURCES = ("sl_step.cu", "sl_sweep.cuh", "sl_sweep.cu", "sl_sweep_so.cu", "sl_pair.cuh", "sl_df64.cuh",
                    "sl_internal.cuh", "sl_build.cu", "sl_api.cu")


def kernel_sources_sha():
    """sha256 (16 hex digits) of the kernel sources a profile depends on."""
    import hashlib
    h = hashlib.sha256()
    for name in PROFILED_SOURCES:
        with open(os.path.join(ROOT, "paper_1801_10233_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled(workload, kernel):
    """The current profile entry of (workload, kernel), or None if absent or stale."""
    e = PROFILED_DRAM.get((workload, kernel))
    return e if e and e.get("sources_sha") == kernel_sources_sha() else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=DEFAULT_STEPS, help="timed steps (1000: the 100^3-cell workload's run)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=["fe_bcc_64x64x64_nve", "fe_bcc_10x10x10_nve", "fe_bcc_100x100x100_nve",
                             "fe_bcc_batch256", "fe_bcc_64x64x64_spin_orbit", "fe_bcc_64x64x64_eam",
                             "fe_bcc_64x64x64_eam_tab"])
    ap.add_argument("--no-forms", action="store_true", help="skip the extra per-form measurements")
    ap.add_argument("--no-learned", action="store_true", help="skip training and judging the learned Hamiltonian")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--launch-shape", default=None, help="VARIANT,BLOCK: set the headline's launch shape "
                    "instead of autotuning it (to profile a known shape)")
    ap.add_argument("--learned-frames", type=int, default=20000, help="training snapshots (10^3-cell frames)")
    ap.add_argument("--learned-epochs", type=int, default=4)
    ap.add_argument("--learned-steps", type=int, default=500, help="judged steps on 40^3 cells")
    ap.add_argument("--learned-big-steps", type=int, default=1000, help="judged steps on 100^3 cells")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--full-workload", action="store_true",
                    help="with --impl reference: time the oracle on the whole workload instead of the sample")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, world, device):
    """The largest of every rank's value x (float), all ranks receive it."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(atoms_per_rank, world, steps, seconds):
    """Atom-steps per second of the whole job: every rank advanced
    atoms_per_rank atoms by `steps` steps; `seconds` is the slowest rank's time."""
    return world * atoms_per_rank * steps / seconds


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def oracle_sample(seed_offset=0):
    from paper_1801_10233_gb300 import inputs
    w = inputs.WORKLOADS[DEFAULT_WORKLOAD]
    return inputs.bcc_fe_system(SAMPLE_CELLS, w["seed"] + seed_offset, T=w["T"], spins=w["spins"])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def time_oracle(steps, warmup, threads=1, system=None):
    """Atom-steps/s of the CPU oracle on the bounded sample (or on system =
    (params, r, v, s)); with threads > 1 same-colour sectors and per-atom sums
    are split over OpenMP threads (results bit-identical to one thread).
    Returns (rate, seconds, atoms, threads used)."""
    import oracle
    p, r, v, s = system if system is not None else oracle_sample()
    o = oracle.Oracle(p, r, v, s, threads=threads)
    o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return p["n_atoms"] * steps / dt, dt, p["n_atoms"], o.threads


def cpu_desc():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def build_workload(name, rank=0):
    """(params or params list, r, v, s, description) of a named workload;
    rank shifts the seeds so replicas on different GPUs differ."""
    from paper_1801_10233_gb300 import inputs
    if name == "fe_bcc_batch256":
        p, r, v, s = inputs.batch_workload(256, seed=18012 + 1000 * rank)
        return p, r, v, s, ("256 bcc-Fe replicas, sizes drawn from {8,12,16,20,24}^3 cells, Langevin spin "
                            "bath 50..1200 K (lambda 0.01), lattice NVE, dt 0.1 fs, one batched context")
    w = inputs.WORKLOADS[name]
    p, r, v, s = inputs.bcc_fe_system(w["ncells"], w["seed"] + rank, T=w["T"], spins=w["spins"],
                                      **w.get("params", {}))
    extra = w.get("params", {})
    so = (" + uniaxial anisotropy, Neel and DMI terms" if "aniso_K_eV" in extra else "") + \
         (" + Finnis-Sinclair embedding, ground-state exchange subtracted" if "eam_A_eV" in extra else "") + \
         (" with the Morse pairs replaced by a tabulated embedded-atom potential (synthetic tables, natural "
          "cubic splines), ground-state exchange subtracted" if extra.get("eam_tabulated") else "")
    return p, r, v, s, (f"bcc Fe {w['ncells']}^3 cells ({p['n_atoms']} atoms), Morse + Bethe-Slater exchange + "
                        f"1 T Zeeman{so}, {w['T']:.0f} K, {w['spins']} spins, NVE, dt 0.1 fs")


def prepare(sysm, name):
    """Per-workload set-up after the context exists: the tabulated
    embedded-atom workload gets its (synthetic) tables."""
    if name.endswith("_eam_tab"):
        from paper_1801_10233_gb300 import inputs
        sysm.set_eam_tables(*inputs.eam_tables())


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    steps, warmup = max(1, args.steps), max(0, args.warmup)
    if args.full_workload:
        if args.workload == "fe_bcc_batch256":
            print(json.dumps({"impl": "reference", "unavailable": "--full-workload times one system, "
                              "not a replica batch"}))
            return
        p, r, v, s, desc = build_workload(args.workload)
        t0 = time.perf_counter()
        val, secs, n, nt = time_oracle(steps, warmup, host_cores(), (p, r, v, s))
        total = time.perf_counter() - t0
        sample = (f"{steps} timesteps of the whole workload ({desc}) after the initial lists and forces "
                  f"and {warmup} untimed steps ({total - secs:.1f} s together); CPU oracle, {nt} OpenMP "
                  f"threads ({cpu_desc()})")
    else:
        val, secs, n, nt = time_oracle(steps, warmup, host_cores())
        sample = (f"{steps} timesteps of a {SAMPLE_CELLS}^3-cell ({n}-atom) bcc-Fe box built by the workload's "
                  f"recipe, after {warmup} untimed steps; CPU oracle, {nt} OpenMP threads ({cpu_desc()})")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * secs / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample_atoms": n},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _rate(sysm, steps, torch):
    """atom-steps/s and ms/step of `steps` timed steps (CUDA events, 3 warm-up steps)."""
    sysm.step(3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sysm.stream)
    sysm.step(steps)
    e1.record(sysm.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return sysm.n / (ms * 1e-3), ms


def learned_forms(args, dev, torch):
    """Train the learned Hamiltonian on snapshots of analytic trajectories,
    then run it beside the analytic Hamiltonian on the 40^3- and 100^3-cell
    workloads: rates of both, the gain, and the judge's error report."""
    from paper_1801_10233_gb300 import System, inputs, learned
    t0 = time.perf_counter()
    plist, data = learned.training_set(n_frames=args.learned_frames, n_replicas=64, every=10, device=dev)
    torch.cuda.synchronize()
    t_snap = time.perf_counter() - t0
    params, norm, losses, secs = learned.train_model(plist, data, epochs=args.learned_epochs, device=dev)
    atoms = int(data["r"].shape[1])
    out = {"training": {"frames": int(data["r"].shape[0]) * len(plist), "frame_atoms": 2000,
                        "epochs": args.learned_epochs, "adam_steps": len(losses), "seconds": secs,
                        "snapshot_seconds": t_snap, "atoms_per_s": len(losses) * atoms / secs,
                        "loss_first": [float(x) for x in losses[0]], "loss_last": [float(x) for x in losses[-1]],
                        "loss_terms": "L, energy, force, omega"}}
    del data
    torch.cuda.empty_cache()
    for name, steps, every in (("fe_bcc_40x40x40_nve", args.learned_steps, 50),
                               ("fe_bcc_100x100x100_nve", args.learned_big_steps, 100)):
        if steps <= 0:
            continue
        p, r, v, s = inputs.workload(name)
        judge = learned.judge(params, norm, p, r, v, s, steps, every, device=dev)
        plain = System(p, r, v, s, device=dev)
        rp, mp = _rate(plain, 20, torch)
        plain.close()
        lsys = learned.learned_system(learned.learned_params(p), r, v, s, norm, params, device=dev)
        rl, ml = _rate(lsys, 20, torch)
        lsys.set_timing(True)
        lsys.step(5)
        ph = lsys.timing()
        lsys.set_timing(False)
        kp = lsys.counters()["kernels_per_step"]
        lsys.close()
        out[name] = {"n_atoms": p["n_atoms"], "plain": {"value": rp, "ms_per_step": mp},
                     "learned": {"value": rl, "ms_per_step": ml, "kernels_per_step": kp,
                                 "phase_ms_per_step": {k: v_[0] / max(1, v_[1]) for k, v_ in ph.items()}},
                     "gain_learned_over_plain": rl / rp, "unit": UNIT, "judge": judge}
        torch.cuda.empty_cache()
    return out


def df_peak_tflops():
    """Measured double-float multiply-add throughput of this GPU (TFLOP/s,
    2 flop per multiply-add), from the library's own probe kernel."""
    from paper_1801_10233_gb300 import _lib
    f, _ = _lib.df_fma_rate(4096)
    return f / 1e12


def kernel_roofline(phases, n, workload, step_s_ms, peak=None):
    """Roofline entry of the kernel family with the most device time per
    step: achieved = its algorithmic ops per atom-step x atoms / its time per
    step (the same per launch), against the measured double-float peak."""
    per_kernel = {}
    for ph, (tot, cnt) in phases.items():
        k = PHASE_KERNEL[ph]
        per_kernel[k] = per_kernel.get(k, 0.0) + tot / max(1, cnt)
    dom = max((k for k in per_kernel if k in KERNEL_OPS_PER_ATOM_STEP), key=lambda k: per_kernel[k])
    t = per_kernel[dom] * 1e-3
    peak = peak if peak is not None else df_peak_tflops()
    achieved = KERNEL_OPS_PER_ATOM_STEP[dom] * n / t / 1e12
    launches = KERNEL_LAUNCHES_PER_STEP[dom]
    prof = profiled(workload, dom)
    traffic = prof["dram_bytes_per_launch"] if prof else None
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": traffic, "kernel": dom, "launches_per_step": launches,
           "ms_per_launch": per_kernel[dom] / launches, "ops_per_atom_step": KERNEL_OPS_PER_ATOM_STEP[dom],
           "peak_kind": "measured: double-float multiply-add throughput of the library's probe kernel "
                        "(sl_df_fma_rate, 2 flop each), this GPU, this run",
           "fp64_pipe_nominal_tflops": FP64_NOMINAL_TFLOPS,
           "kernel_ms_per_step": per_kernel,
           "phase_ms_per_step": {k: v_[0] / max(1, v_[1]) for k, v_ in phases.items()}}
    hbm = measured_peaks().get("hbm_gbs")
    if hbm:
        out["hbm_peak_gbs"] = hbm
        out["hbm_frac_state_traffic"] = STATE_BYTES_PER_ATOM_STEP * n / (step_s_ms * 1e-3) / 1e9 / hbm
    if traffic:
        out["traffic_profile"] = prof["profile"]
        out["hbm_frac_kernel_traffic"] = traffic / (out["ms_per_launch"] * 1e-3) / 1e9 / hbm if hbm else None
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        from paper_1801_10233_gb300.build import build
        build()
    if world > 1:
        dist.barrier()
    from paper_1801_10233_gb300 import System, inputs

    # every rank runs its own replica (different seed)
    p, r, v, s, wdesc = build_workload(args.workload, rank)
    n = int(sum(q["n_atoms"] for q in p)) if isinstance(p, list) else p["n_atoms"]
    sysm = System(p, r, v, s, device=dev)
    prepare(sysm, args.workload)
    p0 = p[0] if isinstance(p, list) else p
    stream = sysm.stream
    # launch shapes from the autotuner (state restored bitwise, outside the timed region)
    if args.launch_shape:
        sv, sb = (int(x) for x in args.launch_shape.split(","))
        sysm.set_launch_shape(sv, sb)
        tune = {"variant": sv, "block": sb, "set_by": "--launch-shape"}
    else:
        tune = None if args.no_autotune else sysm.autotune(3)
    # the compute roof of the double-float kernels, measured on this GPU
    # before the timed region (the probe kernel runs ~10 ms)
    peak = df_peak_tflops()
    sysm.step(args.warmup)
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sysm.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    value = whole_job_rate(n, world, args.steps, ms * 1e-3)
    counters = sysm.counters()
    launches = counters["kernels_per_step"] * args.steps

    # live per-phase timing (CUDA events on the library's stream, same steps)
    sysm.set_timing(True)
    tsteps = max(3, min(args.steps, 20))
    sysm.step(tsteps)
    phases = sysm.timing()
    sysm.set_timing(False)
    roofline = kernel_roofline(phases, n, args.workload, ms / args.steps, peak)

    # end to end through the public API with host buffers: per step, upload the
    # state from pinned memory, advance one step, read the state back
    hr = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    hv, hs = torch.empty_like(hr).pin_memory(), torch.empty_like(hr).pin_memory()
    sysm.state_host(hr, hv, hs)
    esteps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(esteps):
        sysm.set_state_host(hr, hv, hs)
        sysm.step(1)
        sysm.state_host(hr, hv, hs)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e = {"value": whole_job_rate(n, world, esteps, e2e_s), "unit": UNIT, "h2d_bytes_per_step": 3 * n * 3 * 8,
           "d2h_bytes_per_step": 3 * n * 3 * 8, "steps": esteps}

    forms = None
    if rank == 0 and world == 1 and not args.no_forms and args.workload == DEFAULT_WORKLOAD:
        forms = {}
        # timed steps as in each workload's run (the 64^3-cell system's 200,
        # the batch's 500 and the 2,000-atom system's 1,000), 200 for the
        # spin-orbit and embedding forms
        for name, steps in (("fe_bcc_64x64x64_nve", 200), ("fe_bcc_batch256", 500), ("fe_bcc_10x10x10_nve", 1000),
                            ("fe_bcc_64x64x64_spin_orbit", 200), ("fe_bcc_64x64x64_eam", 200),
                            ("fe_bcc_64x64x64_eam_tab", 200)):
            fp, fr, fv, fs, fdesc = build_workload(name, 0)
            fn = int(sum(q["n_atoms"] for q in fp)) if isinstance(fp, list) else fp["n_atoms"]
            fsys = System(fp, fr, fv, fs, device=dev)
            prepare(fsys, name)
            ftune = None if args.no_autotune else fsys.autotune(2)
            fsys.step(3)
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(fsys.stream)
            fsys.step(steps)
            f1.record(fsys.stream)
            torch.cuda.synchronize()
            fms = f0.elapsed_time(f1) / steps
            fsys.set_timing(True)
            fsys.step(5)
            fph = fsys.timing()
            fsys.set_timing(False)
            forms[name] = {"value": fn / (fms * 1e-3), "unit": UNIT, "ms_per_step": fms, "steps": steps,
                           "n_atoms": fn, "workload": fdesc, "launch_shape": ftune,
                           "roofline": kernel_roofline(fph, fn, name, fms, peak)}
            fsys.close()
            del fsys
        if not args.no_learned:
            forms["learned"] = learned_forms(args, dev, torch)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ost, ost1 = 1000, 40
        val, secs, ns, nt = time_oracle(ost, 1, host_cores())
        val1, secs1, _, _ = time_oracle(ost1, 1, 1)
        cpu = {"value": val, "unit": UNIT, "cores": nt, "kind": "oracle",
               "sample": f"{ost} timesteps of a {SAMPLE_CELLS}^3-cell ({ns}-atom) box of the same recipe "
                         f"({secs:.1f} s, {nt} OpenMP threads, {cpu_desc()}; same-colour sectors and "
                         f"per-atom sums split over threads, results bit-identical to one thread)",
               "serial": {"value": val1, "unit": UNIT, "cores": 1,
                          "sample": f"{ost1} timesteps of the same box on one thread ({secs1:.1f} s)"}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "df64", "data": "synthetic",
            "arith": ARITH,
            "config": {"workload": args.workload, "description": wdesc, "n_atoms": n, "dt_ps": p0["dt_ps"],
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "working set > 129 MB L2 (no flush needed)", "graph": counters["graph"],
                       "launch_shape": tune},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches, "forms": forms,
        }
        print(json.dumps(line))
    sysm.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
