#!/usr/bin/env python
"""Benchmark of the coupled spin-lattice timestep (arXiv 1801.10233) on GB300.

Default workload: bcc Fe, 64x64x64 cells (524,288 atoms), Morse lattice
potential + Bethe-Slater exchange + 1 T Zeeman field, FP64 state, dt = 0.1 fs,
seeded synthetic inputs.  One bench step = one full timestep of
Eq. general_ST_decomposition (half-kick, 16 colour passes, drift + rebuild
check + exchange table, 16 colour passes, forces + half-kick).

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
DEFAULT_WORKLOAD = "fe_bcc_64x64x64_nve"
# Oracle sample: the same recipe on a 16x16x16-cell box (8,192 atoms); the
# oracle's cost per atom-step does not depend on the box size.
SAMPLE_CELLS = 16

# Algorithmic FP64 work per atom and step of each phase, counting add, mul
# and fma-halves as 1, a square root or division as 10 and an exponential,
# sine or cosine as 20.  Pair terms count each unordered pair once (bcc at
# 6 A: 32 Morse pairs and 7 exchange pairs per atom), although the kernels
# evaluate every pair from both atoms (deterministic per-atom sums without
# atomics); the spin sweep needs all 14 exchange neighbours per update.
MORSE_PAIR_FLOPS = 3 + 5 + 10 + 2 + 20 + 3 + 10 + 6      # dr, r^2, sqrt, arg, exp, V'/r, accumulate
EXCH_FORCE_FLOPS = 5 + 6                                # s_i.s_j, accumulate
JTABLE_PAIR_FLOPS = 3 + 5 + 2 + 20 + 6                  # dr, r^2, x, exp, J
EXCH_DJ_FLOPS = 10 + 5                                  # J'/r from the same exponential (tabulated with J)
ROTATION_FLOPS = 14 * 6 + 3 + 5 + 20 + 20 + 9 + 12 + 6  # field, u, |w|, sincos, A/B, cross, increment
PHASE_FLOPS_PER_ATOM = {
    "kick": 6,
    "spin_half_op_1": 2 * ROTATION_FLOPS,
    "drift_rebuild": 6 + 8,
    "exchange_table": 7 * (JTABLE_PAIR_FLOPS + EXCH_DJ_FLOPS),
    "spin_half_op_2": 2 * ROTATION_FLOPS,
    "force_kick": 32 * MORSE_PAIR_FLOPS + 7 * EXCH_FORCE_FLOPS + 6,
}
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 pipe, nominal at 2070 MHz
# The kernels run the FP64-accurate arithmetic as double-float on the FP32
# pipes: 152 SMs x 128 FP32 lanes x 2.07 GHz = 40.3e12 FP32 instructions/s;
# a double-float multiply-add costs ~20 FP32 instructions (two_prod, two
# corrections, two_sum, renormalisation), so FP64-accurate arithmetic peaks at
# 40.3e12 / 20 x 2 flop = 4.03 TFLOP/s on this chip.
DF_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 20 * 2 / 1e12
# DRAM bytes (read + write) of one launch of each phase's kernel from an ncu
# capture of the current kernels on the 64^3-cell workload
# (profiles/force_fe_bcc_64x64x64_nve.md, profiles/jtable_fe_bcc_64x64x64_nve.md).
NCU_TRAFFIC_64CUBED = {"force_kick": 327.1e6, "exchange_table": 120.6e6}
# DRAM bytes per atom-step of the whole step on the same workload, warm L2
# (ncu --cache-control none, one pass per launch; profiles/dram_per_step_fe_bcc_64x64x64_nve.md)
NCU_DRAM_PER_ATOM_STEP_64CUBED = 2139.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200, help="timed steps (200: the 64^3-cell workload's run)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=["fe_bcc_64x64x64_nve", "fe_bcc_10x10x10_nve", "fe_bcc_100x100x100_nve",
                             "fe_bcc_batch256", "fe_bcc_64x64x64_spin_orbit", "fe_bcc_64x64x64_eam"])
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
         (" + Finnis-Sinclair embedding, ground-state exchange subtracted" if "eam_A_eV" in extra else "")
    return p, r, v, s, (f"bcc Fe {w['ncells']}^3 cells ({p['n_atoms']} atoms), Morse + Bethe-Slater exchange + "
                        f"1 T Zeeman{so}, {w['T']:.0f} K, {w['spins']} spins, NVE, dt 0.1 fs")


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
    p0 = p[0] if isinstance(p, list) else p
    stream = sysm.stream
    # launch shapes from the autotuner (state restored bitwise, outside the timed region)
    if args.launch_shape:
        sv, sb = (int(x) for x in args.launch_shape.split(","))
        sysm.set_launch_shape(sv, sb)
        tune = {"variant": sv, "block": sb, "set_by": "--launch-shape"}
    else:
        tune = None if args.no_autotune else sysm.autotune(3)
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
    dom = max(phases, key=lambda k: phases[k][0])
    dom_ms = phases[dom][0] / max(1, phases[dom][1])
    flops = PHASE_FLOPS_PER_ATOM[dom] * n
    achieved = flops / (dom_ms * 1e-3) / 1e12
    traffic = NCU_TRAFFIC_64CUBED.get(dom) if args.workload == DEFAULT_WORKLOAD else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": DF_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / DF_PEAK_TFLOPS, "traffic": traffic, "kernel": dom,
                "peak_kind": "FP64-accurate (double-float on FP32 pipes) peak derived from unit counts and clock",
                "fp64_pipe_nominal_tflops": FP64_NOMINAL_TFLOPS,
                "phase_ms_per_step": {k: v_[0] / max(1, v_[1]) for k, v_ in phases.items()}}
    hbm = measured_peaks().get("hbm_gbs")
    # compulsory state traffic: r, v, s read and written once per step (144 B/atom)
    if hbm:
        roofline["hbm_frac_state_traffic"] = 144.0 * n / (ms / args.steps * 1e-3) / 1e9 / hbm
    if args.workload == DEFAULT_WORKLOAD:
        # measured DRAM traffic of a whole step (ncu), and its rate at this run's step time
        roofline["dram_bytes_per_atom_step"] = NCU_DRAM_PER_ATOM_STEP_64CUBED
        if hbm:
            roofline["hbm_frac_measured_traffic"] = (NCU_DRAM_PER_ATOM_STEP_64CUBED * n /
                                                     (ms / args.steps * 1e-3) / 1e9 / hbm)

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
        # timed steps as in each workload's run (the batch's 500 and the
        # 2,000-atom system's 1,000), 200 for the spin-orbit and embedding forms
        for name, steps in (("fe_bcc_batch256", 500), ("fe_bcc_10x10x10_nve", 1000),
                            ("fe_bcc_64x64x64_spin_orbit", 200), ("fe_bcc_64x64x64_eam", 200)):
            fp, fr, fv, fs, fdesc = build_workload(name, 0)
            fn = int(sum(q["n_atoms"] for q in fp)) if isinstance(fp, list) else fp["n_atoms"]
            fsys = System(fp, fr, fv, fs, device=dev)
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
                           "phase_ms_per_step": {k: v_[0] / max(1, v_[1]) for k, v_ in fph.items()}}
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
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
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
