"""Spin-lattice relaxation with one thermostat at a time (the two-thermostat
experiment of Sec. 4.2, on the bcc-Fe / Morse / Bethe-Slater Hamiltonian).

Run A: the spin bath (Eq. s_advance_T, lambda = 0.01) at T, lattice at rest on
perfect bcc sites (T_L = 0), spins drawn from a T magnetic equilibrium (a
spin-only run with the bath on a frozen lattice).  Run B: the lattice bath
(Eq. p_advance_T) at T, spins within 2-degree cones about the field (T_S of a
few K), velocities from a Maxwell-Boltzmann distribution at T.  (Spins
exactly along the field would never move: with isotropic exchange and the
field along z the collinear state feels no torque however the lattice moves;
the paper's cobalt model breaks that symmetry with spin-orbit terms.)  Each run records T_L and T_S
(Eqs. lattice_temperature, spin_temperature): the unthermostatted part heats
up through the spin-lattice coupling.

    python -m paper_1801_10233_gb300.relax --cells 10 --ps 20 --dt 0.0005
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import inputs
from .system import System


def _series(sysm, steps, every, dt):
    ts, tl, tsp = [], [], []
    for k in range(0, steps + 1, every):
        if k:
            sysm.step(every)
        e = sysm.energy()
        ts.append(k * dt)
        tl.append(float(e[5]))
        tsp.append(float(e[6]))
    return ts, tl, tsp


def _tau(ts, temps, target):
    """Time at which the heated part first reaches 1 - 1/e of the target."""
    for t, x in zip(ts, temps):
        if x >= (1.0 - math.exp(-1.0)) * target:
            return t
    return None


def run(cells=10, T=300.0, ps=20.0, dt=5e-4, every=None, gamma=10.0, lam=0.01, prep_ps=2.0, seed=18016,
        device=None, extra=None):
    """Both runs; returns a dict of their T_L and T_S series and e-folding times.
    `extra`: further Hamiltonian parameters for both runs (for instance the
    Neel pair term, which lets lattice motion torque collinear spins)."""
    extra = dict(extra or {})
    steps = int(round(ps / dt))
    every = every or max(1, steps // 100)
    out = {"cells": cells, "T_K": T, "dt_ps": dt, "ps": ps, "lambda": lam, "lattice_gamma_ps": gamma,
           "extra": extra}

    # run A: spin bath only; spins first equilibrated at T on the frozen perfect lattice
    p, r, v, s = inputs.bcc_fe_system(cells, seed, T=T, sigma=0.0, spins="uniform", dt_ps=dt, **extra)
    pa = dict(p, **{"lambda": lam, "temperature_K": T, "seed": seed})
    prep = System(dict(pa, fix_lattice=1), r, np.zeros_like(v), s, device=device)
    prep.step(int(round(prep_ps / dt)))
    _, _, s_eq = prep.state()
    prep.close()
    a = System(pa, r, np.zeros_like(v), s_eq, device=device)
    t0 = time.perf_counter()
    ts, tl, tsp = _series(a, steps, every, dt)
    a.close()
    out["spin_bath"] = {"t_ps": ts, "T_L": tl, "T_S": tsp, "tau_L_ps": _tau(ts, tl, T)}

    # run B: lattice bath only; spins within 2-degree cones about the field
    p, r, v, s = inputs.bcc_fe_system(cells, seed + 1, T=T, sigma=0.0, spins="cone2", dt_ps=dt, **extra)
    pb = dict(p, lattice_gamma_ps=gamma, lattice_temperature_K=T, seed=seed + 1)
    b = System(pb, r, v, s, device=device)
    ts, tl, tsp = _series(b, steps, every, dt)
    b.close()
    out["lattice_bath"] = {"t_ps": ts, "T_L": tl, "T_S": tsp, "tau_S_ps": _tau(ts, tsp, T)}
    torch.cuda.synchronize()
    out["seconds"] = time.perf_counter() - t0
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--cells", type=int, default=10)
    ap.add_argument("--T", type=float, default=300.0)
    ap.add_argument("--ps", type=float, default=20.0)
    ap.add_argument("--dt", type=float, default=5e-4)
    ap.add_argument("--gamma", type=float, default=10.0, help="lattice damping rate gamma_L/m, 1/ps")
    ap.add_argument("--lam", type=float, default=0.01)
    ap.add_argument("--neel", type=float, default=0.0,
                    help="Neel pair term alpha in eV (gamma 0.1, delta 1.7 A; 0: none)")
    args = ap.parse_args(argv)
    extra = dict(neel_alpha_eV=args.neel, neel_gamma=0.1, neel_delta_A=1.7) if args.neel else None
    from . import build
    build.build()
    print(json.dumps(run(args.cells, args.T, args.ps, args.dt, gamma=args.gamma, lam=args.lam, extra=extra)))


if __name__ == "__main__":
    main()
