"""Seeded synthetic inputs for the coupled spin-lattice timestep.

This module only *generates* inputs: a bcc lattice with Gaussian
displacements, Maxwell-Boltzmann velocities and unit spins, plus the
parameter set of the bcc-Fe / Morse / Bethe-Slater workload.  It holds none
of the method's arithmetic and is the one module shared by the CUDA path's
callers and the CPU oracle's tests.

Units are the paper's "metal" set: Angstrom, ps, eV, amu, K, Tesla.
"""
from __future__ import annotations

import math

import numpy as np

# Used only to draw Maxwell-Boltzmann velocities here.
_KB_EV_PER_K = 8.617333262e-5
_EV_PER_A_AMU_TO_A_PER_PS2 = 9648.533212

LATTICE_A = 2.8665          # bcc Fe lattice constant, Angstrom
MASS_FE = 55.845            # amu


def fe_params(box, n_atoms, **overrides):
    """Parameter dict of the bcc-Fe workload (Morse lattice potential,
    Bethe-Slater exchange of Eq. BSfunction, Zeeman field 1 T along z,
    mu = 2.2 mu_B, dt = 0.1 fs).  Keys match the C-ABI struct fields."""
    p = dict(
        n_atoms=int(n_atoms),
        box=[float(b) for b in box],
        mass_amu=MASS_FE,
        mu_s_muB=2.2,
        H_tesla=[0.0, 0.0, 1.0],
        dt_ps=1.0e-4,
        ex_alpha_eV=0.02726,
        ex_gamma=0.2171,
        ex_delta_A=1.841,
        ex_rc_A=3.4,
        morse_D0_eV=0.4174,
        morse_alpha_invA=1.3885,
        morse_r0_A=2.845,
        morse_rc_A=6.0,
        skin_A=0.3,
        rotation=0,
        fix_lattice=0,
        rebuild_every=0,
        morse_shift_energy=1,
        hamiltonian=0,
        lattice_gamma_ps=0.0,
        lattice_temperature_K=0.0,
        aniso_K_eV=0.0,
        aniso_axis=[0.0, 0.0, 1.0],
        neel_alpha_eV=0.0,
        neel_gamma=0.0,
        neel_delta_A=1.841,
        dmi_alpha_eV=0.0,
        dmi_gamma=0.0,
        dmi_delta_A=1.841,
        eam_A_eV=0.0,
        eam_d_A=3.569745,
        eam_beta=1.8,
        subtract_ground_exchange=0,
        eam_tabulated=0,
        max_ex_neighbors=0,
        max_morse_neighbors=0,
    )
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p


def bcc_positions(ncells, a=LATTICE_A):
    """Perfect bcc lattice of nx*ny*nz cubic cells (2 atoms each); ncells is
    an int (cube) or a triple.  Atom id = 2 * (ix + nx*(iy + ny*iz)) + basis."""
    nx, ny, nz = (int(ncells),) * 3 if np.isscalar(ncells) else tuple(int(c) for c in ncells)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    # order: iz slowest, then iy, then ix, then basis
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    base = np.repeat(cells, 2, axis=0)
    base[1::2] += 0.5
    return base * a, np.array([nx * a, ny * a, nz * a], dtype=np.float64)


def unit_spins_uniform(rng, n):
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    s = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)
    return s / np.linalg.norm(s, axis=1, keepdims=True)


def unit_spins_cone(rng, n, sigma_deg=10.0):
    """Ferromagnetic along +z, each spin tilted by |N(0, sigma^2)| with a
    uniform azimuth."""
    th = np.abs(rng.normal(0.0, math.radians(sigma_deg), n))
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.stack([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)], axis=1)
    return s / np.linalg.norm(s, axis=1, keepdims=True)


def maxwell_boltzmann(rng, n, T, mass=MASS_FE):
    """Velocities (A/ps) drawn from N(0, k_B T / m), centre-of-mass motion
    removed, rescaled so the kinetic temperature with 3N-3 degrees of
    freedom is exactly T (zero for T = 0 or n < 2)."""
    if T <= 0.0 or n < 2:
        return np.zeros((n, 3))
    sig = math.sqrt(_KB_EV_PER_K * T / mass * _EV_PER_A_AMU_TO_A_PER_PS2)
    v = rng.normal(0.0, sig, (n, 3))
    v -= v.mean(axis=0, keepdims=True)
    ek = 0.5 * mass * float((v * v).sum()) / _EV_PER_A_AMU_TO_A_PER_PS2
    t_now = 2.0 * ek / ((3 * n - 3) * _KB_EV_PER_K)
    return v * math.sqrt(T / t_now)


def bcc_fe_system(ncells, seed, T=200.0, sigma=0.01, spins="uniform", a=LATTICE_A, **param_overrides):
    """A seeded bcc-Fe system: returns (params, r, v, s), arrays [N, 3] float64."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    r, box = bcc_positions(ncells, a)
    n = r.shape[0]
    r = r + rng.normal(0.0, sigma, r.shape) if sigma > 0 else r
    v = maxwell_boltzmann(rng, n, T)
    if spins == "uniform":
        s = unit_spins_uniform(rng, n)
    elif spins.startswith("cone"):
        s = unit_spins_cone(rng, n, float(spins[4:] or 10.0))
    elif spins == "fm":
        s = np.tile(np.array([0.0, 0.0, 1.0]), (n, 1))
    else:
        raise ValueError(spins)
    return fe_params(box, n, **param_overrides), np.ascontiguousarray(r), np.ascontiguousarray(v), np.ascontiguousarray(s)


# Spin-orbit terms of the 64^3-cell spin-orbit workload (App. A.2): uniaxial
# anisotropy along z, Neel pseudo-dipolar and DMI pair terms of the
# Eq. BSfunction form, a few per cent of the exchange.  Chosen to exercise
# and time the terms, not fitted to a material.
SPIN_ORBIT = dict(aniso_K_eV=1e-4, aniso_axis=[0.0, 0.0, 1.0], neel_alpha_eV=1e-3, neel_gamma=0.1,
                  neel_delta_A=1.7, dmi_alpha_eV=1e-3, dmi_gamma=0.3, dmi_delta_A=1.9)

# Embedding term of the 64^3-cell embedded-atom workload (App. B): the
# Finnis-Sinclair form F(rho) = -A sqrt(rho), f(r) = (r - d)^2 + beta (r - d)^3/d
# on top of the Morse pairs, with the collinear magnetic ground state
# subtracted (Eq. app:mech1).  d = 3.4 A (the exchange cutoff) takes the
# first two bcc shells; A and beta are chosen to exercise and time the
# terms, not fitted.
EMBEDDING = dict(eam_A_eV=0.5, eam_d_A=3.4, eam_beta=1.8, subtract_ground_exchange=1)

# Tabulated embedded-atom workload (App. B): the paper's potential comes as
# tables of F(rho), rho(r) and phi(r); the Pun-Mishin tables are not
# available here, so synthetic tables of smooth stand-in functions take their
# place (eam_tables below).
EMBEDDING_TABULATED = dict(eam_tabulated=1, subtract_ground_exchange=1)


def eam_tables(nr=2003, dr=0.003, nrho=2001, drho=0.01, A=0.5, d=3.4, beta=1.8, shifted_force=True,
               D0=0.4174, alpha=1.3885, r0=2.845, rc=6.0, cut=True):
    """Synthetic tables for the tabulated embedded-atom form: (F, drho, rho,
    phi, dr), F on rho = k drho (nrho points), rho(r) and phi(r) on r = k dr
    (nr points, reaching past rc).  Stand-in shapes, not a fitted potential:
    F(rho) = -A sqrt(rho); rho(r) = (r - d)^2 + beta (r - d)^3 / d below d, 0
    beyond; phi(r) the Morse pair energy D0 (e^{-2a(r-r0)} - 2 e^{-a(r-r0)}),
    by default shifted in value and slope to vanish at rc and 0 beyond (with
    cut = False the Morse form continues past rc)."""
    r = np.arange(nr) * dr
    x = r - d
    rho = np.where(r < d, x * x + beta * x ** 3 / d, 0.0)
    def morse(y):
        e = np.exp(-alpha * (y - r0))
        return D0 * (e * e - 2.0 * e)
    def dmorse(y):
        e = np.exp(-alpha * (y - r0))
        return D0 * (-2.0 * alpha * e * e + 2.0 * alpha * e)
    phi = morse(r)
    if shifted_force:
        phi = phi - morse(rc) - (r - rc) * dmorse(rc)
    if cut:
        phi = np.where(r < rc, phi, 0.0)
    F = -A * np.sqrt(np.arange(nrho) * drho)
    return F, drho, rho, phi, dr


# The workloads: plain 10^3 cells, plain 64^3 cells, 256 batched
# replicas, learned 40^3 cells, large 100^3 cells, 64^3 cells with the
# spin-orbit terms, 64^3 cells with the embedding term in the Finnis-Sinclair
# and in the tabulated form.
WORKLOADS = {
    "fe_bcc_10x10x10_nve": dict(ncells=10, seed=18010, T=200.0, spins="uniform", steps=1000),
    "fe_bcc_64x64x64_nve": dict(ncells=64, seed=18011, T=200.0, spins="cone10", steps=200),
    "fe_bcc_40x40x40_nve": dict(ncells=40, seed=18013, T=200.0, spins="uniform", steps=500),
    "fe_bcc_100x100x100_nve": dict(ncells=100, seed=18014, T=300.0, spins="uniform", steps=1000),
    "fe_bcc_64x64x64_spin_orbit": dict(ncells=64, seed=18017, T=200.0, spins="cone10", steps=200,
                                       params=SPIN_ORBIT),
    "fe_bcc_64x64x64_eam": dict(ncells=64, seed=18018, T=200.0, spins="cone10", steps=200, params=EMBEDDING),
    "fe_bcc_64x64x64_eam_tab": dict(ncells=64, seed=18019, T=200.0, spins="cone10", steps=200,
                                    params=EMBEDDING_TABULATED),
}


def workload(name, **param_overrides):
    w = WORKLOADS[name]
    kw = dict(w.get("params", {}), **param_overrides)
    return bcc_fe_system(w["ncells"], w["seed"], T=w["T"], spins=w["spins"], **kw)


def replica_batch(n_replicas=256, seed=18012, cell_choices=(8, 12, 16, 20, 24), t_lo=50.0, t_hi=1200.0):
    """Sizes and temperatures of the batched-replica workload: replica k has
    ncells drawn by seed from cell_choices and temperature evenly spaced in
    [t_lo, t_hi]."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    cells = rng.choice(np.asarray(cell_choices), size=n_replicas)
    temps = t_lo + np.arange(n_replicas) * (t_hi - t_lo) / max(1, n_replicas - 1)
    return [int(c) for c in cells], [float(t) for t in temps]


def replica_systems(cells, temps, seed, lam=0.01, **param_overrides):
    """A batch of bcc-Fe replicas: replica k has cells[k]^3 cells, Maxwell-
    Boltzmann velocities and a spin bath at temps[k], uniform spins, noise
    counter word k.  Returns (params list, r, v, s) with the atoms of all
    replicas back to back."""
    plist, rs, vs, ss = [], [], [], []
    for k, (nc, T) in enumerate(zip(cells, temps)):
        p, r, v, s = bcc_fe_system(nc, int(seed) * 1000 + k, T=T, spins="uniform", **param_overrides)
        p.update({"lambda": float(lam), "temperature_K": float(T), "seed": int(seed), "replica": k})
        plist.append(p)
        rs.append(r); vs.append(v); ss.append(s)
    return plist, np.concatenate(rs), np.concatenate(vs), np.concatenate(ss)


def batch_workload(n_replicas=256, seed=18012, **param_overrides):
    """The batched workload: n_replicas replicas with sizes drawn by seed from
    {8, 12, 16, 20, 24}^3 cells and bath temperatures 50..1200 K, lambda 0.01."""
    cells, temps = replica_batch(n_replicas, seed)
    return replica_systems(cells, temps, seed, **param_overrides)


# ---------------------------------------------------------------------------
# Learned per-atom Hamiltonian: initial weights (random draws only)
# ---------------------------------------------------------------------------
def ml_init_params(seed, n_in=48, n_hidden=64, e0=0.0):
    """Seeded initial parameters of the 48 -> 64 -> 64 -> 1 network as one
    float32 vector in the order W1[n_hidden][n_in], b1, W2[n_hidden][n_hidden],
    b2, w3[n_hidden], b3.  Weights uniform in +-sqrt(6/(fan_in+fan_out))
    (Glorot and Bengio, 2010), the output layer scaled by 0.1, biases zero
    except b3 = e0."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))

    def glorot(fo, fi, scale=1.0):
        b = scale * math.sqrt(6.0 / (fi + fo))
        return rng.uniform(-b, b, size=(fo, fi))

    parts = [glorot(n_hidden, n_in).ravel(), np.zeros(n_hidden), glorot(n_hidden, n_hidden).ravel(),
             np.zeros(n_hidden), glorot(1, n_hidden, 0.1).ravel(), np.array([e0])]
    return np.concatenate(parts).astype(np.float32)


def training_replicas(n_replicas=64, seed=18015, ncells=10, t_lo=50.0, t_hi=1200.0, lam=0.01):
    """Replicas whose trajectories give the learned model's training
    snapshots: ncells^3-cell bcc Fe at bath temperatures evenly spaced in
    [t_lo, t_hi] (lattice Maxwell-Boltzmann at the same T), spin baths with
    damping lam, and three spin starts in turn: uniform on the sphere, 10 deg
    cones about +z, and cones whose width grows with T (10..90 deg)."""
    plist, rs, vs, ss = [], [], [], []
    for k in range(n_replicas):
        T = t_lo + k * (t_hi - t_lo) / max(1, n_replicas - 1)
        kind = k % 3
        spins = "uniform" if kind == 0 else ("cone10" if kind == 1 else f"cone{10.0 + 80.0 * (T - t_lo) / (t_hi - t_lo)}")
        p, r, v, s = bcc_fe_system(ncells, int(seed) * 1000 + k, T=T, sigma=0.02, spins=spins)
        p.update({"lambda": float(lam), "temperature_K": float(T), "seed": int(seed), "replica": k})
        plist.append(p)
        rs.append(r); vs.append(v); ss.append(s)
    return plist, np.concatenate(rs), np.concatenate(vs), np.concatenate(ss)
