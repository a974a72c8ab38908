"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle (oracle/sl_oracle.c) against something other than
itself: a closed-form solution, a lattice sum from bcc geometry, a finite
difference of an independently coded energy, an invariant of the exact
dynamics, or a published known-answer vector.  None needs a GPU.
"""
import math
import os

import numpy as np
import pytest

from paper_1801_10233_gb300 import inputs

HBAR = 6.582119569e-4      # eV ps (CODATA 2018)
MUB = 5.7883818060e-5      # eV / T (CODATA 2018)
KB = 8.617333262e-5        # eV / K (CODATA 2018)
FTOA = 9648.533212         # (eV / A) / amu in A / ps^2
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def J_bs(p, r):
    """Eq. BSfunction (App. A.1), below the cutoff."""
    x = (r / p["ex_delta_A"]) ** 2
    return 4 * p["ex_alpha_eV"] * x * (1 - p["ex_gamma"] * x) * math.exp(-x)


def V_morse(p, r):
    e = math.exp(-p["morse_alpha_invA"] * (r - p["morse_r0_A"]))
    return p["morse_D0_eV"] * (e * e - 2 * e)


def two_atoms(d, box=20.0, **kw):
    r = np.array([[8.0, 10.0, 10.0], [8.0 + d, 10.0, 10.0]])
    p = inputs.fe_params([box] * 3, 2, **kw)
    return p, r


# --------------------------------------------------------------------------
# Counter-based generator
# --------------------------------------------------------------------------
def test_philox_known_answers(orc):
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for row in rows:
        assert orc.philox4x32_10(row[0:4], row[4:6]) == row[6:10]


def test_gaussian_moments(orc):
    g = np.array([orc.gauss3(1234, 7, st, sp, a) for st in range(20) for sp in range(4) for a in range(100)])
    assert g.shape == (8000, 3)
    assert abs(g.mean()) < 0.03
    assert abs(g.var() - 1.0) < 0.04
    # distinct sub-passes give distinct draws
    assert not np.allclose(orc.gauss3(1, 0, 5, 0, 3), orc.gauss3(1, 0, 5, 1, 3))


# --------------------------------------------------------------------------
# Single spin in a Zeeman field: exact Larmor precession
# --------------------------------------------------------------------------
def _larmor(orc, rotation, dt, nsteps):
    p = inputs.fe_params([20.0] * 3, 1, fix_lattice=1, rotation=rotation, dt_ps=dt)
    th0 = math.radians(60.0)
    s0 = np.array([[math.sin(th0), 0.0, math.cos(th0)]])
    o = orc.Oracle(p, np.array([[10.0, 10.0, 10.0]]), np.zeros((1, 3)), s0)
    o.step(nsteps)
    _, _, s = o.state()
    return s[0], th0, 2.2 * MUB * 1.0 / HBAR


@pytest.mark.parametrize("dt,nsteps", [(1e-4, 1000), (0.05, 40), (1.0, 7)])
def test_larmor_rodrigues_exact(orc, dt, nsteps):
    """ds/dt = omega x s with omega = mu_s mu_B B / hbar z: s(t) = R_z(w t) s(0)
    for any dt (each single-spin factor is an exact rotation)."""
    s, th0, w = _larmor(orc, 0, dt, nsteps)
    t = dt * nsteps
    ref = np.array([math.sin(th0) * math.cos(w * t), math.sin(th0) * math.sin(w * t), math.cos(th0)])
    assert np.abs(s - ref).max() < 1e-12
    assert abs(w - 0.193470) < 1e-6  # Larmor rate of 2.2 mu_B in 1 T


def test_larmor_cayley_angle(orc):
    """The Cayley-type propagator of Sec. 3 rotates by 2 atan(|w| tau / 2) per
    factor; a step holds four factors of tau = dt/4."""
    dt, nsteps = 1.0, 5
    s, th0, w = _larmor(orc, 1, dt, nsteps)
    ang = nsteps * 8.0 * math.atan(w * dt / 8.0)
    ref = np.array([math.sin(th0) * math.cos(ang), math.sin(th0) * math.sin(ang), math.cos(th0)])
    assert np.abs(s - ref).max() < 1e-12
    # and it is measurably not the exact angle
    exact = nsteps * w * dt
    assert abs(ang - exact) > 1e-5


# --------------------------------------------------------------------------
# Two spins with exchange: precession about the conserved total spin
# --------------------------------------------------------------------------
def _two_spin_error(orc, dt, T, d=2.4825, H=(0.0, 0.0, 0.0)):
    p, r = two_atoms(d, fix_lattice=1, dt_ps=dt, H_tesla=list(H))
    s1 = np.array([1.0, 0.0, 0.0])
    s2 = np.array([math.cos(1.2), math.sin(1.2) * 0.6, math.sin(1.2) * 0.8])
    o = orc.Oracle(p, r, np.zeros((2, 3)), np.stack([s1, s2]))
    n = int(round(T / dt))
    o.step(n)
    _, _, s = o.state()
    S = s1 + s2
    Sn = S / np.linalg.norm(S)
    rate = J_bs(p, d) * np.linalg.norm(S) / HBAR

    def rot(v, axis, ang):
        return v * math.cos(ang) + np.cross(axis, v) * math.sin(ang) + axis * axis.dot(v) * (1 - math.cos(ang))

    t = n * dt
    e1 = rot(s1, Sn, rate * t)
    e2 = rot(s2, Sn, rate * t)
    wz = 2.2 * MUB * H[2] / HBAR
    z = np.array([0.0, 0.0, 1.0])
    e1 = rot(e1, z, wz * t)
    e2 = rot(e2, z, wz * t)
    return max(np.abs(s[0] - e1).max(), np.abs(s[1] - e2).max()), s


def test_two_spin_exchange_second_order(orc):
    errs = [_two_spin_error(orc, dt, 0.2)[0] for dt in (2e-3, 1e-3, 5e-4)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, errs
    assert errs[2] < 2e-3


def test_two_spin_total_spin_conserved(orc):
    err, s = _two_spin_error(orc, 1e-3, 0.2)
    s1 = np.array([1.0, 0.0, 0.0])
    s2 = np.array([math.cos(1.2), math.sin(1.2) * 0.6, math.sin(1.2) * 0.8])
    # each sub-rotation of one spin changes S; over a symmetric sweep |S| is
    # conserved only to O(dt^2): bounded by the same splitting error
    assert abs(np.linalg.norm(s[0] + s[1]) - np.linalg.norm(s1 + s2)) < 1e-3


def test_two_spin_with_field_commutes(orc):
    """Isotropic exchange commutes with a uniform field: the motion is the
    exchange precession followed by a global rotation about z."""
    e_f = [_two_spin_error(orc, dt, 0.2, H=(0.0, 0.0, 5.0))[0] for dt in (1e-3, 5e-4)]
    assert 3.6 < e_f[0] / e_f[1] < 4.4


# --------------------------------------------------------------------------
# Morse dimer: classical period T(E) = pi sqrt(2 mu / |E|) / alpha
# --------------------------------------------------------------------------
def test_morse_dimer_period(orc):
    p0 = inputs.fe_params([20.0] * 3, 2)
    r0 = p0["morse_r0_A"]
    d0 = r0 + 0.3
    dt = 5e-5
    p, r = two_atoms(d0, ex_alpha_eV=0.0, H_tesla=[0.0, 0.0, 0.0], dt_ps=dt)
    o = orc.Oracle(p, r, np.zeros((2, 3)), np.array([[0, 0, 1.0], [0, 0, 1.0]]))
    E = V_morse(p, d0)
    mu = p["mass_amu"] / 2.0 / FTOA   # eV ps^2 / A^2
    T_ref = math.pi * math.sqrt(2 * mu / abs(E)) / p["morse_alpha_invA"]
    nsteps = int(3.3 * T_ref / dt)
    seps = []
    for _ in range(nsteps):
        o.step(1)
        rr, _, _ = o.state()
        seps.append(rr[1, 0] - rr[0, 0])
    x = np.asarray(seps)
    # times of the outer turning points (local maxima), parabolic refinement
    idx = [k for k in range(1, len(x) - 1) if x[k] >= x[k - 1] and x[k] > x[k + 1]]
    tmax = []
    for k in idx:
        a, b, c = x[k - 1], x[k], x[k + 1]
        off = 0.5 * (a - c) / (a - 2 * b + c)
        tmax.append((k + 1 + off) * dt)
    assert len(tmax) >= 3
    period = (tmax[-1] - tmax[0]) / (len(tmax) - 1)
    assert abs(period / T_ref - 1.0) < 2e-6, (period, T_ref)
    # total momentum stays zero
    _, v, _ = o.state()
    assert np.abs(v.sum(axis=0)).max() < 1e-12


# --------------------------------------------------------------------------
# Perfect bcc lattice: energies from a shell sum, zero forces
# --------------------------------------------------------------------------
def _bcc_shells(a, rmax):
    pts = []
    rng = range(-4, 5)
    for i in rng:
        for j in rng:
            for k in rng:
                for b in (0.0, 0.5):
                    v = a * np.array([i + b, j + b, k + b])
                    d = float(np.linalg.norm(v))
                    if 0 < d < rmax:
                        pts.append(d)
    return np.array(pts)


def test_bcc_lattice_sums(orc):
    p, r, v, s = inputs.bcc_fe_system(10, 1, T=0.0, sigma=0.0, spins="fm")
    o = orc.Oracle(p, r, v, s)
    e = o.energy()
    n = p["n_atoms"]
    a = inputs.LATTICE_A
    dm = _bcc_shells(a, p["morse_rc_A"])
    dx = _bcc_shells(a, p["ex_rc_A"])
    assert len(dm) == 64 and len(dx) == 14
    vc = V_morse(p, p["morse_rc_A"])
    em = 0.5 * sum(V_morse(p, d) - vc for d in dm)
    ex = -0.5 * sum(J_bs(p, d) for d in dx)
    assert abs(e[1] / n - em) < 1e-12 * abs(em)
    assert abs(e[2] / n - ex) < 1e-12 * abs(ex)
    assert abs(e[3] / n + 2.2 * MUB) < 1e-15
    # unshifted Morse lattice energy and the ferromagnetic exchange energy
    assert abs(0.5 * sum(V_morse(p, d) for d in dm) - (-3.9526149)) < 1e-6
    assert abs(ex - (-0.1111654)) < 1e-6
    assert np.abs(o.forces()).max() < 1e-11
    assert o.pair_count("exchange") == 14 * n and o.pair_count("morse") == 64 * n
    # aligned spins along the field: no torque, T_S = 0
    assert e[6] == 0.0 or abs(e[6]) < 1e-9


# --------------------------------------------------------------------------
# Forces and precession vectors are the gradients of the energy
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_disordered():
    p, r, v, s = inputs.bcc_fe_system(5, 77, T=300.0, sigma=0.12, spins="uniform")
    return p, r, v, s


def test_forces_are_minus_energy_gradient(orc, small_disordered):
    p, r, v, s = small_disordered
    o = orc.Oracle(p, r, v, s)
    F = o.forces()
    rw, _, _ = o.state()   # wrapped positions
    h = 1e-5
    rng = np.random.default_rng(3)
    fmax = np.abs(F).max()
    for i in rng.choice(p["n_atoms"], 6, replace=False):
        for a in range(3):
            rp = rw.copy(); rp[i, a] += h
            rm = rw.copy(); rm[i, a] -= h
            g = (orc.potential_energy(p, rp, s)[3] - orc.potential_energy(p, rm, s)[3]) / (2 * h)
            assert abs(F[i, a] + g) < 1e-7 * fmax, (i, a, F[i, a], -g)


def test_magnetoelastic_force_term(orc, small_disordered):
    """Switching the spins from aligned to random changes the forces by the
    gradient of the exchange energy alone."""
    p, r, v, s = small_disordered
    fm = np.tile([0.0, 0.0, 1.0], (p["n_atoms"], 1))
    dF = orc.Oracle(p, r, v, s).forces() - orc.Oracle(p, r, v, fm).forces()
    rw, _, _ = orc.Oracle(p, r, v, s).state()
    h = 1e-5
    for i in (0, 17, 101):
        for a in range(3):
            rp = rw.copy(); rp[i, a] += h
            rm = rw.copy(); rm[i, a] -= h
            g = ((orc.potential_energy(p, rp, s)[1] - orc.potential_energy(p, rm, s)[1])
                 - (orc.potential_energy(p, rp, fm)[1] - orc.potential_energy(p, rm, fm)[1])) / (2 * h)
            assert abs(dF[i, a] + g) < 1e-8, (i, a)


def test_omega_is_minus_energy_gradient_over_hbar(orc, small_disordered):
    p, r, v, s = small_disordered
    o = orc.Oracle(p, r, v, s)
    w = o.omega()
    rw, _, _ = o.state()
    h = 1e-6
    for i in (0, 5, 77, 249):
        for a in range(3):
            sp = s.copy(); sp[i, a] += h
            sm = s.copy(); sm[i, a] -= h
            g = (orc.potential_energy(p, rw, sp)[3] - orc.potential_energy(p, rw, sm)[3]) / (2 * h)
            assert abs(w[i, a] + g / HBAR) < 1e-6 * np.abs(w).max(), (i, a)


# --------------------------------------------------------------------------
# Invariants of the integrator
# --------------------------------------------------------------------------
def test_spin_norm_preserved(orc, small_disordered):
    p, r, v, s = small_disordered
    o = orc.Oracle(p, r, v, s)
    o.step(300)
    _, _, s1 = o.state()
    assert np.abs(np.linalg.norm(s1, axis=1) - 1.0).max() < 1e-14


def test_total_momentum_conserved(orc, small_disordered):
    p, r, v, s = small_disordered
    o = orc.Oracle(p, r, v, s)
    P0 = v.sum(axis=0)
    o.step(100)
    _, v1, _ = o.state()
    assert np.abs(v1.sum(axis=0) - P0).max() < 1e-10
    # atoms moved: the check is not vacuous
    assert np.abs(v1 - v).max() > 1e-3


def test_time_reversal(orc, small_disordered):
    """10 steps at +dt then 10 at -dt return to the start (symmetric splitting,
    exact inverse of every factor)."""
    p, r, v, s = small_disordered
    o = orc.Oracle(p, r, v, s)
    r0, v0, s0 = o.state()
    o.step(10)
    r1, _, s1 = o.state()
    assert np.abs(r1 - r0).max() > 1e-4 and np.abs(s1 - s0).max() > 1e-3
    o.set_dt(-p["dt_ps"])
    o.step(10)
    r2, v2, s2 = o.state()
    assert np.abs(r2 - r0).max() < 1e-10
    assert np.abs(s2 - s0).max() < 1e-10
    assert np.abs(v2 - v0).max() < 1e-10 * max(1.0, np.abs(v0).max())


def test_energy_fluctuation_second_order(orc):
    """Eq. relative_deviation: the mean relative deviation of the total energy
    over a fixed time grows as dt^2."""
    p, r, v, s = inputs.bcc_fe_system(5, 5, T=200.0, sigma=0.01, spins="uniform")
    T = 0.04
    dev = []
    for dt in (8e-4, 4e-4, 2e-4):
        q = dict(p, dt_ps=dt)
        o = orc.Oracle(q, r, v, s)
        E = []
        for _ in range(int(round(T / dt))):
            o.step(1)
            E.append(o.energy()[4])
        E = np.asarray(E)
        dev.append(np.mean(np.abs((E - E.mean()) / E.mean())))
    r1, r2 = dev[0] / dev[1], dev[1] / dev[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, dev


def test_cell_list_matches_brute_force(orc, small_disordered):
    p, r, v, s = small_disordered
    big = inputs.bcc_fe_system(8, 3, T=300.0, sigma=0.05)  # 8^3 cells: cell list path
    for (q, rr, vv, ss) in [(p, r, v, s), big]:
        a = orc.Oracle(q, rr, vv, ss)
        b = orc.Oracle(q, rr, vv, ss, brute_force=True)
        a.step(3); b.step(3)
        for x, y in zip(a.state(), b.state()):
            assert np.array_equal(x, y)


# --------------------------------------------------------------------------
# Sectoring (Sec. 5.1)
# --------------------------------------------------------------------------
def test_same_colour_sectors_do_not_interact(orc):
    p, r, v, s = inputs.workload("fe_bcc_10x10x10_nve")
    o = orc.Oracle(p, r, v, s)
    info = o.order()
    rw, _, _ = o.state()
    L = np.asarray(p["box"])
    reach = p["ex_rc_A"] + p["skin_A"]
    col, sec = info["colour"], info["sector"]
    assert list(info["nsec"]) == [6, 6, 6]
    assert np.all(np.diff(info["colour_start"]) == np.bincount(col, minlength=8))
    for i in range(0, p["n_atoms"], 7):
        d = rw - rw[i]
        d -= L * np.round(d / L)
        near = np.where((np.einsum("ij,ij->i", d, d) < reach * reach))[0]
        near = near[near != i]
        same = near[(col[near] == col[i])]
        assert np.all(sec[same] == sec[i])
    # the sweep order is (colour, sector, id)
    order = info["order"]
    key = np.stack([col[order], sec[order], order], axis=1)
    assert np.all(np.diff(key[:, 0]) >= 0)
    for k in range(len(order) - 1):
        assert tuple(key[k]) < tuple(key[k + 1])


def test_resectoring_on_displacement(orc):
    """The sector assignment is redone when an atom has moved more than
    skin/2 since the last one; on a fixed schedule with rebuild_every."""
    p, r, v, s = inputs.bcc_fe_system(5, 9, T=200.0)
    v = v.copy()
    v[3] = [2000.0, 0.0, 0.0]   # 0.2 A per step: beyond skin/2 after one step
    o = orc.Oracle(p, r, v, s)
    assert o.rebuilds == 1
    o.step(1)
    assert o.rebuilds == 2
    q = dict(p, rebuild_every=3)
    o2 = orc.Oracle(q, *inputs.bcc_fe_system(5, 9, T=200.0)[1:])
    o2.step(7)
    assert o2.rebuilds == 1 + 2


def test_box_and_norm_validation(orc):
    p, r, v, s = inputs.bcc_fe_system(4, 1)   # 11.5 A < 2 (6 + 0.3)
    with pytest.raises(orc.OracleError) as e:
        orc.Oracle(p, r, v, s)
    assert e.value.code == orc.ORC_ERR_BOX
    p, r, v, s = inputs.bcc_fe_system(5, 1)
    s = s.copy(); s[4] *= 1.001
    with pytest.raises(orc.OracleError) as e:
        orc.Oracle(p, r, v, s)
    assert e.value.code == orc.ORC_ERR_SPIN_NORM


# --------------------------------------------------------------------------
# Langevin spin bath (Sec. 4.1): Curie-Langevin law
# --------------------------------------------------------------------------
@pytest.mark.parametrize("x", [0.7, 2.0, 5.0])
def test_langevin_spins_reach_curie_langevin(orc, x):
    """Non-interacting spins in a field B with the stochastic precession of
    Eq. sLLG relax to <s.z> = coth(x) - 1/x, x = mu_s mu_B B / k_B T.  This
    fixes the noise strength D_S = lambda (1+lambda^2) k_B T / hbar."""
    B = 100.0
    T = 2.2 * MUB * B / (KB * x)
    p, r, v, s = inputs.bcc_fe_system(5, 21, T=0.0, sigma=0.0, spins="uniform",
                                      fix_lattice=1, ex_alpha_eV=0.0, H_tesla=[0.0, 0.0, B], dt_ps=1e-3)
    o = orc.Oracle(p, r, v, s, lam=0.5, temperature=T, seed=99)
    o.step(600)   # relaxation time ~ (1+lambda^2)/(lambda w) ~ 0.13 ps
    acc = []
    for _ in range(60):
        o.step(25)
        acc.append(o.magnetization()[2])
    m = float(np.mean(acc))
    ref = 1.0 / math.tanh(x) - 1.0 / x
    assert abs(m - ref) < 0.02, (m, ref)


# --------------------------------------------------------------------------
# Temperatures (Sec. 4.2)
# --------------------------------------------------------------------------
def test_lattice_temperature(orc):
    """Eq. lattice_temperature uses 3N degrees of freedom; the inputs are
    rescaled to exactly T over 3N-3 (centre of mass removed)."""
    p, r, v, s = inputs.bcc_fe_system(5, 4, T=250.0)
    n = p["n_atoms"]
    e = orc.Oracle(p, r, v, s).energy()
    assert abs(e[5] - 250.0 * (3 * n - 3) / (3 * n)) < 1e-9
    ek = 0.5 * p["mass_amu"] * float((v * v).sum()) / FTOA
    assert abs(e[0] - ek) < 1e-12 * ek


def test_spin_temperature_closed_form(orc):
    """Eq. spin_temperature for uncoupled spins tilted by theta in a field:
    T_S = hbar w sin^2(theta) / (2 k_B cos(theta))."""
    th = 0.4
    p, r, v, _ = inputs.bcc_fe_system(5, 4, T=0.0, sigma=0.0, ex_alpha_eV=0.0, H_tesla=[0.0, 0.0, 3.0])
    n = p["n_atoms"]
    phi = np.linspace(0, 2 * math.pi, n, endpoint=False)
    s = np.stack([math.sin(th) * np.cos(phi), math.sin(th) * np.sin(phi), np.full(n, math.cos(th))], axis=1)
    e = orc.Oracle(p, r, v, s).energy()
    w = 2.2 * MUB * 3.0 / HBAR
    ref = HBAR * w * math.sin(th) ** 2 / (2 * KB * math.cos(th))
    assert abs(e[6] - ref) < 1e-10 * ref
    assert abs(e[3] + n * 2.2 * MUB * 3.0 * math.cos(th)) < 1e-12 * n


# ---------------------------------------------------------------------------
# Lattice bath (Eq. p_advance_T, Sec. 4.2)
# ---------------------------------------------------------------------------
def _free_atoms(ncells, gen_seed, **kw):
    """Atoms without forces (D0 = 0, J = 0): only the bath moves the velocities."""
    p, r, v, s = inputs.bcc_fe_system(ncells, gen_seed, T=300.0, sigma=0.02, spins="uniform",
                                      morse_D0_eV=0.0, ex_alpha_eV=0.0, **kw)
    return p, r, v, s


def test_lattice_bath_at_zero_temperature_is_exact_decay(orc):
    g, n = 7.0, 40
    p, r, v, s = _free_atoms(5, 3, lattice_gamma_ps=g, lattice_temperature_K=0.0, rebuild_every=10)
    o = orc.Oracle(p, r, v, s)
    o.step(n)
    r1, v1, _ = o.state()
    dt = p["dt_ps"]
    np.testing.assert_allclose(v1, v * math.exp(-g * n * dt), rtol=1e-13, atol=1e-13)
    # the drift sees v after the first O(dt/2) of each step: r_n = r_0 + dt v_0 sum_k e^{-g (k + 1/2) dt}
    shift = dt * sum(math.exp(-g * (k + 0.5) * dt) for k in range(n))
    L = np.array(p["box"])
    dr = r1 - (r + shift * v)
    dr -= L * np.round(dr / L)
    assert np.abs(dr).max() < 1e-12


def test_lattice_bath_reaches_equipartition(orc):
    g, T = 40.0, 500.0
    p, r, v, s = _free_atoms(5, 4, lattice_gamma_ps=g, lattice_temperature_K=T)
    o = orc.Oracle(p, r, v * 0.0, s, seed=77)
    kT_m = 8.617333262e-5 * T * 9648.533212 / p["mass_amu"]
    samples = []
    o.step(250)                                 # g t = 1: well past the start
    for _ in range(6):
        o.step(250)                             # 1/g apart: nearly independent
        samples.append(o.state()[1].ravel())
    x = np.concatenate(samples)
    # exact OU flow: the stationary velocity distribution is N(0, k_B T/m)
    assert abs(x.mean()) < 5 * math.sqrt(kT_m / x.size)
    assert x.var() / kT_m == pytest.approx(1.0, abs=5 * math.sqrt(2.0 / x.size) * 2)
