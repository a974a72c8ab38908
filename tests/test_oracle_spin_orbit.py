"""Pins of the spin-orbit terms of App. A.2 in the oracle: uniaxial
anisotropy, Neel pseudo-dipolar and Dzyaloshinskii-Moriya (bulk form
D_ij = d(r) e_ij), against closed forms, the exchange term, finite
differences of the energy, and the dynamics' invariants."""
import math

import numpy as np
import pytest

import oracle as orcm
from paper_1801_10233_gb300 import inputs

HBAR = 6.582119569e-4
MUB = 5.7883818060e-5
EX = dict(neel_alpha_eV=0.02726, neel_gamma=0.2171, neel_delta_A=1.841)   # g1 = J


def test_uniaxial_anisotropy_along_the_field_is_exact_precession():
    K, th0, n = 0.004, math.radians(60.0), 50
    p = inputs.fe_params([20.0] * 3, 1, fix_lattice=1, dt_ps=2e-4, aniso_K_eV=K, aniso_axis=[0.0, 0.0, 1.0])
    s0 = np.array([[math.sin(th0), 0.0, math.cos(th0)]])
    o = orcm.Oracle(p, np.array([[10.0, 10.0, 10.0]]), np.zeros((1, 3)), s0)
    o.step(n)
    w = (p["mu_s_muB"] * MUB * 1.0 + 2.0 * K * math.cos(th0)) / HBAR
    ph = w * p["dt_ps"] * n
    want = np.array([math.sin(th0) * math.cos(ph), math.sin(th0) * math.sin(ph), math.cos(th0)])
    np.testing.assert_allclose(o.state()[2][0], want, atol=1e-13)


def _dimer(sa, sb, **kw):
    p = inputs.fe_params([20.0] * 3, 2, fix_lattice=1, morse_D0_eV=0.0, **kw)
    r = np.array([[5.0, 5.0, 5.0], [7.6, 5.0, 5.0]])
    return orcm.Oracle(p, r, np.zeros((2, 3)), np.array([sa, sb], dtype=float))


def test_neel_dimer_against_exchange():
    # g1 = J: with both spins along e the Neel pair energy is -(2/3) J; across e, +J/3
    ex = _dimer([1, 0, 0], [1, 0, 0]).energy()[2]          # -J
    e_par = _dimer([1, 0, 0], [1, 0, 0], **EX).energy()[7]
    e_perp = _dimer([0, 1, 0], [0, 1, 0], **EX).energy()[7]
    assert e_par == pytest.approx(2.0 / 3.0 * ex, rel=1e-14)
    assert e_perp == pytest.approx(-1.0 / 3.0 * ex, rel=1e-14)


def test_dmi_dimer_against_exchange():
    # d = J; e = +x from atom 0 to atom 1: e.(y x z) = 1, e.(z x y) = -1
    ex = _dimer([1, 0, 0], [1, 0, 0]).energy()[2]          # -J
    kw = dict(dmi_alpha_eV=0.02726, dmi_gamma=0.2171, dmi_delta_A=1.841)
    assert _dimer([0, 1, 0], [0, 0, 1], **kw).energy()[7] == pytest.approx(-ex, rel=1e-14)
    assert _dimer([0, 0, 1], [0, 1, 0], **kw).energy()[7] == pytest.approx(ex, rel=1e-14)
    assert _dimer([1, 0, 0], [1, 0, 0], **kw).energy()[7] == 0.0


ALL = dict(aniso_K_eV=0.003, aniso_axis=[0.6, 0.0, 0.8], neel_alpha_eV=0.01, neel_gamma=0.1, neel_delta_A=1.7,
           dmi_alpha_eV=0.008, dmi_gamma=0.3, dmi_delta_A=1.9)


@pytest.fixture(scope="module")
def small():
    p, r, v, s = inputs.bcc_fe_system(5, 21, T=300.0, sigma=0.05, spins="uniform", **ALL)
    return p, r, v, s


def test_forces_and_fields_are_energy_gradients(small):
    """The spin-orbit parts of F and of the spin field are minus the
    gradients of the spin-orbit energy alone (a few eV in total, so central
    differences resolve them to ~1e-10)."""
    p, r, v, s = small
    q0 = dict(p, aniso_K_eV=0.0, neel_alpha_eV=0.0, dmi_alpha_eV=0.0)
    o, o0 = orcm.Oracle(p, r, v, s), orcm.Oracle(q0, r, v, s)
    rw = o.state()[0]
    F = o.forces() - o0.forces()
    B = (o.omega() - o0.omega()) * HBAR
    assert np.abs(F).max() > 1e-3 and np.abs(B).max() > 1e-3
    h = 1e-5
    for a in (0, 31, 177):
        for q in range(3):
            rp = rw.copy(); rp[a, q] += h
            rm = rw.copy(); rm[a, q] -= h
            fd = -(orcm.potential_energy(p, rp, s)[4] - orcm.potential_energy(p, rm, s)[4]) / (2 * h)
            assert fd == pytest.approx(F[a, q], abs=1e-9)
            sp = s.copy(); sp[a, q] += h
            sm = s.copy(); sm[a, q] -= h
            fd = -(orcm.potential_energy(p, rw, sp)[4] - orcm.potential_energy(p, rw, sm)[4]) / (2 * h)
            assert fd == pytest.approx(B[a, q], abs=1e-9)


def test_energy_error_is_second_order_in_dt(small):
    p, r, v, s = small
    dev = []
    for dt in (2e-4, 1e-4):
        o = orcm.Oracle(dict(p, dt_ps=dt, rebuild_every=10), r, v, s)
        e0 = o.energy()[4]
        ex = 0.0
        steps = int(round(0.004 / dt))
        for _ in range(4):
            o.step(steps // 4)
            ex = max(ex, abs(o.energy()[4] - e0))
        dev.append(ex)
    assert dev[0] / dev[1] > 3.0, dev


def test_time_reversal_with_neel_and_dmi(small):
    """Neel and DMI fields do not depend on s_i, so every spin sub-step is
    an exact rotation and the palindromic step is reversible.  No list
    rebuild falls inside the window: a rebuild re-sorts atoms into sectors
    from the current positions, so a rebuild at step 5 going forward and
    one at step 15 going back would sweep in different orders."""
    p, r, v, s = small
    q = dict(p, aniso_K_eV=0.0, rebuild_every=0)
    o = orcm.Oracle(q, r, v, s)
    o.step(10)
    o.set_dt(-q["dt_ps"])
    o.step(10)
    r1, v1, s1 = o.state()
    L = np.array(q["box"])
    dr = r1 - r
    dr -= L * np.round(dr / L)
    assert np.abs(dr).max() < 1e-10 and np.abs(s1 - s).max() < 1e-10
    assert np.abs(np.linalg.norm(s1, axis=1) - 1).max() < 1e-14


@pytest.mark.parametrize("rotation", [0, 1])
def test_time_reversal_with_anisotropy(small, rotation):
    """The anisotropy half turns keep s.n, so the reversed step undoes them
    exactly, with either single-spin propagator."""
    p, r, v, s = small
    q = dict(p, rebuild_every=0, rotation=rotation)
    o = orcm.Oracle(q, r, v, s)
    o.step(10)
    assert np.abs(o.state()[2] - s).max() > 1e-4
    o.set_dt(-q["dt_ps"])
    o.step(10)
    r1, v1, s1 = o.state()
    L = np.array(q["box"])
    dr = r1 - r
    dr -= L * np.round(dr / L)
    assert np.abs(dr).max() < 1e-12 and np.abs(s1 - s).max() < 1e-12


def test_anisotropy_alone_precesses_about_its_axis():
    """H = 0, no neighbours: the spin turns about n at the constant rate
    (2K/hbar)(s.n), whatever the axis."""
    K, n_ax = -0.002, np.array([2.0, -1.0, 2.0]) / 3.0
    p = inputs.fe_params([20.0] * 3, 1, fix_lattice=1, dt_ps=3e-4, H_tesla=[0.0, 0.0, 0.0], aniso_K_eV=K,
                         aniso_axis=list(n_ax))
    s0 = np.array([0.48, 0.6, 0.64])
    o = orcm.Oracle(p, np.array([[10.0, 10.0, 10.0]]), np.zeros((1, 3)), s0[None, :])
    o.step(40)
    c = s0 @ n_ax
    th = 2.0 * K * c / HBAR * 40 * p["dt_ps"]
    want = s0 * math.cos(th) + np.cross(n_ax, s0) * math.sin(th) + n_ax * c * (1.0 - math.cos(th))
    np.testing.assert_allclose(o.state()[2][0], want, atol=1e-13)


def test_anisotropy_under_the_spin_bath_samples_boltzmann():
    """Isolated spins (no neighbours, H = 0) with uniaxial anisotropy under the
    stochastic LLG bath relax to p(x) ~ exp(K x^2 / k_B T) for x = s.n,
    x uniform on [-1, 1] a priori; <x^2> is checked against that integral."""
    kB = 8.617333262e-5
    K, T = 0.003, 30.0
    g = 10
    side = 7.0
    idx = np.stack(np.meshgrid(np.arange(g), np.arange(g), np.arange(g), indexing="ij"), -1).reshape(-1, 3)
    r = (idx + 0.5) * side
    n = r.shape[0]
    rng = np.random.default_rng(4)
    s = rng.normal(size=(n, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    p = inputs.fe_params([g * side] * 3, n, fix_lattice=1, dt_ps=1e-3, H_tesla=[0.0, 0.0, 0.0], aniso_K_eV=K,
                         aniso_axis=[0.0, 0.6, 0.8])
    o = orcm.Oracle(p, r, np.zeros_like(r), s, lam=0.5, temperature=T, seed=7)
    o.step(3000)
    acc = []
    for _ in range(40):
        o.step(50)
        x = o.state()[2] @ np.array([0.0, 0.6, 0.8])
        acc.append(np.mean(x * x))
    b = K / (kB * T)
    xs = np.linspace(-1.0, 1.0, 200001)
    w = np.exp(b * xs * xs)
    want = np.trapezoid(xs * xs * w, xs) / np.trapezoid(w, xs)
    got = float(np.mean(acc))
    # 1000 spins x 40 correlated samples: standard error ~ 0.005
    assert abs(got - want) < 0.02, (got, want)
    assert abs(want - 1.0 / 3.0) > 0.1
