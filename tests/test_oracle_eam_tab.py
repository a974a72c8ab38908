"""Pins of the oracle's tabulated embedded-atom potential (App. B: F(rho),
rho(r), phi(r) given as tables on uniform grids, interpolated here by natural
cubic splines): the spline against what the mathematics fixes (exact knots,
exact linear functions, C2 joins, zero end curvature, fourth-order error on a
smooth function within the classical bound), the tabulated potential against
the same functions in closed form, forces against finite differences of the
tabulated energy, and time reversibility of the integrator with it."""
import math

import numpy as np
import pytest

import oracle as orcm
from paper_1801_10233_gb300 import inputs

D_FS = 3.569745
FS = dict(eam_A_eV=0.5, eam_d_A=D_FS, eam_beta=1.8)


def test_spline_hits_the_knots_and_is_exact_for_lines():
    rng = np.random.default_rng(7)
    h = 0.37
    y = rng.normal(size=12)
    x = np.arange(12) * h
    v, _ = orcm.spline_eval(y, h, x)
    assert np.allclose(v, y, rtol=0, atol=1e-14)
    # a natural spline through a line is that line, value and slope
    xl = rng.uniform(0, 11 * h, 50)
    v, dv = orcm.spline_eval(3.0 * x - 2.0, h, xl)
    assert np.abs(v - (3.0 * xl - 2.0)).max() < 1e-13
    assert np.abs(dv - 3.0).max() < 1e-12


def test_spline_joins_are_c2_and_ends_are_natural():
    rng = np.random.default_rng(8)
    h = 0.5
    y = rng.normal(size=9)
    eps = 1e-6
    knots = np.arange(1, 8) * h
    _, dm = orcm.spline_eval(y, h, knots - eps)
    _, d0 = orcm.spline_eval(y, h, knots)
    _, dp = orcm.spline_eval(y, h, knots + eps)
    # first derivative continuous; second derivative (difference quotients
    # from both sides) continuous
    assert np.abs(dp - dm).max() < 1e-4
    assert np.abs((dp - d0) / eps - (d0 - dm) / eps).max() < 1e-3
    # zero curvature at both ends: the slope changes only at second order there
    for a in (0.0, 8 * h):
        _, s = orcm.spline_eval(y, h, np.array([a, a + (eps if a == 0.0 else -eps)]))
        assert abs(s[1] - s[0]) < 1e-9


@pytest.mark.parametrize("n", [21, 41])
def test_spline_error_is_fourth_order_within_the_classical_bound(n):
    """sin on [0, pi] has zero second derivative at both ends, so the natural
    spline is the spline with exact end curvature: |f - S| <= (5/384) h^4
    max|f''''| and |f' - S'| <= (1/24) h^3 max|f''''| (Hall and Meyer)."""
    h = math.pi / (n - 1)
    x = np.linspace(0.0, math.pi, 4001)
    v, dv = orcm.spline_eval(np.sin(np.arange(n) * h), h, x)
    err, derr = np.abs(v - np.sin(x)).max(), np.abs(dv - np.cos(x)).max()
    assert err <= 5.0 / 384.0 * h ** 4
    assert derr <= h ** 3 / 24.0
    # and the order: halving h divides the error by about 16
    v2, _ = orcm.spline_eval(np.sin(np.arange(2 * n - 1) * h / 2), h / 2, x)
    assert 12.0 < err / np.abs(v2 - np.sin(x)).max() < 20.0


def _tab_oracle(p, r, v, s, tables):
    o = orcm.Oracle(p, r, v, s)
    F, drho, rho, phi, dr = tables
    o.set_eam_tables(F, drho, rho, phi, dr)
    return o


def test_tabulated_potential_matches_the_closed_forms():
    """Tables of the Morse pair energy and the Finnis-Sinclair density and
    embedding, on fine grids: energy and forces equal the closed-form
    potential's to within the spline's error."""
    p, r, v, s = inputs.bcc_fe_system(5, 11, T=300.0, sigma=0.06, morse_shift_energy=0)
    ana = orcm.Oracle(dict(p, **FS), r, v, s)
    tabs = inputs.eam_tables(nr=6201, dr=0.001, nrho=40001, drho=0.001, A=FS["eam_A_eV"], d=D_FS,
                             beta=FS["eam_beta"], shifted_force=False, cut=False)
    tab = _tab_oracle(dict(p, eam_tabulated=1), r, v, s, tabs)
    ea, et = ana.energy(), tab.energy()
    assert et[1] == pytest.approx(ea[1], rel=1e-9)
    Fa, Ft = ana.forces(), tab.forces()
    assert np.abs(Ft - Fa).max() <= 1e-7 * np.abs(Fa).max()


@pytest.mark.parametrize("sub", [0, 1])
def test_tabulated_forces_are_minus_energy_gradient(sub):
    p, r, v, s = inputs.bcc_fe_system(5, 12, T=300.0, sigma=0.08, eam_tabulated=1, subtract_ground_exchange=sub)
    o = _tab_oracle(p, r, v, s, inputs.eam_tables())
    rw = o.state()[0]
    F = o.forces()
    h = 1e-5
    rng = np.random.default_rng(3)
    for i in rng.choice(p["n_atoms"], 6, replace=False):
        for a in range(3):
            rp, rm = rw.copy(), rw.copy()
            rp[i, a] += h
            rm[i, a] -= h
            g = (o.potential_energy(rp, s)[3] - o.potential_energy(rm, s)[3]) / (2 * h)
            assert -g == pytest.approx(F[i, a], abs=1e-7 * np.abs(F).max())


def test_tabulated_dynamics_is_time_reversible():
    p, r, v, s = inputs.bcc_fe_system(5, 13, T=300.0, sigma=0.05, eam_tabulated=1, subtract_ground_exchange=1)
    o = _tab_oracle(p, r, v, s, inputs.eam_tables())
    r0, v0, s0 = o.state()
    o.step(10)
    o.set_dt(-p["dt_ps"])
    o.step(10)
    r1, v1, s1 = o.state()
    assert np.abs(r1 - r0).max() < 1e-10
    assert np.abs(s1 - s0).max() < 1e-10
    assert np.abs(v1 - v0).max() < 1e-10 * np.abs(v0).max()


def test_tabulated_mode_needs_its_tables():
    p, r, v, s = inputs.bcc_fe_system(4, 14, T=100.0, eam_tabulated=1, morse_rc_A=5.0)
    o = orcm.Oracle(p, r, v, s)
    assert o.step(1) == orcm.ORC_ERR_ARG
    F, drho, rho, phi, dr = inputs.eam_tables(nr=1000, dr=0.004)    # reaches only 3.996 A < 5 A
    with pytest.raises(orcm.OracleError):
        o.set_eam_tables(F, drho, rho, phi, dr)
    with pytest.raises(orcm.OracleError):
        orcm.Oracle(dict(p, eam_A_eV=0.5), r, v, s)                  # one embedding form at a time
