"""Pins of the mechanical-potential extensions in the oracle (App. B): the
embedding term sum_i F(rho_i) (Finnis-Sinclair form, F = -A sqrt(rho),
rho_i = sum_j f(r_ij)) and the subtraction of the collinear magnetic ground
state (Eq. app:mech1), against lattice geometry, exact reductions, finite
differences of the energy and the integrator's invariants."""
import math

import numpy as np
import pytest

import oracle as orcm
from paper_1801_10233_gb300 import inputs

EAM = dict(eam_A_eV=0.5, eam_d_A=3.569745, eam_beta=1.8)
A_FE = 2.8665


def test_bcc_lattice_density_from_shell_geometry():
    """Perfect bcc: 8 neighbours at a sqrt(3)/2 and 6 at a inside d (the third
    shell, a sqrt 2 = 4.05 A, lies beyond d = 3.57 A), so rho is the same for
    every atom and the embedding energy per atom is F(8 f(r1) + 6 f(r2));
    forces vanish by symmetry."""
    p, r, v, s = inputs.bcc_fe_system(6, 1, T=0.0, sigma=0.0, spins="fm", **EAM)
    p0 = dict(p, eam_A_eV=0.0)
    n = p["n_atoms"]
    d, beta, A = EAM["eam_d_A"], EAM["eam_beta"], EAM["eam_A_eV"]
    f = lambda x: (x - d) ** 2 + beta * (x - d) ** 3 / d   # noqa: E731
    rho = 8 * f(A_FE * math.sqrt(3) / 2) + 6 * f(A_FE)
    e_emb = orcm.Oracle(p, r, v, s).energy()[1] - orcm.Oracle(p0, r, v, s).energy()[1]
    assert e_emb / n == pytest.approx(-A * math.sqrt(rho), rel=1e-13)
    F = orcm.Oracle(p, r, v, s).forces()
    assert np.abs(F).max() < 1e-11


def test_zero_embedding_is_the_morse_path_bit_for_bit():
    p, r, v, s = inputs.bcc_fe_system(5, 2, T=300.0, sigma=0.05)
    a = orcm.Oracle(p, r, v, s)
    b = orcm.Oracle(dict(p, eam_A_eV=0.0, eam_d_A=2.0, eam_beta=5.0), r, v, s)
    a.step(5); b.step(5)
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("sub", [0, 1])
def test_forces_are_minus_energy_gradient(sub):
    p, r, v, s = inputs.bcc_fe_system(5, 3, T=300.0, sigma=0.08, subtract_ground_exchange=sub, **EAM)
    o = orcm.Oracle(p, r, v, s)
    rw = o.state()[0]
    F = o.forces()
    fmax = np.abs(F).max()
    h = 1e-5
    for i in (0, 77, 201):
        for a in range(3):
            rp = rw.copy(); rp[i, a] += h
            rm = rw.copy(); rm[i, a] -= h
            g = (orcm.potential_energy(p, rp, s)[3] - orcm.potential_energy(p, rm, s)[3]) / (2 * h)
            assert abs(F[i, a] + g) < 1e-7 * fmax, (i, a, F[i, a], -g)


def test_embedding_energy_matches_brute_force_sum():
    p, r, v, s = inputs.bcc_fe_system(5, 4, T=300.0, sigma=0.1, subtract_ground_exchange=1, **EAM)
    o = orcm.Oracle(p, r, v, s)
    rw = o.state()[0]
    e = o.energy()
    pe = orcm.potential_energy(p, rw, s)
    assert e[1] == pytest.approx(pe[0], rel=1e-12)


def test_ground_subtraction_cancels_exchange_for_collinear_spins():
    """Collinear spins are the magnetic ground state: with the subtraction the
    exchange neither adds energy nor force (Eq. app:mech1)."""
    p, r, v, s = inputs.bcc_fe_system(5, 5, T=300.0, sigma=0.06, spins="fm")
    plain = orcm.Oracle(dict(p, ex_alpha_eV=0.0), r, v, s)
    sub = orcm.Oracle(dict(p, subtract_ground_exchange=1), r, v, s)
    np.testing.assert_allclose(sub.forces(), plain.forces(), rtol=0, atol=1e-12)
    es, ep = sub.energy(), plain.energy()
    assert es[1] + es[2] == pytest.approx(ep[1], rel=1e-13)
    # with disordered spins the subtraction is a pure function of r: the
    # difference of the two mechanical energies is sum J(r_ij) >= 0 here
    p2, r2, v2, s2 = inputs.bcc_fe_system(5, 5, T=300.0, sigma=0.06, spins="uniform")
    d = orcm.Oracle(dict(p2, subtract_ground_exchange=1), r2, v2, s2).energy()[1] - \
        orcm.Oracle(p2, r2, v2, s2).energy()[1]
    assert d > 0.0


def test_time_reversal_and_second_order_energy_error():
    p, r, v, s = inputs.bcc_fe_system(5, 6, T=300.0, sigma=0.05, subtract_ground_exchange=1, **EAM)
    o = orcm.Oracle(p, r, v, s)
    o.step(10)
    o.set_dt(-p["dt_ps"])
    o.step(10)
    r1, v1, s1 = o.state()
    L = np.array(p["box"])
    dr = r1 - r
    dr -= L * np.round(dr / L)
    assert np.abs(dr).max() < 1e-12 and np.abs(s1 - s).max() < 1e-12
    assert np.abs(v1 - v).max() < 1e-10 * np.abs(v).max()
    dev = []
    for dt in (4e-4, 2e-4):
        q = dict(p, dt_ps=dt)
        o = orcm.Oracle(q, r, v, s)
        e0 = o.energy()[4]
        worst = 0.0
        for _ in range(4):
            o.step(int(round(0.008 / dt)) // 4)
            worst = max(worst, abs(o.energy()[4] - e0))
        dev.append(worst)
    assert dev[0] / dev[1] > 3.0, dev


def test_bad_embedding_parameters_are_rejected():
    p, r, v, s = inputs.bcc_fe_system(5, 7, **EAM)
    for bad in (dict(p, eam_d_A=0.0), dict(p, eam_d_A=7.0), dict(p, hamiltonian=1)):
        with pytest.raises(orcm.OracleError):
            orcm.Oracle(bad, r, v, s)
