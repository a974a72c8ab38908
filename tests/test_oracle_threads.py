"""The oracle split over threads reproduces the serial oracle bit for bit.

Sec. 5.1: sectors of one colour are further apart than every cutoff, so the
spins of one colour can turn sector by sector in any order, or side by side,
with the same result as the sequential sweep; forces, pair tables and lists
are sums per atom.  These cases run both ways and compare every number."""
import numpy as np
import pytest

import oracle
from paper_1801_10233_gb300 import inputs
from _ml_models import fitted_norm, model  # noqa: E402


def _both(p, r, v, s, nsteps, threads=4, setup=None, **kw):
    out = []
    for t in (1, threads):
        o = oracle.Oracle(p, r, v, s, threads=t, **kw)
        if setup:
            setup(o)
        if t > 1 and o.threads == 1:
            pytest.skip("oracle built without OpenMP")
        assert o.step(nsteps) == 0
        out.append(o)
    return out


def _same(a, b):
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.forces(), b.forces())
    assert np.array_equal(a.energy(), b.energy())
    assert np.array_equal(a.magnetization(), b.magnetization())
    assert a.rebuilds == b.rebuilds


def _sectors_per_colour(o):
    ns = o.order()["nsec"]
    return int(np.prod(ns)) // 8


@pytest.mark.parametrize("rotation", [0, 1])
def test_threads_bitwise_with_scheduled_rebuilds(rotation):
    p, r, v, s = inputs.bcc_fe_system(8, 41, T=300.0, sigma=0.05, spins="uniform",
                                      rebuild_every=4, rotation=rotation)
    a, b = _both(p, r, v, s, 12)
    assert _sectors_per_colour(a) >= 8 and a.rebuilds == 4
    _same(a, b)


def test_threads_bitwise_with_displacement_rebuilds():
    p, r, v, s = inputs.bcc_fe_system(8, 42, T=1200.0, sigma=0.05, spins="uniform", skin_A=0.05, dt_ps=1e-3)
    a, b = _both(p, r, v, s, 40)
    assert a.rebuilds > 2
    _same(a, b)


def test_threads_bitwise_with_both_baths():
    p, r, v, s = inputs.bcc_fe_system(8, 43, T=300.0, sigma=0.05, spins="uniform",
                                      lattice_gamma_ps=2.0, lattice_temperature_K=300.0)
    a, b = _both(p, r, v, s, 10, lam=0.05, temperature=500.0, seed=7, replica=3)
    _same(a, b)


def test_threads_bitwise_with_spin_orbit_terms():
    so = dict(aniso_K_eV=0.003, aniso_axis=[0.6, 0.0, 0.8], neel_alpha_eV=0.01, neel_gamma=0.1, neel_delta_A=1.7,
              dmi_alpha_eV=0.008, dmi_gamma=0.3, dmi_delta_A=1.9)
    p, r, v, s = inputs.bcc_fe_system(8, 44, T=300.0, sigma=0.05, spins="uniform", **so)
    a, b = _both(p, r, v, s, 10, lam=0.02, temperature=100.0, seed=3)
    _same(a, b)


def test_threads_bitwise_with_embedding():
    p, r, v, s = inputs.bcc_fe_system(8, 45, T=300.0, sigma=0.05, spins="cone10", **inputs.EMBEDDING)
    a, b = _both(p, r, v, s, 10)
    _same(a, b)


def test_threads_bitwise_with_learned_hamiltonian():
    p, r, v, s = inputs.bcc_fe_system(9, 46, T=300.0, sigma=0.05, spins="uniform", hamiltonian=1)
    par, norm = model(), fitted_norm(r, s, p["box"])
    a, b = _both(p, r, v, s, 2, setup=lambda o: o.set_model(par, norm))
    assert _sectors_per_colour(a) >= 8
    _same(a, b)


def test_threads_after_a_skin_error_fall_back_to_the_serial_order():
    """A scheduled rebuild that comes too late sets the skin error; the
    threaded sweep then runs serially (no race), still bit-identical."""
    p, r, v, s = inputs.bcc_fe_system(8, 47, T=1200.0, sigma=0.05, spins="uniform", skin_A=0.02,
                                      dt_ps=1e-3, rebuild_every=1000)
    a = oracle.Oracle(p, r, v, s)
    b = oracle.Oracle(p, r, v, s, threads=4)
    if b.threads == 1:
        pytest.skip("oracle built without OpenMP")
    ea, eb = a.step(30), b.step(30)
    assert ea == eb != 0
    _same(a, b)
