"""GPU (libsl through the C ABI) against the CPU oracle, element by element.

Tolerances follow the parity metric for the FP64 path: after the compared
steps, max |dr| <= 1e-12 L, max |ds| <= 1e-12, max |dv| <= 1e-12 v_rms and
|dE_total| <= 1e-12 |E_total|.  Sector assignment and sweep order are
integer work and must match exactly.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_10233_gb300 import inputs  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module")
def System():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10233_gb300.build import build
    build()
    from paper_1801_10233_gb300 import System as S
    return S


def _np(t):
    return t.detach().cpu().numpy()


def assert_state_parity(gpu, ref, p, tol=TOL):
    rg, vg, sg = (_np(t) for t in gpu.state())
    ro, vo, so = ref.state()
    L = np.asarray(p["box"])
    dr = rg - ro
    dr -= L * np.round(dr / L)
    assert np.abs(dr).max() <= tol * L.max(), ("r", np.abs(dr).max())
    assert np.abs(sg - so).max() <= tol, ("s", np.abs(sg - so).max())
    vrms = math.sqrt(float((vo * vo).mean())) if np.any(vo) else 0.0
    assert np.abs(vg - vo).max() <= tol * vrms, ("v", np.abs(vg - vo).max(), vrms)
    eg, eo = gpu.energy(), ref.energy()
    assert abs(eg[4] - eo[4]) <= tol * abs(eo[4]), ("E", eg[4], eo[4])
    mg, mo = gpu.magnetization(), ref.magnetization()
    assert np.abs(mg - mo).max() <= tol, ("M", mg, mo)
    return eg, eo


def assert_order_parity(gpu, ref):
    g, o = gpu.order(), ref.order()
    assert np.array_equal(g["nsec"], o["nsec"])
    assert np.array_equal(g["colour_start"], o["colour_start"])
    assert np.array_equal(g["order"], o["order"])


CASES = {
    "fe_10x10x10": lambda: inputs.workload("fe_bcc_10x10x10_nve"),
    "ragged_7x6x5_300K": lambda: inputs.bcc_fe_system((7, 6, 5), 3, T=300.0, sigma=0.05),
    "min_sectors_5x5x5": lambda: inputs.bcc_fe_system(5, 4, T=250.0, sigma=0.03),
    "cayley": lambda: inputs.bcc_fe_system(6, 5, T=200.0, rotation=1),
    "spins_only": lambda: inputs.bcc_fe_system(6, 6, T=0.0, sigma=0.05, fix_lattice=1),
    "rebuild_every_3": lambda: inputs.bcc_fe_system(6, 8, T=600.0, sigma=0.05, rebuild_every=3),
    "tilted_field_5T": lambda: inputs.bcc_fe_system(6, 9, T=200.0, H_tesla=[2.0, -3.0, 3.0]),
    "cone10": lambda: inputs.bcc_fe_system(8, 10, T=200.0, spins="cone10"),
    # other sector grids (Sec. 5.1): 4^3 and 8^3 sectors instead of 6^3; the
    # 1.5 A skin lists up to 54 exchange and 168 Morse neighbours
    "wide_skin_4_sectors": lambda: inputs.bcc_fe_system(10, 14, T=300.0, sigma=0.03, skin_A=1.5,
                                                        max_ex_neighbors=64, max_morse_neighbors=192),
    "narrow_skin_8_sectors": lambda: inputs.bcc_fe_system(10, 15, T=300.0, sigma=0.03, skin_A=0.1),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_init_parity(System, case):
    import oracle
    p, r, v, s = CASES[case]()
    gpu = System(p, r, v, s)
    ref = oracle.Oracle(p, r, v, s)
    assert_order_parity(gpu, ref)
    Fg, Fo = _np(gpu.forces()), ref.forces()
    assert np.abs(Fg - Fo).max() <= TOL * max(1.0, np.abs(Fo).max())
    wg, wo = _np(gpu.omega()), ref.omega()
    assert np.abs(wg - wo).max() <= TOL * np.abs(wo).max()
    eg, eo = gpu.energy(), ref.energy()
    for k in range(4):
        assert abs(eg[k] - eo[k]) <= TOL * max(1.0, abs(eo[k])), (k, eg[k], eo[k])
    assert abs(eg[5] - eo[5]) <= 1e-9 * max(1.0, eo[5])
    assert abs(eg[6] - eo[6]) <= 1e-9 * max(1.0, abs(eo[6]))


@pytest.mark.parametrize("case", sorted(CASES))
def test_ten_steps_parity(System, case):
    import oracle
    p, r, v, s = CASES[case]()
    gpu = System(p, r, v, s)
    ref = oracle.Oracle(p, r, v, s)
    gpu.step(10)
    ref.step(10)
    assert_state_parity(gpu, ref, p)
    assert gpu.counters()["steps"] == 10
    assert gpu.counters()["rebuilds"] == ref.rebuilds
    assert_order_parity(gpu, ref)


def test_langevin_parity(System):
    """Thermostatted spins: both sides draw the same Philox4x32-10 normals
    keyed by (seed, replica; atom id, step, sub-pass)."""
    import oracle
    p, r, v, s = inputs.bcc_fe_system(6, 11, T=300.0)
    p = dict(p, **{"lambda": 0.1, "temperature_K": 500.0, "seed": 123456789, "replica": 3})
    gpu = System(p, r, v, s)
    ref = oracle.Oracle(p, r, v, s, lam=0.1, temperature=500.0, seed=123456789, replica=3)
    gpu.step(10)
    ref.step(10)
    assert_state_parity(gpu, ref, p)


def test_lattice_and_spin_bath_parity(System):
    """Both baths on (Eq. p_advance_T and Eq. s_advance_T): the lattice
    noise draws sub-passes 4 and 5 of the same Philox counters."""
    import oracle
    p, r, v, s = inputs.bcc_fe_system(6, 13, T=300.0)
    p = dict(p, **{"lambda": 0.05, "temperature_K": 400.0, "seed": 987654321, "replica": 2,
                   "lattice_gamma_ps": 3.0, "lattice_temperature_K": 700.0})
    gpu = System(p, r, v, s)
    ref = oracle.Oracle(p, r, v, s, lam=0.05, temperature=400.0, seed=987654321, replica=2)
    gpu.step(10)
    ref.step(10)
    assert_state_parity(gpu, ref, p)


def test_lattice_bath_batch_parity(System):
    """Replicas with different lattice-bath temperatures and damping."""
    import oracle
    plist, rs, vs, ss = [], [], [], []
    for k, (cells, T, g) in enumerate([(6, 100.0, 1.0), (7, 900.0, 8.0)]):
        p, r, v, s = inputs.bcc_fe_system(cells, 40 + k, T=300.0)
        p = dict(p, **{"seed": 55, "replica": k, "lattice_gamma_ps": g, "lattice_temperature_K": T})
        plist.append(p); rs.append(r); vs.append(v); ss.append(s)
    gpu = System(plist, np.concatenate(rs), np.concatenate(vs), np.concatenate(ss))
    gpu.step(8)
    rg, vg, sg = (x.cpu().numpy() for x in gpu.state())
    a0 = 0
    for k, p in enumerate(plist):
        n = p["n_atoms"]
        ref = oracle.Oracle(p, rs[k], vs[k], ss[k], seed=55, replica=k)
        ref.step(8)
        ro, vo, so = ref.state()
        L = np.array(p["box"])
        dr = rg[a0:a0 + n] - ro
        dr -= L * np.round(dr / L)
        assert np.abs(dr).max() <= 1e-12 * L.max()
        assert np.abs(vg[a0:a0 + n] - vo).max() <= 1e-12 * np.abs(vo).max()
        assert np.abs(sg[a0:a0 + n] - so).max() <= 1e-12
        a0 += n


def test_displacement_trigger_parity(System):
    import oracle
    p, r, v, s = inputs.bcc_fe_system(6, 12, T=200.0)
    v = v.copy()
    v[17] = [900.0, -300.0, 100.0]     # crosses skin/2 within a few steps
    gpu = System(p, r, v, s)
    ref = oracle.Oracle(p, r, v, s)
    gpu.step(6)
    ref.step(6)
    assert ref.rebuilds >= 2
    assert gpu.counters()["rebuilds"] == ref.rebuilds
    assert_state_parity(gpu, ref, p)
    assert_order_parity(gpu, ref)


def test_single_spin_larmor(System):
    p = inputs.fe_params([20.0] * 3, 1, fix_lattice=1, dt_ps=0.05)
    th0 = math.radians(60.0)
    s0 = np.array([[math.sin(th0), 0.0, math.cos(th0)]])
    gpu = System(p, np.array([[10.0, 10.0, 10.0]]), np.zeros((1, 3)), s0)
    gpu.step(40)
    w = 2.2 * 5.7883818060e-5 / 6.582119569e-4
    t = 2.0
    ref = [math.sin(th0) * math.cos(w * t), math.sin(th0) * math.sin(w * t), math.cos(th0)]
    assert np.abs(_np(gpu.state()[2])[0] - ref).max() < 1e-12


def test_time_reversal(System):
    p, r, v, s = inputs.bcc_fe_system(6, 13, T=300.0, sigma=0.05)
    gpu = System(p, r, v, s)
    r0, v0, s0 = (_np(t) for t in gpu.state())
    gpu.step(10)
    gpu.set_dt(-p["dt_ps"])
    gpu.step(10)
    r1, v1, s1 = (_np(t) for t in gpu.state())
    assert np.abs(r1 - r0).max() < 1e-10
    assert np.abs(s1 - s0).max() < 1e-10
    assert np.abs(v1 - v0).max() < 1e-10 * np.abs(v0).max()


def test_invariants_long_run(System):
    p, r, v, s = inputs.workload("fe_bcc_10x10x10_nve")
    gpu = System(p, r, v, s)
    P0 = v.sum(axis=0)
    E0 = gpu.energy()[4]
    gpu.step(1000)
    _, v1, s1 = (_np(t) for t in gpu.state())
    assert np.abs(np.linalg.norm(s1, axis=1) - 1).max() < 1e-14
    assert np.abs(v1.sum(axis=0) - P0).max() < 1e-9
    E1 = gpu.energy()[4]
    assert abs(E1 - E0) / p["n_atoms"] < 1e-6


def test_host_state_roundtrip(System):
    p, r, v, s = inputs.bcc_fe_system(6, 14, T=200.0)
    gpu = System(p, r, v, s)
    gpu.step(3)
    hr = torch.empty((p["n_atoms"], 3), dtype=torch.float64).pin_memory()
    hv, hs = torch.empty_like(hr).pin_memory(), torch.empty_like(hr).pin_memory()
    gpu.state_host(hr, hv, hs)
    rd, vd, sd = (_np(t) for t in gpu.state())
    assert np.array_equal(hr.numpy(), rd) and np.array_equal(hv.numpy(), vd) and np.array_equal(hs.numpy(), sd)
    E = gpu.energy()
    gpu.set_state_host(hr, hv, hs)
    assert np.array_equal(_np(gpu.state()[0]), rd)
    assert abs(gpu.energy()[4] - E[4]) <= 1e-13 * abs(E[4])


def test_errors_are_reported(System):
    from paper_1801_10233_gb300 import SlError, _lib
    p, r, v, s = inputs.bcc_fe_system(6, 15)
    s_bad = s.copy()
    s_bad[5] *= 1.01
    with pytest.raises(SlError) as e:
        System(p, r, v, s_bad)
    assert e.value.code == _lib.SL_ERR_SPIN_NORM
    with pytest.raises(SlError) as e:
        System(dict(p, max_morse_neighbors=16), r, v, s)
    assert e.value.code == _lib.SL_ERR_NBR_OVERFLOW
    v2 = v.copy()
    v2[3] = [3000.0, 0.0, 0.0]
    gpu = System(dict(p, rebuild_every=1000), r, v2, s)
    gpu.step(3)
    assert gpu.status() == _lib.SL_ERR_SKIN
    with pytest.raises(SlError):
        gpu.step(1)


def test_full_size_64cubed(System):
    """524,288 atoms (the benchmark workload): initial forces, fields and
    energies for every atom, then two steps, against the oracle."""
    import oracle
    p, r, v, s = inputs.workload("fe_bcc_64x64x64_nve")
    gpu = System(p, r, v, s)
    ref = oracle.Oracle(p, r, v, s)
    assert_order_parity(gpu, ref)
    Fg, Fo = _np(gpu.forces()), ref.forces()
    assert np.abs(Fg - Fo).max() <= TOL * np.abs(Fo).max()
    gpu.step(2)
    ref.step(2)
    assert_state_parity(gpu, ref, p)
