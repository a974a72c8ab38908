"""Spin-orbit terms (App. A.2) on the GPU against the oracle: uniaxial
anisotropy, Neel pseudo-dipolar and Dzyaloshinskii-Moriya pair terms.

Same bar as the plain path: after the compared steps max |dr| <= 1e-12 L,
max |ds| <= 1e-12, max |dv| <= 1e-12 v_rms, |dE| <= 1e-12 |E|, and the
initial forces, fields and energies (spin-orbit energy included) to 1e-12.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_10233_gb300 import inputs  # noqa: E402

TOL = 1e-12
ANISO = dict(aniso_K_eV=0.003, aniso_axis=[0.6, 0.0, 0.8])
NEEL = dict(neel_alpha_eV=0.01, neel_gamma=0.1, neel_delta_A=1.7)
DMI = dict(dmi_alpha_eV=0.008, dmi_gamma=0.3, dmi_delta_A=1.9)
ALL = dict(ANISO, **NEEL, **DMI)


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


def _state_parity(gpu, ref, p):
    rg, vg, sg = (_np(t) for t in gpu.state())
    ro, vo, so = ref.state()
    L = np.asarray(p["box"])
    dr = rg - ro
    dr -= L * np.round(dr / L)
    assert np.abs(dr).max() <= TOL * L.max(), ("r", np.abs(dr).max())
    assert np.abs(sg - so).max() <= TOL, ("s", np.abs(sg - so).max())
    vrms = math.sqrt(float((vo * vo).mean())) if np.any(vo) else 1.0
    assert np.abs(vg - vo).max() <= TOL * vrms, ("v", np.abs(vg - vo).max())
    eg, eo = gpu.energy(), ref.energy()
    assert abs(eg[4] - eo[4]) <= TOL * abs(eo[4]), ("E", eg[4], eo[4])
    assert abs(eg[7] - eo[7]) <= TOL * max(1.0, abs(eo[4])), ("E_so", eg[7], eo[7])


CASES = {
    "anisotropy": lambda: inputs.bcc_fe_system(6, 31, T=300.0, sigma=0.05, **ANISO),
    "neel": lambda: inputs.bcc_fe_system(6, 32, T=300.0, sigma=0.05, **NEEL),
    "dmi": lambda: inputs.bcc_fe_system(6, 33, T=300.0, sigma=0.05, **DMI),
    "all_ragged_7x6x5": lambda: inputs.bcc_fe_system((7, 6, 5), 34, T=300.0, sigma=0.05, **ALL),
    "all_cayley": lambda: inputs.bcc_fe_system(6, 35, T=200.0, rotation=1, **ALL),
    "all_spins_only": lambda: inputs.bcc_fe_system(6, 36, T=0.0, sigma=0.05, fix_lattice=1, **ALL),
    "all_cone10_rebuild_3": lambda: inputs.bcc_fe_system(6, 37, T=600.0, sigma=0.05, spins="cone10",
                                                         rebuild_every=3, **ALL),
    "easy_plane_tilted_field": lambda: inputs.bcc_fe_system(6, 38, T=200.0, H_tesla=[2.0, -3.0, 3.0],
                                                            aniso_K_eV=-0.004, aniso_axis=[0.0, 0.6, -0.8]),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_init_parity(System, case):
    import oracle
    p, r, v, s = CASES[case]()
    gpu = System(p, r, v, s)
    ref = oracle.Oracle(p, r, v, s)
    Fg, Fo = _np(gpu.forces()), ref.forces()
    assert np.abs(Fg - Fo).max() <= TOL * max(1.0, np.abs(Fo).max())
    wg, wo = _np(gpu.omega()), ref.omega()
    assert np.abs(wg - wo).max() <= TOL * np.abs(wo).max()
    eg, eo = gpu.energy(), ref.energy()
    for k in (0, 1, 2, 3, 4, 7):
        assert abs(eg[k] - eo[k]) <= TOL * max(1.0, abs(eo[k])), (k, eg[k], eo[k])
    assert abs(eg[6] - eo[6]) <= 1e-9 * max(1.0, abs(eo[6]))
    assert eo[7] != 0.0


@pytest.mark.parametrize("case", sorted(CASES))
def test_ten_steps_parity(System, case):
    import oracle
    p, r, v, s = CASES[case]()
    gpu = System(p, r, v, s)
    ref = oracle.Oracle(p, r, v, s)
    gpu.step(10)
    ref.step(10)
    _state_parity(gpu, ref, p)
    assert gpu.counters()["rebuilds"] == ref.rebuilds


def test_spin_bath_with_anisotropy_parity(System):
    """The stochastic LLG with anisotropy: the half turns about n scaled by
    1/(1 + lambda^2), the damping on the whole omega."""
    import oracle
    p, r, v, s = inputs.bcc_fe_system(6, 39, T=300.0, **ALL)
    p = dict(p, **{"lambda": 0.1, "temperature_K": 500.0, "seed": 424242, "replica": 1})
    gpu = System(p, r, v, s)
    ref = oracle.Oracle(p, r, v, s, lam=0.1, temperature=500.0, seed=424242, replica=1)
    gpu.step(10)
    ref.step(10)
    _state_parity(gpu, ref, p)


def test_batch_parity(System):
    """Two replicas of different sizes with the same spin-orbit terms: each
    one's trajectory is the one it has alone."""
    import oracle
    plist, rs, vs, ss = [], [], [], []
    for k, cells in enumerate([6, 7]):
        p, r, v, s = inputs.bcc_fe_system(cells, 60 + k, T=300.0, sigma=0.03, **ALL)
        p = dict(p, replica=k)
        plist.append(p); rs.append(r); vs.append(v); ss.append(s)
    gpu = System(plist, np.concatenate(rs), np.concatenate(vs), np.concatenate(ss))
    gpu.step(6)
    rg, vg, sg = (_np(x) for x in gpu.state())
    eg = gpu.energy_per_replica()
    a0 = 0
    for k, p in enumerate(plist):
        n = p["n_atoms"]
        ref = oracle.Oracle(p, rs[k], vs[k], ss[k], replica=k)
        ref.step(6)
        ro, vo, so = ref.state()
        L = np.array(p["box"])
        dr = rg[a0:a0 + n] - ro
        dr -= L * np.round(dr / L)
        assert np.abs(dr).max() <= TOL * L.max()
        assert np.abs(vg[a0:a0 + n] - vo).max() <= TOL * np.abs(vo).max()
        assert np.abs(sg[a0:a0 + n] - so).max() <= TOL
        eo = ref.energy()
        assert abs(eg[k][7] - eo[7]) <= TOL * abs(eo[4])
        a0 += n


def test_every_tile_shape_gives_the_same_bits(System):
    p, r, v, s = inputs.bcc_fe_system(8, 41, T=300.0, sigma=0.03, **ALL)
    out = []
    for variant in range(5):
        gpu = System(p, r, v, s)
        gpu.set_launch_shape(variant, 128)
        gpu.step(4)
        out.append([_np(t) for t in gpu.state()])
    for o in out[1:]:
        for a, b in zip(out[0], o):
            assert np.array_equal(a, b)


def test_time_reversal(System):
    """Every factor, the anisotropy half turns included, is undone exactly by
    the step at -dt (no rebuild inside the window)."""
    p, r, v, s = inputs.bcc_fe_system(6, 42, T=300.0, sigma=0.05, **ALL)
    gpu = System(p, r, v, s)
    r0, v0, s0 = (_np(t) for t in gpu.state())
    gpu.step(10)
    assert np.abs(_np(gpu.state()[2]) - s0).max() > 1e-4
    gpu.set_dt(-p["dt_ps"])
    gpu.step(10)
    r1, v1, s1 = (_np(t) for t in gpu.state())
    L = np.asarray(p["box"])
    dr = r1 - r0
    dr -= L * np.round(dr / L)
    assert np.abs(dr).max() < 1e-10
    assert np.abs(s1 - s0).max() < 1e-10
    assert np.abs(v1 - v0).max() < 1e-10 * np.abs(v0).max()


def test_energy_conservation(System):
    """NVE with all three terms: energy drift over 2000 steps stays at the
    level of the plain path.  Each single-spin factor is three double-float
    rotations here (two anisotropy half turns and the main turn), each exact
    in |s| to ~2^-48; over 24,000 of them per spin the norm error walks to a
    few 1e-14, so the bar is 5e-14 (1e-14 on the plain path's 4,000)."""
    p, r, v, s = inputs.bcc_fe_system(8, 43, T=200.0, sigma=0.02, **ALL)
    gpu = System(p, r, v, s)
    E0 = gpu.energy()[4]
    gpu.step(2000)
    s1 = _np(gpu.state()[2])
    assert np.abs(np.linalg.norm(s1, axis=1) - 1).max() < 5e-14
    assert abs(gpu.energy()[4] - E0) / p["n_atoms"] < 1e-6


def test_full_size_spin_orbit_workload(System):
    """The 524,288-atom spin-orbit benchmark workload in the bench's launch
    shape: initial forces, fields and energies of every atom, then two
    steps, against the oracle."""
    import oracle
    p, r, v, s = inputs.workload("fe_bcc_64x64x64_spin_orbit")
    gpu = System(p, r, v, s)
    gpu.set_launch_shape(1, 128)
    ref = oracle.Oracle(p, r, v, s)
    Fg, Fo = _np(gpu.forces()), ref.forces()
    assert np.abs(Fg - Fo).max() <= TOL * np.abs(Fo).max()
    wg, wo = _np(gpu.omega()), ref.omega()
    assert np.abs(wg - wo).max() <= TOL * np.abs(wo).max()
    gpu.step(2)
    ref.step(2)
    _state_parity(gpu, ref, p)
