"""Tabulated embedded-atom potential (App. B: F(rho), rho(r), phi(r) from
tables on uniform grids through natural cubic splines) on the GPU against
the oracle with the same tables, to the bar of the plain path: 1e-12 on
forces, state and energies."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_10233_gb300 import inputs  # noqa: E402

TOL = 1e-12
TAB = dict(eam_tabulated=1)
SO = dict(aniso_K_eV=0.003, aniso_axis=[0.6, 0.0, 0.8], neel_alpha_eV=0.01, neel_gamma=0.1, neel_delta_A=1.7,
          dmi_alpha_eV=0.008, dmi_gamma=0.3, dmi_delta_A=1.9)
COARSE = dict(nr=400, dr=0.0155, nrho=300, drho=0.1)


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


CASES = {
    "tab": (lambda: inputs.bcc_fe_system(6, 61, T=300.0, sigma=0.05, **TAB), {}),
    "tab_ground": (lambda: inputs.bcc_fe_system(6, 62, T=300.0, sigma=0.05, subtract_ground_exchange=1, **TAB), {}),
    "tab_ragged_7x6x5": (lambda: inputs.bcc_fe_system((7, 6, 5), 63, T=300.0, sigma=0.05, **TAB), {}),
    "tab_coarse_grids": (lambda: inputs.bcc_fe_system(6, 64, T=300.0, sigma=0.05, **TAB), COARSE),
    "tab_rebuild_3": (lambda: inputs.bcc_fe_system(6, 65, T=600.0, sigma=0.05, rebuild_every=3, **TAB), {}),
    "tab_ground_spin_orbit": (lambda: inputs.bcc_fe_system(6, 66, T=300.0, sigma=0.05, subtract_ground_exchange=1,
                                                           **TAB, **SO), {}),
}


def _pair(System, p, r, v, s, tables, **okw):
    import oracle
    gpu = System(p, r, v, s)
    gpu.set_eam_tables(*tables)
    ref = oracle.Oracle(p, r, v, s, **okw)
    ref.set_eam_tables(*tables)
    return gpu, ref


def _state_parity(gpu, ref, p):
    rg, vg, sg = (_np(t) for t in gpu.state())
    ro, vo, so = ref.state()
    L = np.asarray(p["box"])
    dr = rg - ro
    dr -= L * np.round(dr / L)
    assert np.abs(dr).max() <= TOL * L.max()
    assert np.abs(sg - so).max() <= TOL
    vrms = math.sqrt(float((vo * vo).mean()))
    assert np.abs(vg - vo).max() <= TOL * vrms
    eg, eo = gpu.energy(), ref.energy()
    assert abs(eg[4] - eo[4]) <= TOL * abs(eo[4])
    assert abs(eg[1] - eo[1]) <= TOL * abs(eo[1])


@pytest.mark.parametrize("case", sorted(CASES))
def test_init_parity(System, case):
    make, grid = CASES[case]
    p, r, v, s = make()
    gpu, ref = _pair(System, p, r, v, s, inputs.eam_tables(**grid))
    Fg, Fo = _np(gpu.forces()), ref.forces()
    assert np.abs(Fg - Fo).max() <= TOL * max(1.0, np.abs(Fo).max())
    eg, eo = gpu.energy(), ref.energy()
    for k in (0, 1, 2, 3, 4, 7):
        assert abs(eg[k] - eo[k]) <= TOL * max(1.0, abs(eo[k])), (k, eg[k], eo[k])


@pytest.mark.parametrize("case", sorted(CASES))
def test_ten_steps_parity(System, case):
    make, grid = CASES[case]
    p, r, v, s = make()
    gpu, ref = _pair(System, p, r, v, s, inputs.eam_tables(**grid))
    gpu.step(10)
    ref.step(10)
    _state_parity(gpu, ref, p)
    assert gpu.counters()["rebuilds"] == ref.rebuilds


def test_batch_parity(System):
    import oracle
    plist, rs, vs, ss = [], [], [], []
    for k, cells in enumerate([6, 7]):
        p, r, v, s = inputs.bcc_fe_system(cells, 80 + k, T=300.0, sigma=0.03, subtract_ground_exchange=1, **TAB)
        plist.append(dict(p, replica=k)); rs.append(r); vs.append(v); ss.append(s)
    tables = inputs.eam_tables()
    gpu = System(plist, np.concatenate(rs), np.concatenate(vs), np.concatenate(ss))
    gpu.set_eam_tables(*tables)
    gpu.step(6)
    rg, vg, sg = (_np(x) for x in gpu.state())
    eg = gpu.energy_per_replica()
    a0 = 0
    for k, p in enumerate(plist):
        n = p["n_atoms"]
        ref = oracle.Oracle(p, rs[k], vs[k], ss[k], replica=k)
        ref.set_eam_tables(*tables)
        ref.step(6)
        ro, vo, so = ref.state()
        L = np.array(p["box"])
        dr = rg[a0:a0 + n] - ro
        dr -= L * np.round(dr / L)
        assert np.abs(dr).max() <= TOL * L.max()
        assert np.abs(vg[a0:a0 + n] - vo).max() <= TOL * np.abs(vo).max()
        assert np.abs(sg[a0:a0 + n] - so).max() <= TOL
        assert abs(eg[k][1] - ref.energy()[1]) <= TOL * abs(ref.energy()[1])
        a0 += n


def test_tables_are_required_and_checked(System):
    from paper_1801_10233_gb300 import SlError, _lib
    p, r, v, s = inputs.bcc_fe_system(6, 67, T=300.0, **TAB)
    gpu = System(p, r, v, s)
    with pytest.raises(SlError) as e:
        gpu.step(1)
    assert e.value.code == _lib.SL_ERR_ARG
    F, drho, rho, phi, dr = inputs.eam_tables(nr=1000, dr=0.005)          # reaches 4.995 A < 6 A
    with pytest.raises(SlError):
        gpu.set_eam_tables(F, drho, rho, phi, dr)
    F, drho, rho, phi, dr = inputs.eam_tables()
    bad = phi.copy()
    bad[7] = np.nan
    with pytest.raises(SlError):
        gpu.set_eam_tables(F, drho, rho, bad, dr)
    plain = System(dict(p, eam_tabulated=0), r, v, s)
    with pytest.raises(SlError):
        plain.set_eam_tables(F, drho, rho, phi, dr)
    gpu.set_eam_tables(F, drho, rho, phi, dr)
    gpu.step(1)


def test_time_reversal_and_energy(System):
    p, r, v, s = inputs.bcc_fe_system(8, 68, T=300.0, sigma=0.03, subtract_ground_exchange=1, **TAB)
    gpu = System(p, r, v, s)
    gpu.set_eam_tables(*inputs.eam_tables())
    r0, v0, s0 = (_np(t) for t in gpu.state())
    E0 = gpu.energy()[4]
    gpu.step(10)
    gpu.set_dt(-p["dt_ps"])
    gpu.step(10)
    r1, v1, s1 = (_np(t) for t in gpu.state())
    L = np.asarray(p["box"])
    dr = r1 - r0
    dr -= L * np.round(dr / L)
    assert np.abs(dr).max() < 1e-10 and np.abs(s1 - s0).max() < 1e-10
    assert np.abs(v1 - v0).max() < 1e-10 * np.abs(v0).max()
    gpu.set_dt(p["dt_ps"])
    gpu.step(2000)
    assert abs(gpu.energy()[4] - E0) / p["n_atoms"] < 1e-6


def test_full_size_tabulated_workload(System):
    """The 524,288-atom tabulated benchmark workload in the bench's launch
    shape: initial forces and energies of every atom, then two steps,
    against the oracle."""
    p, r, v, s = inputs.workload("fe_bcc_64x64x64_eam_tab")
    gpu, ref = _pair(System, p, r, v, s, inputs.eam_tables(), threads=_cores())
    gpu.set_launch_shape(1, 128)
    Fg, Fo = _np(gpu.forces()), ref.forces()
    assert np.abs(Fg - Fo).max() <= TOL * np.abs(Fo).max()
    eg, eo = gpu.energy(), ref.energy()
    assert abs(eg[1] - eo[1]) <= TOL * abs(eo[1])
    gpu.step(2)
    ref.step(2)
    _state_parity(gpu, ref, p)


def _cores():
    import os
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1
