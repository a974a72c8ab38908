"""Embedding term (Finnis-Sinclair form) and collinear ground-state
subtraction (Eq. app:mech1) on the GPU against the oracle, to the bar of
the plain path: 1e-12 on forces, state and energies."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_10233_gb300 import inputs  # noqa: E402

TOL = 1e-12
EAM = dict(eam_A_eV=0.5, eam_d_A=3.569745, eam_beta=1.8)
SO = dict(aniso_K_eV=0.003, aniso_axis=[0.6, 0.0, 0.8], neel_alpha_eV=0.01, neel_gamma=0.1, neel_delta_A=1.7,
          dmi_alpha_eV=0.008, dmi_gamma=0.3, dmi_delta_A=1.9)


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
    "eam": lambda: inputs.bcc_fe_system(6, 51, T=300.0, sigma=0.05, **EAM),
    "ground_sub": lambda: inputs.bcc_fe_system(6, 52, T=300.0, sigma=0.05, subtract_ground_exchange=1),
    "eam_ground_ragged_7x6x5": lambda: inputs.bcc_fe_system((7, 6, 5), 53, T=300.0, sigma=0.05,
                                                            subtract_ground_exchange=1, **EAM),
    "eam_wide_d_rebuild_3": lambda: inputs.bcc_fe_system(6, 54, T=600.0, sigma=0.05, rebuild_every=3,
                                                         eam_A_eV=0.3, eam_d_A=4.6, eam_beta=0.5),
    "eam_within_exchange_cutoff": lambda: inputs.bcc_fe_system(6, 57, T=300.0, sigma=0.05,
                                                               eam_A_eV=0.4, eam_d_A=3.3, eam_beta=1.2),
    "eam_at_exchange_cutoff_so": lambda: inputs.bcc_fe_system(6, 58, T=300.0, sigma=0.05,
                                                              subtract_ground_exchange=1, eam_A_eV=0.5,
                                                              eam_d_A=3.4, eam_beta=1.8, **SO),
    "eam_ground_spin_orbit": lambda: inputs.bcc_fe_system(6, 55, T=300.0, sigma=0.05,
                                                          subtract_ground_exchange=1, **EAM, **SO),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_init_parity(System, case):
    import oracle
    p, r, v, s = CASES[case]()
    gpu = System(p, r, v, s)
    ref = oracle.Oracle(p, r, v, s)
    Fg, Fo = _np(gpu.forces()), ref.forces()
    assert np.abs(Fg - Fo).max() <= TOL * max(1.0, np.abs(Fo).max())
    eg, eo = gpu.energy(), ref.energy()
    for k in (0, 1, 2, 3, 4, 7):
        assert abs(eg[k] - eo[k]) <= TOL * max(1.0, abs(eo[k])), (k, eg[k], eo[k])


@pytest.mark.parametrize("case", sorted(CASES))
def test_ten_steps_parity(System, case):
    import oracle
    p, r, v, s = CASES[case]()
    gpu = System(p, r, v, s)
    ref = oracle.Oracle(p, r, v, s)
    gpu.step(10)
    ref.step(10)
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
    assert gpu.counters()["rebuilds"] == ref.rebuilds


def test_batch_parity(System):
    import oracle
    plist, rs, vs, ss = [], [], [], []
    for k, cells in enumerate([6, 7]):
        p, r, v, s = inputs.bcc_fe_system(cells, 70 + k, T=300.0, sigma=0.03, subtract_ground_exchange=1, **EAM)
        plist.append(dict(p, replica=k)); rs.append(r); vs.append(v); ss.append(s)
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
        assert abs(eg[k][1] - ref.energy()[1]) <= TOL * abs(ref.energy()[1])
        a0 += n


def test_time_reversal_and_energy(System):
    p, r, v, s = inputs.bcc_fe_system(8, 56, T=300.0, sigma=0.03, subtract_ground_exchange=1, **EAM)
    gpu = System(p, r, v, s)
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


def test_full_size_embedding_workload(System):
    """The 524,288-atom embedding benchmark workload (density inside the
    exchange-table kernel) in the bench's launch shape: initial forces and
    energies of every atom, then two steps, against the oracle."""
    import oracle
    p, r, v, s = inputs.workload("fe_bcc_64x64x64_eam")
    gpu = System(p, r, v, s)
    gpu.set_launch_shape(1, 128)
    ref = oracle.Oracle(p, r, v, s)
    Fg, Fo = _np(gpu.forces()), ref.forces()
    assert np.abs(Fg - Fo).max() <= TOL * np.abs(Fo).max()
    eg, eo = gpu.energy(), ref.energy()
    assert abs(eg[1] - eo[1]) <= TOL * abs(eo[1])
    gpu.step(2)
    ref.step(2)
    rg, vg, sg = (_np(t) for t in gpu.state())
    ro, vo, so = ref.state()
    L = np.asarray(p["box"])
    dr = rg - ro
    dr -= L * np.round(dr / L)
    assert np.abs(dr).max() <= TOL * L.max()
    assert np.abs(sg - so).max() <= TOL
    assert np.abs(vg - vo).max() <= TOL * math.sqrt(float((vo * vo).mean()))
    assert abs(gpu.energy()[4] - ref.energy()[4]) <= TOL * abs(ref.energy()[4])
