"""Batched replicas through sl_init_batch: every replica against the CPU
oracle run of that replica alone (same Philox noise stream), and against the
same replica run alone on the GPU (bitwise)."""
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


def _split(x, plist):
    out, k = [], 0
    for p in plist:
        out.append(x[k:k + p["n_atoms"]])
        k += p["n_atoms"]
    return out


def test_batch_matches_oracle_per_replica(System):
    import oracle
    plist, r, v, s = inputs.replica_systems([5, 7, 6, 5], [50.0, 400.0, 900.0, 1200.0], seed=77, lam=0.05)
    gpu = System(plist, r, v, s)
    gpu.step(5)
    rg, vg, sg = (t.cpu().numpy() for t in gpu.state())
    eg = gpu.energy_per_replica()
    for k, (p, rk, vk, sk) in enumerate(zip(plist, _split(r, plist), _split(v, plist), _split(s, plist))):
        o = oracle.Oracle(p, rk, vk, sk, lam=p["lambda"], temperature=p["temperature_K"], seed=p["seed"],
                          replica=p["replica"])
        o.step(5)
        ro, vo, so = o.state()
        L = np.asarray(p["box"])
        dr = _split(rg, plist)[k] - ro
        dr -= L * np.round(dr / L)
        assert np.abs(dr).max() <= TOL * L.max()
        assert np.abs(_split(sg, plist)[k] - so).max() <= TOL
        vrms = float(np.sqrt((vo * vo).mean()))
        assert np.abs(_split(vg, plist)[k] - vo).max() <= TOL * vrms
        eo = o.energy()
        assert abs(eg[k, 4] - eo[4]) <= TOL * abs(eo[4])


def test_batch_replica_equals_single_run(System):
    plist, r, v, s = inputs.replica_systems([6, 5, 8], [300.0, 700.0, 100.0], seed=5, lam=0.02)
    batch = System(plist, r, v, s)
    batch.step(4)
    rb, vb, sb = (t.cpu().numpy() for t in batch.state())
    for k, (p, rk, vk, sk) in enumerate(zip(plist, _split(r, plist), _split(v, plist), _split(s, plist))):
        one = System(p, rk, vk, sk)
        one.step(4)
        r1, v1, s1 = (t.cpu().numpy() for t in one.state())
        assert np.array_equal(_split(rb, plist)[k], r1)
        assert np.array_equal(_split(vb, plist)[k], v1)
        assert np.array_equal(_split(sb, plist)[k], s1)


def test_batch_totals_are_sums(System):
    plist, r, v, s = inputs.replica_systems([5, 6], [200.0, 600.0], seed=9)
    g = System(plist, r, v, s)
    per = g.energy_per_replica()
    tot = g.energy()
    assert abs(tot[4] - per[:, 4].sum()) <= 1e-12 * abs(tot[4])
    m = g.magnetization_per_replica()
    n = np.array([p["n_atoms"] for p in plist])
    mt = g.magnetization()
    assert np.abs(mt[:3] - (m[:, :3] * n[:, None]).sum(axis=0) / n.sum()).max() < 1e-14


def test_batch_at_workload_sizes_matches_oracle(System):
    """Replicas of the batched workload's sizes ({8, 12, 16, 20, 24}^3 cells,
    1,024 to 27,648 atoms, two of 24^3) at bath temperatures spanning its
    50..1200 K ends, lambda 0.01: every replica against its own oracle run
    after 10 steps (same Philox draws), at 1e-12."""
    import os
    import oracle
    cells = [24, 8, 12, 16, 20, 24, 12, 8]
    temps = list(np.linspace(50.0, 1200.0, len(cells)))
    plist, r, v, s = inputs.replica_systems(cells, temps, seed=18012, lam=0.01)
    gpu = System(plist, r, v, s)
    gpu.step(10)
    rg, vg, sg = (_split(t.cpu().numpy(), plist) for t in gpu.state())
    eg = gpu.energy_per_replica()
    mg = gpu.magnetization_per_replica()
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else 1
    for k, (p, rk, vk, sk) in enumerate(zip(plist, _split(r, plist), _split(v, plist), _split(s, plist))):
        o = oracle.Oracle(p, rk, vk, sk, lam=p["lambda"], temperature=p["temperature_K"], seed=p["seed"],
                          replica=p["replica"], threads=threads)
        o.step(10)
        ro, vo, so = o.state()
        L = np.asarray(p["box"])
        dr = rg[k] - ro
        dr -= L * np.round(dr / L)
        assert np.abs(dr).max() <= TOL * L.max(), (k, cells[k])
        assert np.abs(sg[k] - so).max() <= TOL, (k, cells[k])
        vrms = float(np.sqrt((vo * vo).mean()))
        assert np.abs(vg[k] - vo).max() <= TOL * vrms, (k, cells[k])
        eo = o.energy()
        assert abs(eg[k, 4] - eo[4]) <= TOL * abs(eo[4]), (k, cells[k])
        assert np.abs(mg[k] - o.magnetization()).max() <= TOL, (k, cells[k])
