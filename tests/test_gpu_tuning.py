"""Launch-shape autotuner: every tile shape gives bitwise the same
trajectory, and tuning leaves the state bitwise unchanged."""
import numpy as np
import pytest

from paper_1801_10233_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run(p, r, v, s, steps, shape=None, tune=False):
    from paper_1801_10233_gb300 import System
    g = System(p, r, v, s)
    info = None
    if shape is not None:
        g.set_launch_shape(*shape)
    if tune:
        before = [x.cpu().numpy() for x in g.state()]
        info = g.autotune(2)
        after = [x.cpu().numpy() for x in g.state()]
        for a, b in zip(before, after):
            assert np.array_equal(a, b)
    g.step(steps)
    out = [x.cpu().numpy() for x in g.state()]
    g.close()
    return out, info


@pytest.mark.parametrize("batch", [False, True])
def test_every_shape_is_bitwise_identical(batch):
    if batch:
        p, r, v, s = inputs.replica_systems([8, 10, 9], [100.0, 600.0, 1100.0], 31)
    else:
        p, r, v, s = inputs.bcc_fe_system(12, 5, T=300.0, spins="uniform", rebuild_every=4)
    ref, _ = run(p, r, v, s, 8)
    for shape in [(1, 64), (2, 256), (3, 128), (4, 64), (0, 256), (5, 128), (6, 64), (7, 256), (8, 128), (9, 64)]:
        got, _ = run(p, r, v, s, 8, shape=shape)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), shape


def test_autotune_keeps_state_and_results():
    p, r, v, s = inputs.bcc_fe_system(12, 6, T=300.0, spins="uniform", rebuild_every=4)
    ref, _ = run(p, r, v, s, 8)
    got, info = run(p, r, v, s, 8, tune=True)
    assert info["candidates"] == 30 and info["ns_per_step"] > 0 and info["default_ns_per_step"] > 0
    assert info["ns_per_step"] <= info["default_ns_per_step"]
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_autotune_rejects_small_scratch():
    from paper_1801_10233_gb300 import System, _lib
    import ctypes
    p, r, v, s = inputs.bcc_fe_system(6, 1)
    g = System(p, r, v, s)
    scratch = torch.empty(1024, dtype=torch.uint8, device="cuda")
    out = (ctypes.c_int64 * 8)()
    assert g._L.sl_autotune(g._h, scratch.data_ptr(), 1024, 2, out) == _lib.SL_ERR_WORKSPACE
    assert g._L.sl_set_launch_shape(g._h, 10, 128) == _lib.SL_ERR_ARG
    assert g._L.sl_set_launch_shape(g._h, 0, 96) == _lib.SL_ERR_ARG
    g.close()
