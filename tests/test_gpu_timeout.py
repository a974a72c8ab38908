"""A wait that never completes ends with an error status, not a hung GPU.

The tensor-core kernels wait for their MMA completion on a shared-memory
barrier with a bound on the time (mbar_wait_ns); after the bound a kernel
reports SL_ERR_TIMEOUT.  sl_check_bounded_wait runs that same wait on a
barrier nothing completes, with a short bound, and one that an arrival
completes; afterwards the GPU is still usable."""
import ctypes
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_10233_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10233_gb300.build import build
    build()
    from paper_1801_10233_gb300 import _lib
    return _lib


def _wait(L, limit_ns, arrive):
    st = ctypes.c_int32(-100)
    rc = L.sl_check_bounded_wait(int(limit_ns), int(arrive), ctypes.byref(st))
    return rc, st.value


def test_a_wait_nothing_completes_times_out_and_the_gpu_stays_usable(lib):
    L = lib.load()
    t0 = time.perf_counter()
    rc, st = _wait(L, 2_000_000, 0)          # 2 ms, nobody arrives
    assert rc == 0 and st == lib.SL_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    rc, st = _wait(L, 2_000_000, 1)          # the arrival completes the wait
    assert rc == 0 and st == lib.SL_OK
    # the device still runs the library's kernels
    from paper_1801_10233_gb300 import System
    p, r, v, s = inputs.bcc_fe_system(6, 71, T=200.0)
    g = System(p, r, v, s)
    g.step(3)
    assert g.status() == 0
    assert np.isfinite(g.energy()[4])


def test_bounds_are_checked_on_the_host(lib):
    L = lib.load()
    st = ctypes.c_int32(0)
    assert L.sl_check_bounded_wait(-1, 0, ctypes.byref(st)) == lib.SL_ERR_ARG
    assert L.sl_check_bounded_wait(3_000_000_000, 0, ctypes.byref(st)) == lib.SL_ERR_ARG
    assert L.sl_check_bounded_wait(1000, 0, None) == lib.SL_ERR_ARG
