"""sl_magnetization_static: the allocation-free entry point.

It serves callers that cannot call cudaMalloc (inside allocator hooks, in
plugins that only receive device pointers, in processes whose device memory is
fixed after start-up).  Its block partial sums live in a file-scope device
array instead of caller workspace.  These checks call it through the C ABI and
compare with sl_magnetization of a context built on the same spins, twice in a
row and across two systems of different size, so stale scratch contents from a
previous call would show.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_10233_gb300 import inputs  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10233_gb300.build import build
    build()
    from paper_1801_10233_gb300 import _lib
    return _lib


def _static_m(L, s_dev, n, stream):
    out = torch.full((4,), float("nan"), dtype=torch.float64, device=s_dev.device)
    rc = L.sl_magnetization_static(ctypes.c_void_p(s_dev.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, rc
    stream.synchronize()
    return out.cpu().numpy()


def test_static_magnetization_matches_context_entry_point(lib):
    from paper_1801_10233_gb300 import System
    L = lib.load()
    big = System(*inputs.bcc_fe_system(10, 31, T=200.0, spins="cone10"))
    small = System(*inputs.bcc_fe_system(6, 32, T=200.0, spins="uniform"))
    stream = torch.cuda.current_stream()
    for sysm in (big, big, small, big):
        ref = sysm.magnetization()
        _, _, s = sysm.state()
        got = _static_m(L, s, sysm.n, stream)
        assert np.abs(got - ref).max() <= TOL, (got, ref)
    big.step(2)
    ref = big.magnetization()
    got = _static_m(L, big.state()[2], big.n, stream)
    assert np.abs(got - ref).max() <= TOL


def test_static_magnetization_rejects_bad_sizes(lib):
    L = lib.load()
    s = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for n in (0, -5, (1 << 21) + 1):
        assert L.sl_magnetization_static(ctypes.c_void_p(s.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                         None) == lib.SL_ERR_ARG
    assert L.sl_magnetization_static(None, 4, ctypes.c_void_p(out.data_ptr()), None) == lib.SL_ERR_ARG
