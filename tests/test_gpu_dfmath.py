"""Accuracy of the double-float functions the pair and rotation kernels are
built from (exp, 1/sqrt, sqrt), evaluated on the GPU through sl_df_eval,
against numpy's FP64 functions at the same (double-float-rounded) inputs.
The bars are the errors the kernels' accuracy claims rest on: 7e-14
relative for exp over [-12, 6] (the Morse and Bethe-Slater arguments; 6.1e-14
measured), 5e-14 for 1/sqrt over r^2 in [1, 64] A^2 (4.6e-14) and 2e-14 for
sqrt (1.5e-14)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_10233_gb300.build import build
    build()
    from paper_1801_10233_gb300 import _lib
    return _lib


def _df_round(x):
    """The library's FP64 -> double-float split: hi = the top 24 significant
    bits of x (truncated), lo = the rest rounded to a float."""
    b = x.view(np.uint64) & ~np.uint64((1 << 29) - 1)
    hi = b.view(np.float64)
    lo = (x - hi).astype(np.float32).astype(np.float64)
    return hi + lo


def _eval(lib, fn, x):
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    lib.df_eval(fn, xd.data_ptr(), yd.data_ptr(), x.size, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _inputs(lo, hi, n, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.uniform(lo, hi, n), np.linspace(lo, hi, 4097)])


def test_exp(lib):
    x = _inputs(-12.0, 6.0, 1 << 20, 1)
    y = _eval(lib, lib.SL_DF_EXP, x)
    ref = np.exp(_df_round(x))
    assert np.abs(y / ref - 1.0).max() < 7e-14
    # exact powers of two and 1 at the table's nodes
    z = np.array([0.0, np.log(2.0) * 3, -np.log(2.0) * 5])
    assert np.abs(_eval(lib, lib.SL_DF_EXP, z) / np.exp(_df_round(z)) - 1.0).max() < 7e-14


def test_rsqrt(lib):
    x = _inputs(1.0, 64.0, 1 << 20, 2)
    y = _eval(lib, lib.SL_DF_RSQRT, x)
    ref = 1.0 / np.sqrt(_df_round(x))
    assert np.abs(y / ref - 1.0).max() < 5e-14


def test_sqrt(lib):
    x = _inputs(0.5, 64.0, 1 << 20, 3)
    y = _eval(lib, lib.SL_DF_SQRT, x)
    ref = np.sqrt(_df_round(x))
    assert np.abs(y / ref - 1.0).max() < 2e-14


def test_arguments_checked(lib):
    from paper_1801_10233_gb300 import SlError
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(SlError):
        lib.df_eval(7, x.data_ptr(), x.data_ptr(), 4)
    with pytest.raises(SlError):
        lib.df_eval(lib.SL_DF_EXP, x.data_ptr(), x.data_ptr(), -1)
    lib.df_eval(lib.SL_DF_EXP, x.data_ptr(), x.data_ptr(), 0)
