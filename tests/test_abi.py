"""The C ABI without a GPU: header layout vs. the binding, exported symbols,
error strings and host-side validation (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sl.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1801_10233_gb300.build import build
    build()
    from paper_1801_10233_gb300 import _lib
    return _lib


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sl_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    L = lib.load()
    names = _declared_functions()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing
    assert sorted(lib.EXPORTS) == names


def test_param_struct_layout_matches_header(lib, tmp_path):
    fields = [f[0] for f in lib.sl_params._fields_]
    cfields = [("lambda" if f == "lambda_" else f) for f in fields]
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof(sl_params, {f}));\n' for f in cfields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sl.h"\nint main(void){\n'
                   '  printf("%zu\\n", sizeof(sl_params));\n' + body + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(lib.sl_params)
    for f, off in zip(fields, out[1:]):
        assert getattr(lib.sl_params, f).offset == off, f


def test_error_strings(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8, -9):
        assert lib.strerror(code) and lib.strerror(code) != "unknown error"
    assert lib.strerror(-100) == "unknown error"


def test_workspace_and_validation_on_host(lib):
    from paper_1801_10233_gb300 import inputs
    p, *_ = inputs.workload("fe_bcc_10x10x10_nve")
    b = lib.workspace_bytes(p)
    assert b > 2000 * 9 * 32
    # linear in N for the big arrays
    p2, *_ = inputs.bcc_fe_system(20, 1)
    assert lib.workspace_bytes(p2) > 7 * b
    small, *_ = inputs.bcc_fe_system(4, 1)      # 11.5 A box < 2 (6 + 0.3)
    with pytest.raises(lib.SlError) as e:
        lib.workspace_bytes(small)
    assert e.value.code == lib.SL_ERR_BOX
    bad = dict(p, n_atoms=0)
    with pytest.raises(lib.SlError) as e:
        lib.workspace_bytes(bad)
    assert e.value.code == lib.SL_ERR_ARG
    bad = dict(p, rotation=7)
    with pytest.raises(lib.SlError):
        lib.workspace_bytes(bad)


def test_init_rejects_bad_arguments_without_gpu(lib):
    L = lib.load()
    from paper_1801_10233_gb300 import inputs
    p, *_ = inputs.workload("fe_bcc_10x10x10_nve")
    q = lib.make_params(p)
    h = ctypes.c_void_p()
    # NULL state pointers and NULL workspace are rejected before any CUDA call
    assert L.sl_init(ctypes.byref(q), None, None, None, None, 0, None, ctypes.byref(h)) == lib.SL_ERR_ARG
    assert L.sl_init(ctypes.byref(q), 8, 8, 8, None, 0, None, ctypes.byref(h)) == lib.SL_ERR_WORKSPACE
    assert L.sl_init(ctypes.byref(q), 8, 8, 8, 4096 + 8, 1 << 40, None, ctypes.byref(h)) == lib.SL_ERR_WORKSPACE
    assert not h.value
    assert L.sl_step(None, 1) == lib.SL_ERR_ARG
    assert L.sl_status(None) == lib.SL_ERR_ARG


def test_batch_validation_on_host(lib):
    from paper_1801_10233_gb300 import inputs
    plist, *_ = inputs.replica_systems([5, 6], [100.0, 200.0], seed=3)
    b2 = lib.workspace_bytes(plist)
    assert b2 > lib.workspace_bytes(plist[0])
    bad = [dict(plist[0]), dict(plist[1], dt_ps=2e-4)]       # shared field differs
    with pytest.raises(lib.SlError) as e:
        lib.workspace_bytes(bad)
    assert e.value.code == lib.SL_ERR_ARG
    L = lib.load()
    arr = lib.params_array(plist)
    import ctypes as C
    size = C.c_size_t(0)
    assert L.sl_workspace_bytes_batch(arr, 0, C.byref(size)) == lib.SL_ERR_ARG


def test_spin_orbit_validation_on_host(lib):
    """Spin-orbit terms: a unit anisotropy axis, positive ranges, analytic
    Hamiltonian only, the same terms in every replica; the pair tables add
    workspace."""
    from paper_1801_10233_gb300 import inputs
    p, *_ = inputs.workload("fe_bcc_10x10x10_nve")
    b0 = lib.workspace_bytes(p)
    so = dict(p, aniso_K_eV=0.003, aniso_axis=[0.6, 0.0, 0.8], neel_alpha_eV=0.01, neel_delta_A=1.7,
              dmi_alpha_eV=0.008, dmi_delta_A=1.9)
    assert lib.workspace_bytes(so) > b0
    for bad in (dict(so, aniso_axis=[0.6, 0.0, 0.81]), dict(so, neel_delta_A=0.0), dict(so, dmi_delta_A=-1.0),
                dict(so, neel_gamma=float("nan")), dict(so, hamiltonian=1)):
        with pytest.raises(lib.SlError) as e:
            lib.workspace_bytes(bad)
        assert e.value.code == lib.SL_ERR_ARG
    # an axis that is not unit is fine while K = 0
    assert lib.workspace_bytes(dict(p, aniso_axis=[1.0, 1.0, 1.0])) == b0
    plist, *_ = inputs.replica_systems([5, 6], [100.0, 200.0], seed=3)
    with pytest.raises(lib.SlError):
        lib.workspace_bytes([dict(plist[0], dmi_alpha_eV=0.01), dict(plist[1])])


def test_embedding_validation_on_host(lib):
    """Embedding term: 0 < d <= morse_rc, analytic Hamiltonian only, a 0/1
    subtraction flag, the same in every replica; it adds one per-atom table."""
    from paper_1801_10233_gb300 import inputs
    p, *_ = inputs.workload("fe_bcc_10x10x10_nve")
    b0 = lib.workspace_bytes(p)
    e = dict(p, eam_A_eV=0.5, eam_d_A=3.57, eam_beta=1.8)
    assert lib.workspace_bytes(e) > b0
    assert lib.workspace_bytes(dict(p, subtract_ground_exchange=1)) == b0
    for bad in (dict(e, eam_d_A=0.0), dict(e, eam_d_A=6.5), dict(e, hamiltonian=1),
                dict(p, subtract_ground_exchange=2), dict(p, subtract_ground_exchange=1, hamiltonian=1),
                dict(e, eam_beta=float("inf"))):
        with pytest.raises(lib.SlError) as err:
            lib.workspace_bytes(bad)
        assert err.value.code == lib.SL_ERR_ARG
    plist, *_ = inputs.replica_systems([5, 6], [100.0, 200.0], seed=3)
    with pytest.raises(lib.SlError):
        lib.workspace_bytes([dict(plist[0], eam_A_eV=0.5), dict(plist[1])])


def test_box_limit_of_fixed_point_positions(lib):
    """Positions are also held as rint(r 2^48) in 64-bit integers: box edges
    of 4096 A or more are rejected on the host."""
    from paper_1801_10233_gb300 import inputs
    p, *_ = inputs.workload("fe_bcc_10x10x10_nve")
    assert lib.workspace_bytes(dict(p, box=[4000.0, 30.0, 30.0])) > 0
    with pytest.raises(lib.SlError) as e:
        lib.workspace_bytes(dict(p, box=[4096.0, 30.0, 30.0]))
    assert e.value.code == lib.SL_ERR_BOX


def test_exponential_ranges_are_validated_on_host(lib):
    """The pair kernels' double-float exp keeps its accuracy for |x| <= 11:
    parameter sets whose exponentials inside a cutoff reach further
    (e^{-r^2/delta^2} for r < ex_rc, e^{-a (r - r0)} for 0 < r < morse_rc)
    are rejected."""
    from paper_1801_10233_gb300 import inputs
    p, *_ = inputs.workload("fe_bcc_10x10x10_nve")
    assert lib.workspace_bytes(dict(p, ex_delta_A=3.4 / 11.0 ** 0.5 + 1e-6)) > 0
    bad = (dict(p, ex_delta_A=0.3), dict(p, ex_delta_A=3.4 / 11.0 ** 0.5 - 1e-6),
           dict(p, neel_alpha_eV=0.01, neel_delta_A=0.9), dict(p, dmi_alpha_eV=0.01, dmi_delta_A=0.5),
           dict(p, morse_alpha_invA=4.0), dict(p, morse_r0_A=0.2, morse_alpha_invA=1.9))
    for q in bad:
        with pytest.raises(lib.SlError) as e:
            lib.workspace_bytes(q)
        assert e.value.code == lib.SL_ERR_ARG
    # a small Neel/DMI range is fine while the term is off
    assert lib.workspace_bytes(dict(p, neel_delta_A=0.1, dmi_delta_A=0.1)) > 0


def test_sector_grid_of_a_commensurate_box(lib, orc):
    """A box whose edge is an exact multiple of the spin reach (cutoff +
    skin): the sectors must still be wider than the reach, so that no listed
    exchange pair joins two sectors of one colour; library and oracle agree."""
    import numpy as np
    from paper_1801_10233_gb300 import inputs
    p, r, v, s = inputs.bcc_fe_system(11, 21, T=100.0, a=32.0 / 11.0, ex_rc_A=3.5, skin_A=0.5)
    p = dict(p, box=[32.0, 32.0, 32.0])
    reach = p["ex_rc_A"] + p["skin_A"]
    assert 32.0 / reach == 8.0
    nsec, edge = lib.sector_grid(p)
    assert nsec == [6, 6, 6]
    assert all(e >= reach * (1 + 1e-6) for e in edge)
    o = orc.Oracle(p, np.mod(r, 32.0), v, s)
    assert list(o.order()["nsec"]) == nsec
    # a box just wide enough for 8 sectors with the margin keeps 8
    q = dict(p, box=[32.0 * (1 + 2e-6)] * 3)
    assert lib.sector_grid(q)[0] == [8, 8, 8]
