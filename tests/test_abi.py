"""The C-ABI library builds for sm_103a, loads on a machine without a GPU,
and exports every entry point include/mpm.h declares (no compute calls)."""
import ctypes as C

from paper_1909_13380_gb300 import mpm


def test_library_exports_every_declared_entry_point():
    lib = mpm.load()
    names = mpm.header_entry_points()
    assert "mpm_step" in names and "mpm_create_mesh" in names and len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_struct_layouts_match_header_sizes():
    # int32 dim, int32[3], double h, double[3], int32[6], double[6], double[3], double dt,
    # int32 scheme, int32 precision, double mass_tol, void* stream
    assert C.sizeof(mpm.mpm_mesh_desc) == 4 + 12 + 8 + 24 + 24 + 48 + 24 + 8 + 4 + 4 + 8 + 8
    assert C.sizeof(mpm.mpm_material) == 8 + 6 * 8


def test_argument_errors_need_no_gpu():
    # validation happens before any device call
    d = mpm.make_desc(4, (4, 4, 4), 0.1)
    h = C.c_void_p()
    assert mpm.load().mpm_create_mesh(C.byref(d), C.byref(h)) == mpm.MPM_ERR_ARG
    d = mpm.make_desc(3, (4, 0, 4), 0.1)
    assert mpm.load().mpm_create_mesh(C.byref(d), C.byref(h)) == mpm.MPM_ERR_ARG
    assert mpm.load().mpm_sort_keys(None, None, 10, 0, None) == mpm.MPM_ERR_ARG
