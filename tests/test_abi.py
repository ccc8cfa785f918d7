"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/bp1104.h declares; argument validation that happens on the host
before any CUDA call is checked here without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1104_5243_gb300 import _native as N
from paper_1104_5243_gb300 import build as B

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
HEADER = os.path.join(INCLUDE, "bp1104.h")
HEADER_F64 = os.path.join(INCLUDE, "bp1104_f64.h")


def declared_symbols(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.lib()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("bp_create", "bp_add_projections", "bp_adjoint", "bp_finalize", "bp_reset",
                 "bp_destroy", "bp_last_error", "bp_get_state", "bp_set_state"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_exactly_the_header():
    assert sorted(N.SIGNATURES) == declared_symbols()


def needed_libraries(path):
    """DT_NEEDED entries of a shared object's dynamic section (readelf -d)."""
    import subprocess
    out = subprocess.run(["readelf", "-d", path], capture_output=True, text=True, check=True).stdout
    return re.findall(r"\(NEEDED\)\s+Shared library: \[([^\]]+)\]", out)


def test_library_links_no_torch(lib):
    # the ABI is plain C: neither shared object may depend on libtorch/c10
    for path in (N.library_path(), B.build_f64()):
        needed = needed_libraries(path)
        assert needed, path
        assert not any("torch" in n or "c10" in n for n in needed), needed


def test_f64_check_library_exports_its_header():
    """The float64 gradient-check library (test support) exports exactly what
    include/bp1104_f64.h declares, and its binding covers it."""
    from paper_1104_5243_gb300 import _f64
    B.build_f64()
    f64 = _f64.lib()
    syms = declared_symbols(HEADER_F64)
    assert syms == sorted(_f64.SIGNATURES)
    for name in syms:
        assert hasattr(f64, name), name
    # host-side validation, before any CUDA call
    O = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    assert f64.bp_f64_backproject(0, 1.0, O, 8, 8, None, None, 1, None, None) == N.BP_EINVAL
    assert f64.bp_f64_adjoint(8, 1.0, O, 8, 8, None, None, 1, None, None) == N.BP_EINVAL
    assert b"bp_f64_adjoint" in f64.bp_f64_last_error()
    # the product library holds no float64 kernel entry point
    assert not any(name.startswith("bp_f64") for name in declared_symbols())


def test_create_rejects_bad_sizes_without_touching_the_gpu(lib):
    h = ctypes.c_void_p()
    O = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    for (L, R, isx, isy, dt) in [(0, 1.0, 8, 8, 0), (8, 0.0, 8, 8, 0), (8, -1.0, 8, 8, 0),
                                 (8, 1.0, 0, 8, 0), (8, 1.0, 8, 40000, 0), (8, 1.0, 8, 8, 7)]:
        st = lib.bp_create(ctypes.byref(h), L, R, ctypes.cast(O, ctypes.c_void_p), isx, isy, dt, None)
        assert st == N.BP_EINVAL
        assert h.value is None
        assert "bp_create" in N.bp_last_error(None)
    assert lib.bp_create(None, 8, 1.0, ctypes.cast(O, ctypes.c_void_p), 8, 8, 0, None) == N.BP_EINVAL


def test_null_context_is_rejected(lib):
    assert lib.bp_reset(None) == N.BP_EINVAL
    assert lib.bp_add_projections(None, None, 0, None, 1) == N.BP_EINVAL
    assert lib.bp_finalize(None, None, 0) == N.BP_EINVAL
    assert lib.bp_adjoint(None, None, 0, None, 1, None, 0) == N.BP_EINVAL
    assert lib.bp_add_projections_finalize(None, None, 0, None, 1, None, 0) == N.BP_EINVAL
    assert "bp_add_projections_finalize" in N.bp_last_error(None)
    assert lib.bp_set_option(None, 1, 0) == N.BP_EINVAL
    assert lib.bp_move_slab(None, 0, 1) == N.BP_EINVAL
    assert "bp_move_slab" in N.bp_last_error(None)
    assert lib.bp_destroy(None) == N.BP_OK


def test_context_free_calls_validate_arguments(lib):
    assert lib.bp_ramp_filter(4, 0, 1.0, None, None, None) == N.BP_EINVAL
    assert lib.bp_ramp_filter(4, 16, -1.0, None, None, None) == N.BP_EINVAL
    assert lib.bp_row_filter_fwd(4, 16, 0, None, None, None, None) == N.BP_EINVAL
    assert lib.bp_row_filter_fwd(4, 16, 257, None, None, None, None) == N.BP_EINVAL
    assert lib.bp_carm_matrices(-1, None, 785.0, 1200.0, 1.0, 0.0, 0.0, None, None) == N.BP_EINVAL
    assert lib.bp_carm_matrices(3, None, 785.0, 1200.0, 1.0, 0.0, 0.0, None, None) == N.BP_EINVAL
    assert lib.bp_ellipsoid_project(1, None, 8, 8, 1000, None, None, None) == N.BP_EINVAL
    assert "bp_ellipsoid_project" in N.bp_last_error(None)
    # empty work is a no-op that never reaches the GPU
    assert lib.bp_ramp_filter(0, 16, 1.0, None, None, None) == N.BP_OK
    assert lib.bp_row_filter_fwd(0, 16, 8, None, None, None, None) == N.BP_OK
    assert lib.bp_carm_matrices(0, None, 785.0, 1200.0, 1.0, 0.0, 0.0, None, None) == N.BP_OK


def test_bounded_wait_selftest_validates_arguments_without_the_gpu(lib):
    assert lib.bp_selftest_bounded_wait(2, 10) == N.BP_EINVAL
    assert lib.bp_selftest_bounded_wait(0, 0) == N.BP_EINVAL
    assert lib.bp_selftest_bounded_wait(1, (1 << 20) + 1) == N.BP_EINVAL
    assert "bp_selftest_bounded_wait" in N.bp_last_error(None)


def test_create_slab_validates_the_slab_without_the_gpu(lib):
    h = ctypes.c_void_p()
    O = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    for (L, nz, z0) in [(8, 0, 0), (8, 9, 0), (8, 4, -1), (8, 4, 5), (0, 1, 0)]:
        st = lib.bp_create_slab(ctypes.byref(h), L, nz, z0, 1.0, ctypes.cast(O, ctypes.c_void_p), 8, 8, 0, None)
        assert st == N.BP_EINVAL, (L, nz, z0)
        assert h.value is None


def test_slab_reconstruction_validates_its_arguments_without_the_gpu():
    """backproject_slabs refuses a slab of no slices and an output that is not
    a contiguous (L, L, L) float32 host tensor before any device work."""
    torch = pytest.importorskip("torch")
    from paper_1104_5243_gb300 import api
    imgs = torch.zeros((1, 4, 4))
    A = [[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 1]]]
    with pytest.raises(ValueError):
        api.backproject_slabs(8, 1.0, [0, 0, 0], imgs, A, slab=0)
    with pytest.raises(ValueError):
        api.backproject_slabs(8, 1.0, [0, 0, 0], imgs, A, slab=4, out=torch.zeros((8, 8, 7)))
    with pytest.raises(ValueError):
        api.backproject_slabs(8, 1.0, [0, 0, 0], imgs, A, slab=4, out=torch.zeros((8, 8, 8), dtype=torch.float64))
