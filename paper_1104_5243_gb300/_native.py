"""ctypes binding of libbp1104.so (include/bp1104.h): argument marshalling
only, with the C ABI's names.  There is no fallback: if the CUDA library is
not built, every entry point raises."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

BP_OK, BP_EINVAL, BP_ENOMEM, BP_ECUDA, BP_ESTATE, BP_ETIMEOUT = range(6)
BP_F32, BP_F16, BP_BF16 = 0, 1, 2
BP_OPT_IEEE_RCP, BP_OPT_BATCH, BP_OPT_TIMING, BP_OPT_LANES_X, BP_OPT_PATH, BP_OPT_CULL = 1, 2, 3, 4, 5, 6
BP_OPT_HOST_DIRECT, BP_OPT_BLOCK_CENTRE, BP_OPT_BRICK_DEPTH, BP_OPT_PROJ_SCALE = 7, 8, 9, 10
BP_QUERY_LAST_PATH, BP_QUERY_PROJECTIONS_ADDED, BP_QUERY_UPDATES_COMPUTED, BP_QUERY_LAST_BRICK_DEPTH = 1, 2, 3, 4
BP_QUERY_LAST_LANES_X = 5
STATUS_NAMES = {0: "BP_OK", 1: "BP_EINVAL", 2: "BP_ENOMEM", 3: "BP_ECUDA", 4: "BP_ESTATE", 5: "BP_ETIMEOUT"}

# Every symbol include/bp1104.h declares, with (restype, argtypes).
_vp, _i, _ll, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
SIGNATURES = {
    "bp_create": (_i, [ctypes.POINTER(_vp), _i, _d, _vp, _i, _i, _i, _vp]),
    "bp_create_slab": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _d, _vp, _i, _i, _i, _vp]),
    "bp_destroy": (_i, [_vp]),
    "bp_move_slab": (_i, [_vp, _i, _i]),
    "bp_set_option": (_i, [_vp, _i, _ll]),
    "bp_reset": (_i, [_vp]),
    "bp_add_projections": (_i, [_vp, _vp, _i, _vp, _i]),
    "bp_finalize": (_i, [_vp, _vp, _i]),
    "bp_add_projections_finalize": (_i, [_vp, _vp, _i, _vp, _i, _vp, _i]),
    "bp_get_state": (_i, [_vp, _vp, _i, ctypes.POINTER(_ll)]),
    "bp_set_state": (_i, [_vp, _vp, _i, _ll]),
    "bp_adjoint": (_i, [_vp, _vp, _i, _vp, _i, _vp, _i]),
    "bp_kernel_stats": (_i, [_vp, ctypes.POINTER(_ll), ctypes.POINTER(_d)]),
    "bp_query": (_i, [_vp, _i, ctypes.POINTER(_ll)]),
    "bp_probe_gather": (_i, [_i, ctypes.POINTER(_d)]),
    "bp_selftest_bounded_wait": (_i, [_i, _i]),
    "bp_last_error": (ctypes.c_char_p, [_vp]),
    "bp_carm_matrices": (_i, [_i, _vp, _d, _d, _d, _d, _d, _vp, _vp]),
    "bp_ellipsoid_project": (_i, [_i, _vp, _i, _i, _i, _vp, _vp, _vp]),
    "bp_ellipsoid_voxelize": (_i, [_i, _d, _vp, _i, _vp, _vp, _vp]),
    "bp_fdk_preweight": (_i, [_i, _i, _i, _d, _d, _d, _d, _vp, _i, _d, _vp, _vp, _vp]),
    "bp_ramp_filter": (_i, [_ll, _i, _d, _vp, _vp, _vp]),
    "bp_row_filter_fwd": (_i, [_ll, _i, _i, _vp, _vp, _vp, _vp]),
    "bp_row_filter_bwd": (_i, [_ll, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "bp_row_filter_bwd_noalloc": (_i, [_ll, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
}

_lock = threading.Lock()
_lib = None


class BpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libbp1104.so (raises if it was never built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise ImportError(
                    f"CUDA library {path} is not built; run paper_1104_5243_gb300.build.build() "
                    "(there is no CPU fallback)")
            cdll = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(cdll, name)
                fn.restype = res
                fn.argtypes = args
            _lib = cdll
    return _lib


def check(status: int, ctx=None) -> None:
    if status != BP_OK:
        msg = lib().bp_last_error(ctx)
        raise BpError(status, msg.decode() if msg else "")


def _dbl3(O):
    return (ctypes.c_double * 3)(*[float(v) for v in O])


# ---- thin wrappers with the ABI's names (pointers are ints / None) ----------
def bp_create(L, R, O, isx, isy, dtype=BP_F32, stream=None):
    h = _vp()
    check(lib().bp_create(ctypes.byref(h), int(L), float(R), ctypes.cast(_dbl3(O), _vp),
                          int(isx), int(isy), int(dtype), stream))
    return h.value


def bp_create_slab(L, nz, z0, R, O, isx, isy, dtype=BP_F32, stream=None):
    h = _vp()
    check(lib().bp_create_slab(ctypes.byref(h), int(L), int(nz), int(z0), float(R), ctypes.cast(_dbl3(O), _vp),
                               int(isx), int(isy), int(dtype), stream))
    return h.value


def bp_destroy(ctx):
    check(lib().bp_destroy(ctx))


def bp_move_slab(ctx, z0, nz):
    check(lib().bp_move_slab(ctx, int(z0), int(nz)), ctx)


def bp_set_option(ctx, option, value):
    check(lib().bp_set_option(ctx, int(option), int(value)), ctx)


def bp_reset(ctx):
    check(lib().bp_reset(ctx), ctx)


def bp_add_projections(ctx, images_ptr, images_on_device, A_ptr, n):
    check(lib().bp_add_projections(ctx, images_ptr, int(images_on_device), A_ptr, int(n)), ctx)


def bp_finalize(ctx, vol_ptr, on_device):
    check(lib().bp_finalize(ctx, vol_ptr, int(on_device)), ctx)


def bp_add_projections_finalize(ctx, images_ptr, images_on_device, A_ptr, n, vol_ptr, out_on_device):
    check(lib().bp_add_projections_finalize(ctx, images_ptr, int(images_on_device), A_ptr, int(n), vol_ptr,
                                            int(out_on_device)), ctx)


def bp_get_state(ctx, vol_ptr, on_device):
    n = _ll(0)
    check(lib().bp_get_state(ctx, vol_ptr, int(on_device), ctypes.byref(n)), ctx)
    return n.value


def bp_set_state(ctx, vol_ptr, on_device, n_added):
    check(lib().bp_set_state(ctx, vol_ptr, int(on_device), int(n_added)), ctx)


def bp_adjoint(ctx, vol_ptr, vol_on_device, A_ptr, n, out_ptr, out_on_device):
    check(lib().bp_adjoint(ctx, vol_ptr, int(vol_on_device), A_ptr, int(n), out_ptr,
                           int(out_on_device)), ctx)


def bp_query(ctx, what) -> int:
    v = _ll(0)
    check(lib().bp_query(ctx, int(what), ctypes.byref(v)), ctx)
    return v.value


def bp_kernel_stats(ctx):
    n, ms = _ll(0), _d(0.0)
    check(lib().bp_kernel_stats(ctx, ctypes.byref(n), ctypes.byref(ms)), ctx)
    return n.value, ms.value


def bp_probe_gather(dtype) -> float:
    """Texture 2x2-gather rate (gathers per SM per clock) for a storage type."""
    r = _d(0.0)
    check(lib().bp_probe_gather(int(dtype), ctypes.byref(r)))
    return r.value


def bp_selftest_bounded_wait(arrive: bool, iters: int) -> int:
    """Status of the bounded-wait self-test (BP_OK or BP_ETIMEOUT; other
    statuses raise)."""
    st = lib().bp_selftest_bounded_wait(int(bool(arrive)), int(iters))
    if st not in (BP_OK, BP_ETIMEOUT):
        check(st)
    return st


def bp_last_error(ctx=None) -> str:
    return lib().bp_last_error(ctx).decode()


def bp_carm_matrices(n, beta_ptr, sid, sdd, pitch, cu, cv, A_out_ptr, stream=None):
    check(lib().bp_carm_matrices(int(n), beta_ptr, float(sid), float(sdd), float(pitch), float(cu),
                                 float(cv), A_out_ptr, stream))


def bp_ellipsoid_project(n, A_ptr, isx, isy, count, ell_ptr, out_ptr, stream=None):
    check(lib().bp_ellipsoid_project(int(n), A_ptr, int(isx), int(isy), int(count), ell_ptr, out_ptr,
                                     stream))


def bp_ellipsoid_voxelize(L, R, O, count, ell_ptr, vol_ptr, stream=None):
    check(lib().bp_ellipsoid_voxelize(int(L), float(R), ctypes.cast(_dbl3(O), _vp), int(count),
                                      ell_ptr, vol_ptr, stream))


def bp_fdk_preweight(n, isx, isy, pitch, sdd, cu, cv, beta_ptr, parker, scale, in_ptr, out_ptr,
                     stream=None):
    check(lib().bp_fdk_preweight(int(n), int(isx), int(isy), float(pitch), float(sdd), float(cu),
                                 float(cv), beta_ptr, int(parker), float(scale), in_ptr, out_ptr,
                                 stream))


def bp_ramp_filter(rows, isx, tau, in_ptr, out_ptr, stream=None):
    check(lib().bp_ramp_filter(int(rows), int(isx), float(tau), in_ptr, out_ptr, stream))


def bp_row_filter_fwd(rows, isx, T, h_ptr, in_ptr, out_ptr, stream=None):
    check(lib().bp_row_filter_fwd(int(rows), int(isx), int(T), h_ptr, in_ptr, out_ptr, stream))


def bp_row_filter_bwd(rows, isx, T, h_ptr, in_ptr, g_ptr, gin_ptr, gh_ptr, stream=None):
    check(lib().bp_row_filter_bwd(int(rows), int(isx), int(T), h_ptr, in_ptr, g_ptr, gin_ptr, gh_ptr,
                                  stream))


def bp_row_filter_bwd_noalloc(rows, isx, T, h_ptr, in_ptr, g_ptr, gin_ptr, gh_ptr, stream=None):
    """Same as bp_row_filter_bwd, with fixed in-library scratch (no allocation)."""
    check(lib().bp_row_filter_bwd_noalloc(int(rows), int(isx), int(T), h_ptr, in_ptr, g_ptr, gin_ptr,
                                          gh_ptr, stream))
