"""FP64 CPU oracle for the cone-beam backprojection -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does: it
shares no code, header, table or helper with the oracle.  The arithmetic is in
``bp_oracle.c`` (plain C, FP64, OpenMP over independent outputs); this module
compiles it on first use and wraps it for numpy.

Every function cites the paper passage it follows; the pins that tie it to
something other than itself are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libbp_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_LL = ctypes.POINTER(ctypes.c_longlong)


def build(force: bool = False) -> str:
    """Compile bp_oracle.c into a shared library (gcc, FP64, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call([
            "gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
            "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i, d, ll = ctypes.c_int, ctypes.c_double, ctypes.c_longlong
            sig = {
                "orc_carm_matrices": [i, _D, d, d, d, d, d, _D],
                "orc_backproject": [i, d, _D, i, i, i, _F, _D, _D],
                "orc_backproject_voxels": [i, d, _D, i, i, i, _F, _D, ll, _LL, _D],
                "orc_adjoint": [i, d, _D, i, i, i, _D, _D, _D],
                "orc_source_position": [i, _D, _D],
                "orc_ellipsoid_project": [i, _D, i, i, i, _D, _D],
                "orc_ellipsoid_voxelize": [i, d, _D, i, _D, _D],
                "orc_fdk_preweight": [i, i, i, d, d, d, d, _D, i, d, _D, _D],
                "orc_ramp_filter": [ll, i, d, _D, _D],
                "orc_row_filter_fwd": [ll, i, i, _D, _D, _D],
                "orc_row_filter_bwd": [ll, i, i, _D, _D, _D, _D, _D],
                "orc_ramlak": [ll, d],
                "orc_parker": [d, d, d],
                "orc_num_threads": [],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = None
            lib.orc_ramlak.restype = d
            lib.orc_parker.restype = d
            lib.orc_num_threads.restype = i
            _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _f(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(_F)


def num_threads() -> int:
    return _load().orc_num_threads()


def carm_matrices(scan) -> np.ndarray:
    """3x4 projection matrices (n, 3, 4) float64 for a circular C-arm scan,
    normalised so that w = depth / SID (rows: uw, vw, w)."""
    betas, pb = _d(scan.betas)
    A = np.zeros((scan.n, 3, 4), dtype=np.float64)
    _load().orc_carm_matrices(scan.n, pb, scan.sid, scan.sdd, scan.pitch, scan.cu, scan.cv,
                              A.ctypes.data_as(_D))
    return A


def backproject(vol_shape_L: int, R: float, O, images, A, vol=None) -> np.ndarray:
    """Sect. 3.1, Listing 1: VOL[x] += bilinear(I_i, A_i x) / w^2 over all i.

    images: (n, isy, isx) float32; A: (n, 3, 4) float64.  Returns (L, L, L)
    float64 indexed [z, y, x] (accumulated into ``vol`` when given).
    """
    L = vol_shape_L
    images, pi = _f(images)
    n, isy, isx = images.shape
    A, pa = _d(A)
    assert A.shape == (n, 3, 4)
    Oa, po = _d(np.asarray(O, dtype=np.float64))
    if vol is None:
        vol = np.zeros((L, L, L), dtype=np.float64)
    assert vol.dtype == np.float64 and vol.flags.c_contiguous and vol.shape == (L, L, L)
    _load().orc_backproject(L, R, po, isx, isy, n, pi, pa, vol.ctypes.data_as(_D))
    return vol


def backproject_voxels(L: int, R: float, O, images, A, idx) -> np.ndarray:
    """Listing 1's sum evaluated only at flat voxel indices idx (z*L*L+y*L+x)."""
    images, pi = _f(images)
    n, isy, isx = images.shape
    A, pa = _d(A)
    Oa, po = _d(np.asarray(O, dtype=np.float64))
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(idx.shape[0], dtype=np.float64)
    _load().orc_backproject_voxels(L, R, po, isx, isy, n, pi, pa, idx.shape[0],
                                   idx.ctypes.data_as(_LL), out.ctypes.data_as(_D))
    return out


def adjoint(L: int, R: float, O, vol, A, isx: int, isy: int) -> np.ndarray:
    """Transpose of ``backproject``: (n, isy, isx) float64 projections."""
    vol, pv = _d(vol)
    assert vol.shape == (L, L, L)
    A, pa = _d(A)
    n = A.shape[0]
    Oa, po = _d(np.asarray(O, dtype=np.float64))
    out = np.zeros((n, isy, isx), dtype=np.float64)
    _load().orc_adjoint(L, R, po, isx, isy, n, pv, pa, out.ctypes.data_as(_D))
    return out


def source_positions(A) -> np.ndarray:
    """Source S_i with A_i (S_i, 1) = 0, shape (n, 3)."""
    A, pa = _d(A)
    S = np.zeros((A.shape[0], 3), dtype=np.float64)
    _load().orc_source_position(A.shape[0], pa, S.ctypes.data_as(_D))
    return S


def ellipsoid_project(A, isx: int, isy: int, ell) -> np.ndarray:
    """Analytic line integrals of an additive ellipsoid phantom, (n, isy, isx)."""
    A, pa = _d(A)
    ell, pe = _d(ell)
    out = np.zeros((A.shape[0], isy, isx), dtype=np.float64)
    _load().orc_ellipsoid_project(A.shape[0], pa, isx, isy, ell.shape[0], pe, out.ctypes.data_as(_D))
    return out


def ellipsoid_voxelize(L: int, R: float, O, ell) -> np.ndarray:
    """Phantom density sampled at voxel centres, (L, L, L) [z, y, x]."""
    ell, pe = _d(ell)
    Oa, po = _d(np.asarray(O, dtype=np.float64))
    vol = np.zeros((L, L, L), dtype=np.float64)
    _load().orc_ellipsoid_voxelize(L, R, po, ell.shape[0], pe, vol.ctypes.data_as(_D))
    return vol


def fdk_preweight(scan, proj, parker: bool = True, scale: float = 1.0) -> np.ndarray:
    """Cosine (and Parker short-scan) pre-weighting of projections, FP64."""
    proj, pp = _d(proj)
    betas, pb = _d(scan.betas)
    out = np.zeros_like(proj)
    _load().orc_fdk_preweight(scan.n, scan.isx, scan.isy, scan.pitch, scan.sdd, scan.cu, scan.cv,
                              pb, int(parker), scale, pp, out.ctypes.data_as(_D))
    return out


def ramlak(m: int, tau: float) -> float:
    return _load().orc_ramlak(int(m), float(tau))


def parker(b: float, g: float, delta: float) -> float:
    """Parker short-scan weight of the ray with scan angle b and fan angle g."""
    return _load().orc_parker(float(b), float(g), float(delta))


def ramp_filter(proj, tau: float) -> np.ndarray:
    """Row-wise zero-padded linear convolution with the Ram-Lak kernel."""
    proj, pp = _d(proj)
    isx = proj.shape[-1]
    out = np.zeros_like(proj)
    _load().orc_ramp_filter(proj.size // isx, isx, tau, pp, out.ctypes.data_as(_D))
    return out


def row_filter_fwd(x, h) -> np.ndarray:
    """out[r, j] = sum_t h[t] x[r, j + t - T//2] (zero outside the row)."""
    x, px = _d(x)
    h, ph = _d(h)
    isx = x.shape[-1]
    out = np.zeros_like(x)
    _load().orc_row_filter_fwd(x.size // isx, isx, h.shape[0], ph, px, out.ctypes.data_as(_D))
    return out


def row_filter_bwd(x, h, g):
    """(dL/dx, dL/dh) of ``row_filter_fwd`` given dL/dout = g."""
    x, px = _d(x)
    h, ph = _d(h)
    g, pg = _d(g)
    isx = x.shape[-1]
    gin = np.zeros_like(x)
    gh = np.zeros_like(h)
    _load().orc_row_filter_bwd(x.size // isx, isx, h.shape[0], ph, px, pg,
                               gin.ctypes.data_as(_D), gh.ctypes.data_as(_D))
    return gin, gh


def fdk_scale(scan) -> float:
    """Angular step of the short scan (radians), the FDK integral's d(beta)."""
    return float(np.radians(scan.scan_deg) / max(scan.n - 1, 1))


def iso_pitch(scan) -> float:
    """Detector pitch scaled to the isocenter plane, tau = pitch * SID / SDD."""
    return scan.pitch * scan.sid / scan.sdd


def fdk_filter(scan, line_integrals, parker: bool = True) -> np.ndarray:
    """FDK preprocessing: cosine + Parker pre-weight, ramp filter, d(beta)."""
    pre = fdk_preweight(scan, line_integrals, parker=parker, scale=fdk_scale(scan))
    return ramp_filter(pre, iso_pitch(scan))


def psnr(V, Rf) -> float:
    """Sect. 7.2: 10 log10(M^2 / mean((V - R)^2)); both shifted by min(R) and
    M = max(R) - min(R) (the paper leaves the scaling interval unstated)."""
    V = np.asarray(V, dtype=np.float64)
    Rf = np.asarray(Rf, dtype=np.float64)
    lo = Rf.min()
    M = Rf.max() - lo
    mse = np.mean(((V - lo) - (Rf - lo)) ** 2)
    if mse == 0:
        return float("inf")
    return float(10.0 * np.log10(M * M / mse))


def rel_l2(V, Rf) -> float:
    V = np.asarray(V, dtype=np.float64)
    Rf = np.asarray(Rf, dtype=np.float64)
    return float(np.linalg.norm((V - Rf).ravel()) / np.linalg.norm(Rf.ravel()))
