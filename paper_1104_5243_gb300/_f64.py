"""ctypes binding of the float64 gradient-check library libbp1104_f64.so
(include/bp1104_f64.h) -- TEST SUPPORT ONLY.

The product path computes in float32; this library holds the double
instantiations of the direct backprojection and direct adjoint kernels
(csrc/bp_direct.cuh), so that torch.autograd.gradcheck can check the
differentiable backprojection in float64 with its default step and
tolerances.  ``DirectF64`` offers the calls learned.BackprojectFn makes on a
Backprojector (reset, add_projections, finalize, adjoint).  Argument
marshalling only; raises if the library was never built.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

_vp, _i, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
SIGNATURES = {
    "bp_f64_backproject": (_i, [_i, _d, _vp, _i, _i, _vp, _vp, _i, _vp, _vp]),
    "bp_f64_adjoint": (_i, [_i, _d, _vp, _i, _i, _vp, _vp, _i, _vp, _vp]),
    "bp_f64_last_error": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB_F64
            if not os.path.exists(path):
                raise ImportError(f"{path} is not built; run paper_1104_5243_gb300.build.build_f64()")
            cdll = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(cdll, name)
                fn.restype, fn.argtypes = res, args
            _lib = cdll
    return _lib


def _check(status: int):
    if status != 0:
        raise RuntimeError(f"status {status}: {lib().bp_f64_last_error().decode()}")


def _stream():
    s = torch.cuda.current_stream().cuda_stream
    return ctypes.c_void_p(s) if s else None


def _f64(t: torch.Tensor, name: str) -> torch.Tensor:
    if t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a float64 CUDA tensor, got {t.dtype} on {t.device}")
    return t.contiguous()


class DirectF64:
    """The L^3 backprojection and its transpose in float64 on the GPU, with
    the calls learned.BackprojectFn makes on a Backprojector."""

    def __init__(self, L: int, R: float, O, isx: int, isy: int):
        self.L, self.R, self.isx, self.isy = int(L), float(R), int(isx), int(isy)
        self._O = (ctypes.c_double * 3)(*[float(v) for v in O])
        self.vol = torch.zeros((self.L,) * 3, dtype=torch.float64, device="cuda")

    def reset(self):
        self.vol.zero_()

    def add_projections(self, images: torch.Tensor, A) -> None:
        images = _f64(images, "images")
        A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
        n = A.shape[0]
        if tuple(images.shape) != (n, self.isy, self.isx):
            raise ValueError(f"images must have shape {(n, self.isy, self.isx)}")
        _check(lib().bp_f64_backproject(self.L, self.R, self._O, self.isx, self.isy,
                                        ctypes.c_void_p(images.data_ptr()), ctypes.c_void_p(A.ctypes.data), n,
                                        ctypes.c_void_p(self.vol.data_ptr()), _stream()))

    def finalize(self) -> torch.Tensor:
        return self.vol.clone()

    def adjoint(self, vol: torch.Tensor, A) -> torch.Tensor:
        vol = _f64(vol, "vol")
        A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
        n = A.shape[0]
        out = torch.zeros((n, self.isy, self.isx), dtype=torch.float64, device="cuda")
        _check(lib().bp_f64_adjoint(self.L, self.R, self._O, self.isx, self.isy, ctypes.c_void_p(vol.data_ptr()),
                                    ctypes.c_void_p(A.ctypes.data), n, ctypes.c_void_p(out.data_ptr()), _stream()))
        return out
