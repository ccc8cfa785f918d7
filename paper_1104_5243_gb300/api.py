"""PyTorch-facing wrappers around the C ABI.

PyTorch supplies device memory and the current CUDA stream; every step of
the computation runs in libbp1104.so.  Tensors must be contiguous float32
(matrices float64 numpy arrays, which the ABI reads on the host).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N

_DTYPES = {"f32": N.BP_F32, "f16": N.BP_F16, "bf16": N.BP_BF16}


def _stream_handle(stream=None):
    """cudaStream_t of `stream` (default: torch's current stream); None is
    the legacy default stream, as in the C ABI."""
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream) if s.cuda_stream else None


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32, got {t.dtype}")
    return t.contiguous()


def _matrices(A) -> np.ndarray:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    if A.ndim != 3 or A.shape[1:] != (3, 4):
        raise ValueError(f"matrices must have shape (n, 3, 4), got {A.shape}")
    return A


class Backprojector:
    """An L^3 volume (or, with nz and z0, the z-slab of slices z0 .. z0+nz-1
    of the L^3 grid) accumulating backprojected ISX x ISY projections
    (Sect. 3.1, Listing 1).  Owns the library context.  Volumes are (nz, L, L)
    float32 tensors [z, y, x] (nz = L for the full cube)."""

    def __init__(self, L: int, R: float, O, isx: int, isy: int, dtype: str = "f32",
                 stream: torch.cuda.Stream | None = None, device=None, nz: int | None = None, z0: int = 0):
        self.L, self.R, self.O = int(L), float(R), tuple(float(v) for v in O)
        self.nz, self.z0 = (self.L if nz is None else int(nz)), int(z0)
        self.nz_cap = self.nz   # slab depth the device volume holds (move_slab)
        self.isx, self.isy = int(isx), int(isy)
        self.dtype = dtype
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self._stream = stream
        with torch.cuda.device(self.device):
            if nz is None and self.z0 == 0:
                self._ctx = N.bp_create(self.L, self.R, self.O, self.isx, self.isy, _DTYPES[dtype],
                                        _stream_handle(stream))
            else:
                self._ctx = N.bp_create_slab(self.L, self.nz, self.z0, self.R, self.O, self.isx, self.isy,
                                             _DTYPES[dtype], _stream_handle(stream))

    @property
    def shape(self):
        return (self.nz, self.L, self.L)

    def _volume(self, t: torch.Tensor, name: str) -> torch.Tensor:
        # the library copies nz * L * L floats: refuse a buffer of another size
        t = _f32(t, name)
        if t.numel() != self.nz * self.L * self.L:
            raise ValueError(f"{name} must hold {self.nz} x {self.L} x {self.L} floats, got shape {tuple(t.shape)}")
        return t

    # --------------------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            N.bp_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._ctx

    def set_option(self, option: int, value: int):
        N.bp_set_option(self._ctx, option, value)

    def move_slab(self, z0: int, nz: int):
        """Re-target the context to slices z0 .. z0+nz-1 of the same L^3 grid
        (nz at most the depth it was created with), keeping its device
        allocations; the volume and the counter restart at zero."""
        N.bp_move_slab(self._ctx, z0, nz)
        self.z0, self.nz = int(z0), int(nz)

    def reset(self):
        N.bp_reset(self._ctx)

    def query(self, what: int) -> int:
        """bp_query: N.BP_QUERY_LAST_PATH, _PROJECTIONS_ADDED, _UPDATES_COMPUTED."""
        return N.bp_query(self._ctx, what)

    @property
    def last_path(self) -> str:
        """Data path of the last batch: 'texture', 'tma' or 'none'."""
        return {0: "none", 1: "texture", 2: "tma"}[N.bp_query(self._ctx, N.BP_QUERY_LAST_PATH)]

    def kernel_stats(self):
        """(launches, total ms) of backprojection kernels timed since the
        last call (needs set_option(BP_OPT_TIMING, 1))."""
        return N.bp_kernel_stats(self._ctx)

    def add_projections(self, images: torch.Tensor, A) -> None:
        """VOL += backprojection of images (n, isy, isx) float32 (CUDA or
        host tensor; pin host tensors for overlap) with matrices A (n, 3, 4)."""
        images = _f32(images, "images")
        A = _matrices(A)
        n = A.shape[0]
        if tuple(images.shape) != (n, self.isy, self.isx):
            raise ValueError(f"images must have shape {(n, self.isy, self.isx)}, got {tuple(images.shape)}")
        on_dev = images.is_cuda
        N.bp_add_projections(self._ctx, _ptr(images), on_dev, ctypes.c_void_p(A.ctypes.data), n)
        if not on_dev:
            # the copy may still read the host buffer: keep it alive until finalize
            self._keep = (images, A)

    def finalize(self, out: torch.Tensor | None = None) -> torch.Tensor:
        """The accumulated volume as a (nz, L, L) float32 CUDA tensor [z, y, x]."""
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        out = self._volume(out, "out")
        N.bp_finalize(self._ctx, _ptr(out), out.is_cuda)
        self._keep = None
        return out

    def add_projections_finalize(self, images: torch.Tensor, A, out: torch.Tensor | None = None) -> torch.Tensor:
        """add_projections then finalize in one call: the finished (nz, L, L)
        volume in `out` (CUDA or host tensor; a pinned host tensor receives
        it from the last kernel directly), bit-identical to the two calls."""
        images = _f32(images, "images")
        A = _matrices(A)
        n = A.shape[0]
        if tuple(images.shape) != (n, self.isy, self.isx):
            raise ValueError(f"images must have shape {(n, self.isy, self.isx)}, got {tuple(images.shape)}")
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        out = self._volume(out, "out")
        N.bp_add_projections_finalize(self._ctx, _ptr(images), images.is_cuda, ctypes.c_void_p(A.ctypes.data), n,
                                      _ptr(out), out.is_cuda)
        self._keep = None
        return out

    def get_state(self):
        vol = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        n = N.bp_get_state(self._ctx, _ptr(vol), 1)
        return vol, n

    def set_state(self, vol: torch.Tensor, n_added: int):
        vol = self._volume(vol, "vol")
        N.bp_set_state(self._ctx, _ptr(vol), vol.is_cuda, n_added)

    def adjoint(self, vol: torch.Tensor, A, out: torch.Tensor | None = None) -> torch.Tensor:
        """B^T vol: (n, isy, isx) float32 CUDA tensor."""
        vol = self._volume(vol, "vol")
        A = _matrices(A)
        n = A.shape[0]
        if out is None:
            out = torch.empty((n, self.isy, self.isx), dtype=torch.float32, device=self.device)
        N.bp_adjoint(self._ctx, _ptr(vol), vol.is_cuda, ctypes.c_void_p(A.ctypes.data), n,
                     _ptr(out), out.is_cuda)
        return out


def slab_contexts(L: int, R: float, O, isx: int, isy: int, slab: int, dtype: str = "f32",
                  count: int = 2) -> list:
    """`count` slab contexts of min(slab, L) slices of the L^3 grid, each on
    its own CUDA stream, for backproject_slabs; a caller reconstructing
    several volumes of one geometry keeps them and passes them as `pool`, so
    their device allocations are made once."""
    device = torch.cuda.current_device()
    return [Backprojector(L, R, O, isx, isy, dtype=dtype, nz=min(int(slab), int(L)), z0=0,
                          stream=torch.cuda.Stream(device=device)) for _ in range(int(count))]


def backproject_slabs(L: int, R: float, O, images: torch.Tensor, A, slab: int, dtype: str = "f32",
                      out: torch.Tensor | None = None, contexts: int = 2, pool: list | None = None) -> torch.Tensor:
    """Backproject into an L^3 volume held in HOST memory, slab by slab (the
    paper's split of the z loop, Sect. 6): slab contexts of `slab` slices
    (`contexts` of them made for this call, or the caller's `pool` from
    slab_contexts), moved over the volume with bp_move_slab, take the slabs
    in turn, each on its own CUDA stream and host thread, so one slab's
    staging and read-back overlap the other's kernels; every slab takes every
    projection, and its last launch stores the slab into out[z0 : z0 + nz].
    For volumes larger than the device holds.  images: (n, ISY, ISX)
    float32, host or device; out: (L, L, L) float32 host tensor (allocated
    pinned if None)."""
    from concurrent.futures import ThreadPoolExecutor
    L, slab = int(L), int(slab)
    if slab < 1 or contexts < 1:
        raise ValueError("slab and contexts must be >= 1")
    if out is None:
        out = torch.empty((L, L, L), dtype=torch.float32).pin_memory()
    if out.is_cuda or tuple(out.shape) != (L, L, L) or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous (L, L, L) float32 host tensor")
    n, isy, isx = images.shape
    slabs = [(z0, min(slab, L - z0)) for z0 in range(0, L, slab)]
    if pool is not None:
        if not pool or any(bp.L != L or bp.isx != isx or bp.isy != isy or bp.dtype != dtype or
                           bp.nz_cap < min(slab, L) for bp in pool):
            raise ValueError("pool contexts must match L, the detector, the dtype and hold a slab")
        ctxs = list(pool)[:len(slabs)]
    else:
        ctxs = slab_contexts(L, R, O, isx, isy, slab, dtype, min(contexts, len(slabs)))
    # the contexts' streams read device images produced on the caller's stream
    torch.cuda.current_stream().synchronize()
    device = torch.cuda.current_device()

    def work(k):
        torch.cuda.set_device(device)
        bp = ctxs[k]
        for z0, nz in slabs[k::len(ctxs)]:
            bp.move_slab(z0, nz)
            # out[z0 : z0 + nz] is contiguous: with a pinned `out` the slab's
            # last launch stores it there directly
            bp.add_projections_finalize(images, A, out[z0:z0 + nz])

    try:
        with ThreadPoolExecutor(len(ctxs)) as ex:
            list(ex.map(work, range(len(ctxs))))
    finally:
        if pool is None:
            for bp in ctxs:
                bp.close()
    return out


# ------------------------------------------------------------------------
def carm_matrices(scan, device=None) -> np.ndarray:
    """(n, 3, 4) float64 matrices of a circular C-arm scan, built in FP64 on
    the GPU and returned on the host."""
    betas = np.ascontiguousarray(scan.betas, dtype=np.float64)
    out = torch.empty((scan.n, 3, 4), dtype=torch.float64,
                      device=device or torch.device("cuda", torch.cuda.current_device()))
    N.bp_carm_matrices(scan.n, ctypes.c_void_p(betas.ctypes.data), scan.sid, scan.sdd, scan.pitch,
                       scan.cu, scan.cv, _ptr(out), _stream_handle())
    return out.cpu().numpy()


def ellipsoid_project(A, isx: int, isy: int, ell) -> torch.Tensor:
    """Analytic line integrals (n, isy, isx) float32 of an ellipsoid phantom."""
    dev = torch.device("cuda", torch.cuda.current_device())
    At = torch.as_tensor(_matrices(A), device=dev).contiguous()
    et = torch.as_tensor(np.asarray(ell, dtype=np.float64), device=dev).contiguous()
    out = torch.empty((At.shape[0], isy, isx), dtype=torch.float32, device=dev)
    N.bp_ellipsoid_project(At.shape[0], _ptr(At), isx, isy, et.shape[0], _ptr(et), _ptr(out),
                           _stream_handle())
    return out


def ellipsoid_voxelize(L: int, R: float, O, ell) -> torch.Tensor:
    dev = torch.device("cuda", torch.cuda.current_device())
    et = torch.as_tensor(np.asarray(ell, dtype=np.float64), device=dev).contiguous()
    out = torch.empty((L, L, L), dtype=torch.float32, device=dev)
    N.bp_ellipsoid_voxelize(L, R, O, et.shape[0], _ptr(et), _ptr(out), _stream_handle())
    return out


def fdk_preweight(scan, proj: torch.Tensor, parker: bool = True, scale: float = 1.0,
                  out: torch.Tensor | None = None) -> torch.Tensor:
    proj = _f32(proj, "proj")
    betas = np.ascontiguousarray(scan.betas, dtype=np.float64)
    if out is None:
        out = torch.empty_like(proj)
    N.bp_fdk_preweight(scan.n, scan.isx, scan.isy, scan.pitch, scan.sdd, scan.cu, scan.cv,
                       ctypes.c_void_p(betas.ctypes.data), int(parker), scale, _ptr(proj),
                       _ptr(out), _stream_handle())
    return out


def ramp_filter(x: torch.Tensor, tau: float) -> torch.Tensor:
    x = _f32(x, "x")
    out = torch.empty_like(x)
    isx = x.shape[-1]
    N.bp_ramp_filter(x.numel() // isx, isx, tau, _ptr(x), _ptr(out), _stream_handle())
    return out


def fdk_scale(scan) -> float:
    """d(beta) of the short scan, the FDK angular integration weight."""
    return float(np.radians(scan.scan_deg) / max(scan.n - 1, 1))


def iso_pitch(scan) -> float:
    """Detector pitch scaled to the isocenter plane."""
    return scan.pitch * scan.sid / scan.sdd


def fdk_filter(scan, line_integrals: torch.Tensor, parker: bool = True) -> torch.Tensor:
    """FDK pre-processing on the GPU: cosine + Parker weights, ramp filter."""
    pre = fdk_preweight(scan, line_integrals, parker=parker, scale=fdk_scale(scan))
    return ramp_filter(pre, iso_pitch(scan))


def row_filter_fwd(x: torch.Tensor, h: torch.Tensor) -> torch.Tensor:
    x, h = _f32(x, "x"), _f32(h, "h")
    out = torch.empty_like(x)
    isx = x.shape[-1]
    N.bp_row_filter_fwd(x.numel() // isx, isx, h.numel(), _ptr(h), _ptr(x), _ptr(out), _stream_handle())
    return out


def row_filter_bwd(x: torch.Tensor, h: torch.Tensor, g: torch.Tensor, need_x=True, need_h=True):
    x, h, g = _f32(x, "x"), _f32(h, "h"), _f32(g, "g")
    gin = torch.empty_like(x) if need_x else None
    gh = torch.empty_like(h) if need_h else None
    isx = x.shape[-1]
    N.bp_row_filter_bwd(x.numel() // isx, isx, h.numel(), _ptr(h), _ptr(x), _ptr(g),
                        _ptr(gin) if gin is not None else None, _ptr(gh) if gh is not None else None,
                        _stream_handle())
    return gin, gh
