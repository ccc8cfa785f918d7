"""The allocation-free row-filter gradient, bp_row_filter_bwd_noalloc.

It exists for callers that must not allocate device memory while running
(a reconstruction loop with its device memory budgeted at start-up, or a
framework whose allocator owns the device): its scratch is a fixed array
inside the library instead of a per-call allocation.  Checked here through
the C ABI against the regular entry point and against the FP64 oracle, on
two calls in a row, at the learned filter's training size, on the empty and
partial-output cases, and for the property it exists for: the device's
default memory pool sees no allocation from it (the regular entry point's
stream-ordered scratch shows up there, as a control).

This file is named to be collected last, so that a run stopping at its first
failure has run every other test before it; it also passes on its own in a
fresh process.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle

from gpu_common import native, rel_l2, torch

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    s = torch.cuda.current_stream().cuda_stream
    return ctypes.c_void_p(s) if s else None


def regular(x, h, g, need_gin=True, need_gh=True):
    native()
    from paper_1104_5243_gb300 import _native as N
    rows, isx, T = x.numel() // x.shape[-1], x.shape[-1], h.numel()
    gin = torch.full_like(x, np.nan) if need_gin else None
    gh = torch.full_like(h, np.nan) if need_gh else None
    N.check(N.lib().bp_row_filter_bwd(rows, isx, T, _p(h), _p(x), _p(g), _p(gin), _p(gh), _stream()))
    return gin, gh


def noalloc(x, h, g, need_gin=True, need_gh=True):
    native()
    from paper_1104_5243_gb300 import _native as N
    rows, isx, T = x.numel() // x.shape[-1], x.shape[-1], h.numel()
    gin = torch.full_like(x, np.nan) if need_gin else None
    gh = torch.full_like(h, np.nan) if need_gh else None
    N.check(N.lib().bp_row_filter_bwd_noalloc(rows, isx, T, _p(h), _p(x), _p(g), _p(gin), _p(gh), _stream()))
    return gin, gh


def case(seed, rows, isx, T):
    rng = np.random.default_rng(seed)
    x, h, g = (rng.standard_normal(s).astype(np.float32) for s in ((rows, isx), (T,), (rows, isx)))
    return (x, h, g), tuple(torch.from_numpy(a).cuda() for a in (x, h, g))


@pytest.mark.parametrize("rows,isx,T", [(8 * 240, 312, 64), (37, 53, 128), (3, 16, 1)])
def test_noalloc_matches_regular_entry_point_and_oracle_twice_in_a_row(rows, isx, T):
    # two calls in a row with different data: the second must not see the
    # first call's scratch contents
    for seed in (1, 2):
        (xn, hn, gn), (x, h, g) = case(seed + rows, rows, isx, T)
        ref_gin, ref_gh = regular(x, h, g)
        gin, gh = noalloc(x, h, g)
        torch.cuda.synchronize()
        o_gin, o_gh = oracle.row_filter_bwd(xn, hn, gn)
        assert rel_l2(gin.cpu().numpy(), ref_gin.cpu().numpy()) <= 1e-5
        assert rel_l2(gh.cpu().numpy(), ref_gh.cpu().numpy()) <= 1e-5
        assert rel_l2(gin.cpu().numpy(), o_gin) <= 1e-5
        assert rel_l2(gh.cpu().numpy(), o_gh) <= 1e-5


def test_noalloc_at_the_training_size_against_the_oracle():
    """The learned filter's training batch: 8 phantoms x 120 projections x
    240 rows of 312 pixels, 64 taps (230400 rows).  The fixed grid of 256
    blocks gives each thread about 900 row groups; summing each group
    separately keeps the tap gradient within 1e-5 of the FP64 oracle."""
    rows, isx, T = 8 * 120 * 240, 312, 64
    (xn, hn, gn), (x, h, g) = case(7, rows, isx, T)
    gin, gh = noalloc(x, h, g)
    torch.cuda.synchronize()
    o_gin, o_gh = oracle.row_filter_bwd(xn, hn, gn)
    e_gh, e_gin = rel_l2(gh.cpu().numpy(), o_gh), rel_l2(gin.cpu().numpy(), o_gin)
    print(f"training size: gh rel-L2 {e_gh:.2e}, gin rel-L2 {e_gin:.2e}")
    assert e_gh <= 1e-5 and e_gin <= 1e-5


def test_noalloc_partial_outputs_and_empty_input():
    (xn, hn, gn), (x, h, g) = case(3, 41, 60, 16)
    o_gin, o_gh = oracle.row_filter_bwd(xn, hn, gn)
    gin, gh = noalloc(x, h, g, need_gh=False)
    assert gh is None and rel_l2(gin.cpu().numpy(), o_gin) <= 1e-5
    gin, gh = noalloc(x, h, g, need_gin=False)
    assert gin is None and rel_l2(gh.cpu().numpy(), o_gh) <= 1e-5
    # no rows: the tap gradient is zero, and nothing else is touched
    gin, gh = noalloc(x[:0], h, g[:0])
    torch.cuda.synchronize()
    assert gin.numel() == 0 and torch.equal(gh.cpu(), torch.zeros(16))


def test_noalloc_rejects_filters_larger_than_its_scratch():
    native()
    from paper_1104_5243_gb300 import _native as N
    st = N.lib().bp_row_filter_bwd_noalloc(4, 16, 129, None, None, None, None, None, None)
    assert st == N.BP_EINVAL
    assert "scratch" in N.bp_last_error(None)


class DefaultPool:
    """High-water mark of the device's default memory pool (the pool that
    cudaMallocAsync draws from), read and reset through the CUDA runtime."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8     # cudaMemPoolAttrUsedMemCurrent / UsedMemHigh

    def __init__(self, device: int):
        home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
        for name in (os.path.join(home, "lib64", "libcudart.so"), "libcudart.so.13", "libcudart.so"):
            try:
                self.rt = ctypes.CDLL(name)
                break
            except OSError:
                continue
        else:
            pytest.skip("CUDA runtime library not found")
        self.pool = ctypes.c_void_p()
        assert self.rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool), device) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0


def test_noalloc_draws_nothing_from_the_stream_ordered_pool():
    """The entry point's reason to exist: the regular gradient's scratch shows
    up in the default pool's high-water mark; the allocation-free one's does
    not (its first call in this process included)."""
    (xn, hn, gn), (x, h, g) = case(11, 4096, 312, 64)
    pool = DefaultPool(torch.cuda.current_device())
    torch.cuda.synchronize()
    base = pool.get(pool.USED_MEM_CURRENT)
    pool.reset_high()
    noalloc(x, h, g)
    noalloc(x, h, g)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) == base
    regular(x, h, g)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) >= base + 1024 * 64 * 4   # 1024 row blocks x 64 taps
