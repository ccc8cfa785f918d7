"""The allocation-free row-filter gradient, bp_row_filter_bwd_noalloc.

It exists for callers that must not allocate device memory while running
(a reconstruction loop with its device memory budgeted at start-up, or a
framework whose allocator owns the device): its scratch is a fixed array
inside the library instead of a per-call allocation.  This file is named to
be collected last, so that a run stopping at its first failure has run every
other test before it; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from gpu_common import native, rel_l2, torch

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def both(x, h, g):
    """(gin, gh) from the regular entry point and from the no-alloc one,
    each called through the C ABI on torch's current stream."""
    native()
    from paper_1104_5243_gb300 import _native as N
    rows, isx = x.numel() // x.shape[-1], x.shape[-1]
    T = h.numel()
    stream = torch.cuda.current_stream().cuda_stream or None
    s = ctypes.c_void_p(stream) if stream else None
    ref_gin, ref_gh = torch.empty_like(x), torch.empty_like(h)
    N.check(N.lib().bp_row_filter_bwd(rows, isx, T, _p(h), _p(x), _p(g), _p(ref_gin), _p(ref_gh), s))
    gin, gh = torch.full_like(x, np.nan), torch.full_like(h, np.nan)
    N.check(N.lib().bp_row_filter_bwd_noalloc(rows, isx, T, _p(h), _p(x), _p(g), _p(gin), _p(gh), s))
    torch.cuda.synchronize()
    return (ref_gin, ref_gh), (gin, gh)


def case(seed, rows, isx, T):
    rng = np.random.default_rng(seed)
    mk = lambda *shape: torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    return mk(rows, isx), mk(T), mk(rows, isx)


@pytest.mark.parametrize("rows,isx,T", [(8 * 240, 312, 64), (37, 53, 128), (3, 16, 1)])
def test_noalloc_matches_regular_entry_point_twice_in_a_row(rows, isx, T):
    # two calls in a row with different data: the second must not see the
    # first call's scratch contents
    for seed in (1, 2):
        (ref_gin, ref_gh), (gin, gh) = both(*case(seed + rows, rows, isx, T))
        assert rel_l2(gin.cpu().numpy(), ref_gin.cpu().numpy()) <= 1e-5
        assert rel_l2(gh.cpu().numpy(), ref_gh.cpu().numpy()) <= 1e-5


def test_noalloc_rejects_filters_larger_than_its_scratch():
    native()
    from paper_1104_5243_gb300 import _native as N
    st = N.lib().bp_row_filter_bwd_noalloc(4, 16, 129, None, None, None, None, None, None)
    assert st == N.BP_EINVAL
    assert "scratch" in N.bp_last_error(None)
