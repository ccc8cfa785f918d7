"""bp_add_projections_finalize: the images of a scan in, the finished volume
out, in one call (Sect. 3.1).  On the TMA path the last batch's launch also
stores the final values into the destination (device memory, or page-locked
host memory through its mapping).  The result must equal bp_add_projections
followed by bp_finalize bit for bit, for every kind of destination, and the
context must keep the volume; the oracle checks the value itself."""
import numpy as np
import pytest

import oracle
from paper_1104_5243_gb300 import synth

from gpu_common import native, rel_l2, torch

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def case(L=37, n=70):
    scan = synth.Scan(n=n, isx=53, isy=41, pitch=384.0 / 53)
    vol = synth.Volume(L)
    A = oracle.carm_matrices(scan)
    q = np.random.default_rng(L + n).standard_normal((scan.n, scan.isy, scan.isx)).astype(np.float32)
    return scan, vol, A, q


def two_calls(api, N, vol, scan, A, images, dtype, path, nz=None, z0=0):
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=dtype, nz=nz, z0=z0) as bp:
        bp.set_option(N.BP_OPT_PATH, path)
        bp.add_projections(images, A)
        return bp.finalize().cpu()


def destination(kind, shape):
    if kind == "pinned":
        return torch.empty(shape, dtype=torch.float32).pin_memory()
    if kind == "pageable":
        return torch.empty(shape, dtype=torch.float32)
    return torch.empty(shape, dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("dest", ["pinned", "pageable", "device"])
@pytest.mark.parametrize("dtype,path", [("f32", 0), ("f16", 0), ("bf16", 2), ("f32", 1)])
def test_fused_call_equals_add_then_finalize(dest, dtype, path):
    """37^3 from 70 projections of 53 x 41 (two batches, ragged volume and
    detector), host images; every destination kind, the TMA path (direct
    stores) and the texture path (copy after the launch)."""
    api = native()
    from paper_1104_5243_gb300 import _native as N
    scan, vol, A, q = case()
    qh = torch.from_numpy(q).pin_memory()
    ref = two_calls(api, N, vol, scan, A, qh, dtype, path)
    out = destination(dest, (vol.L,) * 3)
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=dtype) as bp:
        bp.set_option(N.BP_OPT_PATH, path)
        got = bp.add_projections_finalize(qh, A, out)
        assert got.data_ptr() == out.data_ptr()
        assert torch.equal(got.cpu(), ref)
        assert torch.equal(bp.finalize().cpu(), ref)       # the context keeps the volume
        # and keeps accumulating onto it
        bp.add_projections_finalize(qh[:5], A[:5], out)
        again = bp.finalize().cpu()
        assert torch.equal(out.cpu(), again)
    if dtype == "f32":
        assert rel_l2(ref.numpy(), oracle.backproject(vol.L, vol.R, vol.O, q, A)) <= FP32_TOL


def test_fused_call_after_reset_and_device_images():
    """Device images, a reset between two fused calls: each call's volume is
    that call's backprojection alone."""
    api = native()
    from paper_1104_5243_gb300 import _native as N
    scan, vol, A, q = case(L=40, n=20)
    qd = torch.from_numpy(q).cuda()
    ref = two_calls(api, N, vol, scan, A, qd, "f32", 0)
    out = destination("pinned", (vol.L,) * 3)
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy) as bp:
        bp.add_projections_finalize(qd, A, out)
        bp.reset()
        bp.add_projections_finalize(qd, A, out)
    assert torch.equal(out, ref)


def test_fused_call_on_a_slab_and_with_no_images():
    """A z-slab context (slices 8 .. 27 of 37^3) writes its L x L x nz volume;
    n = 0 is a plain finalize."""
    api = native()
    from paper_1104_5243_gb300 import _native as N
    scan, vol, A, q = case()
    qh = torch.from_numpy(q).pin_memory()
    ref = two_calls(api, N, vol, scan, A, qh, "f32", 0, nz=20, z0=8)
    whole = two_calls(api, N, vol, scan, A, qh, "f32", 0)
    out = destination("pinned", (20, vol.L, vol.L))
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, nz=20, z0=8) as bp:
        bp.add_projections_finalize(qh, A, out)
        assert torch.equal(out, ref)
        empty = destination("device", (20, vol.L, vol.L))
        bp.add_projections_finalize(qh[:0], A[:0], empty)
        assert torch.equal(empty.cpu(), ref)
    # the slab's bricks need not line up with the cube's, so per-brick
    # centring rounds each differently: two float32 results, each within
    # about 1e-6 of the exact sums
    assert rel_l2(out.numpy(), whole[8:28].numpy()) <= 2.5e-6


def test_fused_call_rejects_a_null_output():
    api = native()
    from paper_1104_5243_gb300 import _native as N
    scan, vol, A, q = case(L=16, n=3)
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy) as bp:
        with pytest.raises(N.BpError) as e:
            N.bp_add_projections_finalize(bp.handle, None, 0, None, 0, None, 0)
        assert e.value.status == N.BP_EINVAL
