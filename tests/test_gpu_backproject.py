"""GPU parity of the backprojection (CUDA, through the C ABI) against the FP64
oracle on seeded inputs: element by element on small and ragged cases, on
sampled voxels at the full 512^3 x 496 x 1248x960 size, plus the storage
forms, options, streaming, checkpoint/resume and edge cases.

Tolerances (stated per case): FP32 path rel-L2 <= 1e-5 against the oracle;
FP16 storage <= 1e-3; BF16 storage reported with a loose bound (8 mantissa
bits give about 2e-3 per pixel)."""
import numpy as np
import pytest

import oracle
from paper_1104_5243_gb300 import synth

from gpu_common import native, rel_l2, tiny_phantom_case, torch

pytestmark = pytest.mark.gpu

FP32_TOL, FP16_TOL, BF16_TOL = 1e-5, 1e-3, 1e-2


def run_gpu(vol, scan, A, q, dtype="f32", batch=None, ieee=False, on_device=True, chunks=None):
    api = native()
    from paper_1104_5243_gb300 import _native as N
    bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=dtype)
    if batch is not None:
        bp.set_option(N.BP_OPT_BATCH, batch)
    if ieee:
        bp.set_option(N.BP_OPT_IEEE_RCP, 1)
    qt = torch.from_numpy(np.ascontiguousarray(q))
    qt = qt.cuda() if on_device else qt.pin_memory()
    bounds = chunks or [(0, A.shape[0])]
    for (a, b) in bounds:
        bp.add_projections(qt[a:b], A[a:b])
    out = bp.finalize().cpu().numpy()
    bp.close()
    return out


def test_tiny_phantom_fp32_matches_oracle():
    scan, vol, A, ell, q, ref = tiny_phantom_case()
    got = run_gpu(vol, scan, A, q)
    err = rel_l2(got, ref)
    mabs = float(np.abs(got - ref).max() / np.abs(ref).max())
    print(f"tiny fp32 rel-L2 {err:.3e} max-abs {np.abs(got - ref).max():.3e} (relative {mabs:.3e}) "
          f"PSNR {oracle.psnr(got, ref):.1f} dB")
    assert err <= FP32_TOL
    # ramp-filtered data mixes signs: single voxels may carry more of the
    # error than the rel-L2 shows, so the max-abs bar is 4x the rel-L2 bar
    assert mabs <= 4 * FP32_TOL


@pytest.mark.parametrize("dtype,tol", [("f16", FP16_TOL), ("bf16", BF16_TOL)])
def test_tiny_phantom_16bit_storage(dtype, tol):
    scan, vol, A, ell, q, ref = tiny_phantom_case()
    got = run_gpu(vol, scan, A, q, dtype=dtype)
    err = rel_l2(got, ref)
    mabs = float(np.abs(got - ref).max() / np.abs(ref).max())
    print(f"tiny {dtype} rel-L2 {err:.3e} max-abs {np.abs(got - ref).max():.3e} (relative {mabs:.3e}) "
          f"PSNR {oracle.psnr(got, ref):.1f} dB")
    assert err <= tol and mabs <= 4 * tol


def test_ieee_reciprocal_option():
    scan, vol, A, ell, q, ref = tiny_phantom_case()
    got = run_gpu(vol, scan, A, q, ieee=True)
    assert rel_l2(got, ref) <= FP32_TOL


@pytest.mark.parametrize("L,isx,isy,n,batch", [
    (37, 53, 41, 70, None),     # ragged volume/detector, two passes
    (40, 160, 120, 9, 4),       # L % 4 == 0 but not a tile multiple, small batches
    (1, 7, 5, 3, None),         # single voxel
])
def test_ragged_sizes_random_data(L, isx, isy, n, batch):
    scan = synth.Scan(n=n, isx=isx, isy=isy, pitch=384.0 / isx)
    vol = synth.Volume(L)
    A = oracle.carm_matrices(scan)
    q = np.random.default_rng(L + n).standard_normal((n, isy, isx)).astype(np.float32)
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    got = run_gpu(vol, scan, A, q, batch=batch)
    assert rel_l2(got, ref) <= FP32_TOL


def test_detector_smaller_than_volume_zero_padding():
    """A detector that sees only part of the volume: voxels projecting outside
    must read zero (Sect. 3.3 padding), checked element by element."""
    scan = synth.Scan(n=20, isx=24, isy=10, pitch=4.0)
    vol = synth.Volume(32)
    A = oracle.carm_matrices(scan)
    q = np.random.default_rng(3).random((scan.n, scan.isy, scan.isx), dtype=np.float32) + 0.5
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    got = run_gpu(vol, scan, A, q)
    assert (ref == 0).sum() > 1000
    np.testing.assert_array_equal(got[ref == 0], 0.0)
    assert rel_l2(got, ref) <= FP32_TOL


def test_batch_size_and_chunking_do_not_change_the_result():
    scan, vol, A, ell, q, ref = tiny_phantom_case()
    a = run_gpu(vol, scan, A, q)
    b = run_gpu(vol, scan, A, q, batch=5, chunks=[(0, 11), (11, 12), (12, 36)])
    assert rel_l2(b, ref) <= FP32_TOL
    assert rel_l2(a, b) <= 1e-6


def test_host_and_device_inputs_are_bit_identical():
    scan, vol, A, ell, q, ref = tiny_phantom_case()
    for dtype in ("f32", "f16"):
        a = run_gpu(vol, scan, A, q, dtype=dtype, on_device=True)
        b = run_gpu(vol, scan, A, q, dtype=dtype, on_device=False)
        np.testing.assert_array_equal(a, b)


def test_checkpoint_resume_is_bit_exact():
    api = native()
    scan, vol, A, ell, q, ref = tiny_phantom_case()
    qt = torch.from_numpy(q).cuda()
    one = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy)
    one.add_projections(qt[:20], A[:20])
    one.add_projections(qt[20:], A[20:])
    full = one.finalize().cpu()
    two = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy)
    two.add_projections(qt[:20], A[:20])
    state, n = two.get_state()
    assert n == 20
    two.close()
    three = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy)
    three.set_state(state.cpu(), n)
    three.add_projections(qt[20:], A[20:])
    resumed = three.finalize().cpu()
    assert three.get_state()[1] == 36
    assert torch.equal(full, resumed)


def test_reset_and_empty_batch():
    api = native()
    scan, vol, A, ell, q, ref = tiny_phantom_case()
    bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy)
    qt = torch.from_numpy(q).cuda()
    bp.add_projections(qt, A)
    bp.reset()
    bp.add_projections(qt[:0], A[:0])
    assert float(bp.finalize().abs().max()) == 0.0
    bp.add_projections(qt, A)
    assert rel_l2(bp.finalize().cpu().numpy(), ref) <= FP32_TOL


def test_volume_behind_source_is_rejected():
    api = native()
    from paper_1104_5243_gb300 import _native as N
    scan = synth.Scan(n=2, isx=16, isy=16, pitch=20.0, sid=100.0, sdd=200.0)
    vol = synth.Volume(16)
    A = oracle.carm_matrices(scan)      # source inside the 256 mm volume
    bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy)
    with pytest.raises(N.BpError) as e:
        bp.add_projections(torch.zeros((2, 16, 16), device="cuda"), A)
    assert e.value.status == N.BP_EINVAL
    with pytest.raises(N.BpError):
        bp.add_projections(torch.zeros((2, 16, 16), device="cuda"), A * np.nan)


def test_gpu_matrices_match_oracle():
    api = native()
    for name in ("tiny", "full", "train"):
        scan = synth.SCANS[name]
        np.testing.assert_allclose(api.carm_matrices(scan), oracle.carm_matrices(scan), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("L,dtype,tol", [(512, "f32", FP32_TOL), (512, "f16", FP16_TOL), (512, "bf16", BF16_TOL),
                                         (1024, "f32", FP32_TOL), (1024, "f16", FP16_TOL),
                                         (1024, "bf16", BF16_TOL), (256, "f32", FP32_TOL),
                                         (256, "f16", FP16_TOL), (256, "bf16", BF16_TOL)])
def test_full_size_sampled_voxels(L, dtype, tol):
    """256^3, 512^3 and 1024^3 x 496 x 1248x960, uniform timing stack, in the
    launch configuration the benchmark times (batches of 64, device input,
    the automatic path: TMA at 512^3 and 1024^3, the texture path with lanes
    along x and y at 256^3, for every storage type); the oracle evaluates
    4096 sampled voxels one by one."""
    api = native()
    scan, vol = synth.SCANS["full"], synth.Volume(L)
    A = oracle.carm_matrices(scan)
    stack = synth.uniform_stack(scan.n, scan.isy, scan.isx)
    bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=dtype)
    bp.add_projections(torch.from_numpy(stack).cuda(), A)
    from paper_1104_5243_gb300 import _native as N
    if L == 256:
        assert bp.last_path == "texture" and bp.query(N.BP_QUERY_LAST_LANES_X) == 24
    else:
        assert bp.last_path == "tma" and bp.query(N.BP_QUERY_LAST_BRICK_DEPTH) == 16
    got = bp.finalize().view(-1)
    rng = np.random.default_rng(7)
    idx = rng.integers(0, L ** 3, size=4096)
    ref = oracle.backproject_voxels(vol.L, vol.R, vol.O, stack, A, idx)
    g = got[torch.from_numpy(idx).cuda()].cpu().numpy()
    err = rel_l2(g, ref)
    mabs = float(np.abs(g - ref).max() / np.abs(ref).max())
    print(f"{L}^3 {dtype} sampled rel-L2 {err:.3e} max-abs {np.abs(g - ref).max():.3e} "
          f"(max |ref| {np.abs(ref).max():.3e}, relative {mabs:.3e})")
    assert err <= tol
    # the largest single-voxel error, relative to the largest value: within
    # the same bar as the rel-L2 (a voxel sums 496 rounded terms of one sign)
    assert mabs <= tol
    bp.close()


@pytest.mark.parametrize("L,dtype,tol", [(2048, "f32", FP32_TOL), (2048, "f16", FP16_TOL),
                                         (500, "f32", FP32_TOL), (500, "bf16", BF16_TOL)])
def test_largest_and_ragged_volumes_sampled(L, dtype, tol):
    """The largest volume kept resident (2048^3, 32 GiB, 4.2e9 voxels: 64-bit
    volume and record indexing) and a volume that is no multiple of the
    32 x 16 x 8 brick (500^3), each from every 31st of the 496 projections of
    1248x960, the finished volume delivered into device memory by the fused
    call; the oracle evaluates 4096 sampled voxels (the last voxel among
    them)."""
    api = native()
    full = synth.SCANS["full"]
    A = oracle.carm_matrices(full)[::31]
    vol = synth.Volume(L)
    stack = synth.uniform_stack(len(A), full.isy, full.isx, seed=13)
    out = torch.empty((L,) * 3, dtype=torch.float32, device="cuda")
    with api.Backprojector(vol.L, vol.R, vol.O, full.isx, full.isy, dtype=dtype) as bp:
        bp.add_projections_finalize(torch.from_numpy(stack).cuda(), A, out)
        assert bp.last_path == "tma"
    idx = np.random.default_rng(L).integers(0, L ** 3, size=4096)
    idx[-1] = L ** 3 - 1
    ref = oracle.backproject_voxels(vol.L, vol.R, vol.O, stack, A, idx)
    g = out.view(-1)[torch.from_numpy(idx).cuda()].cpu().numpy()
    del out
    torch.cuda.empty_cache()
    err = rel_l2(g, ref)
    mabs = float(np.abs(g - ref).max() / np.abs(ref).max())
    print(f"{L}^3 {dtype} from {len(A)} projections: sampled rel-L2 {err:.3e}, max-abs relative {mabs:.3e}")
    assert err <= tol and mabs <= tol


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("dtype,tol", [("f32", FP32_TOL), ("f16", FP16_TOL)])
def test_full_detector_ramp_filtered_phantom(dtype, tol, path):
    """512^3 with the full 1248x960 detector and a ramp-filtered 50-ellipsoid
    phantom (seed 2), every 16th of the 496 projections (the oracle computes
    the line integrals, the FDK filtering and 4096 sampled voxels)."""
    api = native()
    full = synth.SCANS["full"]
    A = oracle.carm_matrices(full)[::16]
    betas = full.betas[::16]
    sub = synth.Scan(n=len(betas), isx=full.isx, isy=full.isy, pitch=full.pitch,
                     scan_deg=float(np.degrees(betas[-1] - betas[0])))
    vol = synth.Volume(512)
    ell = synth.ellipsoids(50, seed=2, scan=full)
    lines = oracle.ellipsoid_project(A, full.isx, full.isy, ell)
    # cosine weights only: the subsampled arc is shorter than 180 degrees plus
    # the fan, so Parker weights do not apply (FDK quality is not at stake)
    q = oracle.ramp_filter(oracle.fdk_preweight(sub, lines, parker=False,
                                                scale=np.radians(200.0) / 495 * 16),
                           oracle.iso_pitch(full)).astype(np.float32)
    idx = np.random.default_rng(8).integers(0, 512 ** 3, size=4096)
    ref = oracle.backproject_voxels(vol.L, vol.R, vol.O, q, A, idx)
    from paper_1104_5243_gb300 import _native as N
    errs = {}
    for centre in ((1, 0) if dtype == "f32" else (1,)):
        bp = api.Backprojector(vol.L, vol.R, vol.O, full.isx, full.isy, dtype=dtype)
        bp.set_option(N.BP_OPT_BLOCK_CENTRE, centre)
        bp.set_option(N.BP_OPT_PATH, path)
        bp.add_projections(torch.from_numpy(q).cuda(), A)
        got = bp.finalize().view(-1)
        bp.close()
        g = got[torch.from_numpy(idx).cuda()].cpu().numpy()
        errs[centre] = rel_l2(g, ref)
        mabs = float(np.abs(g - ref).max() / np.abs(ref).max())
        print(f"512^3 phantom {dtype} path={path} block_centre={centre} sampled rel-L2 {errs[centre]:.3e} "
              f"max-abs {np.abs(g - ref).max():.3e} (relative {mabs:.3e})")
        if centre == 1:
            # ramp-filtered data mixes signs, so single voxels can carry a
            # larger share of the error than the rel-L2 shows: 4x the bar
            assert mabs <= 4 * tol
    assert errs[1] <= tol
    if dtype == "f32":
        # centring per block instead of per projection: u', v' stay within a
        # block's footprint, so their float32 rounding is several times smaller
        assert errs[1] * 4 <= errs[0]


# ---------------------------------------------------------------------------
# TMA / shared-memory data path: for float32 projections the same arithmetic
# as the texture path with per-projection centring, so the volumes agree bit
# for bit (culled bricks only skip exact zeros); 16-bit storage rounds each
# staged pixel difference once on the TMA path (the texture path differences
# the rounded pixels), so there the two paths agree to the storage rounding.
def run_path(vol, scan, A, q, path, dtype="f32", block_centre=None, depth=None):
    """block_centre=None keeps the default (per-block centring for float32
    projections, with the texture kernel's blocks or the TMA path's bricks as
    the blocks); bit-identity between the paths needs block_centre=0 on both
    for float32 projections.  depth: the TMA path's brick depth (None:
    automatic)."""
    api = native()
    from paper_1104_5243_gb300 import _native as N
    bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=dtype)
    bp.set_option(N.BP_OPT_PATH, path)
    if block_centre is not None:
        bp.set_option(N.BP_OPT_BLOCK_CENTRE, block_centre)
    if depth is not None:
        bp.set_option(N.BP_OPT_BRICK_DEPTH, depth)
    bp.add_projections(torch.from_numpy(np.ascontiguousarray(q)).cuda(), A)
    out = bp.finalize().cpu()
    taken = bp.last_path
    bp.close()
    return out, taken


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_tma_path_against_texture_path(dtype):
    scan, vol, A, ell, q, ref = tiny_phantom_case()
    tex, p1 = run_path(vol, scan, A, q, 1, dtype, block_centre=0)
    tma, p2 = run_path(vol, scan, A, q, 2, dtype, block_centre=0)
    assert (p1, p2) == ("texture", "tma")
    tol = {"f32": FP32_TOL, "f16": FP16_TOL, "bf16": BF16_TOL}[dtype]
    e_tex, e_tma = rel_l2(tex.numpy(), ref), rel_l2(tma.numpy(), ref)
    print(f"{dtype}: rel-L2 texture {e_tex:.3e}, TMA {e_tma:.3e}, max-abs TMA "
          f"{np.abs(tma.numpy() - ref).max():.3e}")
    if dtype == "f32":
        assert torch.equal(tex, tma)
    else:
        # both within the storage bar; the TMA path's coefficient quads
        # round the fractions fu, fv and the two coefficient sums to the
        # storage type once more, about 2.6x the storage error on this
        # ramp-filtered phantom (measured 2.1e-4 against 8.3e-5 for f16,
        # 1.66e-3 against 6.4e-4 for bf16)
        assert e_tma <= tol and e_tex <= tol
        assert e_tma <= 3.0 * e_tex
    # the defaults (per-block centring for float32) match the oracle too
    for path, fixed in ((1, tex), (2, tma)):
        blk, _ = run_path(vol, scan, A, q, path, dtype)
        assert rel_l2(blk.numpy(), ref) <= tol
        if dtype != "f32":
            assert torch.equal(blk, fixed)   # 16-bit storage always centres per projection


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_brick_depths_agree(dtype):
    """The TMA path's bricks of 32 x 16 x 8, 12 and 16 voxels: with
    per-projection centring every voxel sums the same float32 terms in the
    same order, so the volumes agree bit for bit (the depths differ in which
    bricks are culled and which take the global branch, both exact); with
    per-brick centring (the float32 default) each matches the oracle."""
    scan, vol, A, ell, q, ref = tiny_phantom_case()
    tol = {"f32": FP32_TOL, "f16": FP16_TOL, "bf16": BF16_TOL}[dtype]
    outs = [run_path(vol, scan, A, q, 2, dtype, block_centre=0, depth=d)[0] for d in (8, 12, 16)]
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    for d in (8, 12, 16):
        blk, _ = run_path(vol, scan, A, q, 2, dtype, depth=d)
        assert rel_l2(blk.numpy(), ref) <= tol


@pytest.mark.parametrize("L,isx,isy,n", [(37, 53, 41, 70), (1, 7, 5, 3), (40, 24, 10, 20)])
def test_tma_path_ragged_and_partial_detector(L, isx, isy, n):
    scan = synth.Scan(n=n, isx=isx, isy=isy, pitch=384.0 / isx if isx > 24 else 4.0)
    vol = synth.Volume(L)
    A = oracle.carm_matrices(scan)
    q = np.random.default_rng(L + n).standard_normal((n, isy, isx)).astype(np.float32)
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    tex, _ = run_path(vol, scan, A, q, 1, block_centre=0)
    tma, _ = run_path(vol, scan, A, q, 2, block_centre=0)
    assert torch.equal(tex, tma)
    assert rel_l2(tma.numpy(), ref) <= FP32_TOL
    for path in (1, 2):
        blk, _ = run_path(vol, scan, A, q, path)
        assert rel_l2(blk.numpy(), ref) <= FP32_TOL


@pytest.mark.parametrize("depth", [8, 16])
def test_tma_global_fallback_when_footprints_exceed_the_tile(depth):
    """256^3 with the full detector: most brick footprints are larger than the
    shared-memory tile, so the forced TMA path reads the staged images from
    global memory; still bit-identical to the texture path."""
    scan = synth.Scan(n=40, isx=1248, isy=960, pitch=0.308)
    vol = synth.Volume(256)
    A = oracle.carm_matrices(scan)
    q = synth.uniform_stack(scan.n, scan.isy, scan.isx, seed=11)
    tex, _ = run_path(vol, scan, A, q, 1, block_centre=0)
    tma, _ = run_path(vol, scan, A, q, 2, block_centre=0, depth=depth)
    assert torch.equal(tex, tma)
    idx = np.random.default_rng(1).integers(0, 256 ** 3, size=512)
    ref = oracle.backproject_voxels(vol.L, vol.R, vol.O, q, A, idx)
    assert rel_l2(tma.view(-1).numpy()[idx], ref) <= FP32_TOL
    blk, _ = run_path(vol, scan, A, q, 2, depth=depth)
    assert rel_l2(blk.view(-1).numpy()[idx], ref) <= FP32_TOL


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("L,expect,depth", [(512, "tma", 16), (1024, "tma", 16), (384, "tma", 8),
                                            (256, "texture", None), (128, "texture", None)])
def test_automatic_path_choice(dtype, L, expect, depth):
    """Automatic: the TMA path with the deepest brick whose box holds the
    footprints where voxels are fine (0.5 mm and 0.25 mm on the 1248x960
    detector: 16-deep bricks; 0.67 mm: 8-deep bricks, most footprints fit),
    the texture path where they are coarse (1 mm, 2 mm: a brick's footprint
    is wider than any staged box).  Eight projections of the full scan; the
    result equals the forced choice."""
    api = native()
    from paper_1104_5243_gb300 import _native as N
    scan = synth.SCANS["full"]
    A = oracle.carm_matrices(scan)[:8]
    q = torch.from_numpy(synth.uniform_stack(8, scan.isy, scan.isx, seed=3)).cuda()
    vol = synth.Volume(L)
    outs = []
    for path in (0, 2 if expect == "tma" else 1):
        with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=dtype) as bp:
            bp.set_option(N.BP_OPT_PATH, path)
            if path == 2:
                bp.set_option(N.BP_OPT_BRICK_DEPTH, depth)
            bp.add_projections(q, A)
            assert bp.last_path == expect
            if expect == "tma":
                assert bp.query(N.BP_QUERY_LAST_BRICK_DEPTH) == depth
            else:
                # coarse voxels (5 and 10 pixels per step): lanes along x and y
                assert bp.query(N.BP_QUERY_LAST_LANES_X) == 24
            outs.append(bp.finalize().view(-1)[::97].cpu())
    assert torch.equal(outs[0], outs[1])


LAYOUTS = (0, 8, 16, 32, 44, 42, 82, 24, 108)


@pytest.mark.parametrize("dtype,tol", [("f32", FP32_TOL), ("f16", FP16_TOL)])
@pytest.mark.parametrize("case", ["tiny", "coarse"])
def test_texture_layouts_match_oracle_and_each_other(case, dtype, tol):
    """Every warp layout of the texture kernel, on the tiny scan (64^3 at
    4 mm, 160x120 at 7.68 mm: 0.8 pixels per voxel step, where the automatic
    layout is 8 for float32 and 108 for 16-bit projections) and on a coarse
    case (96^3 at 2.67 mm, 24 projections of 624x480 at 0.616 mm: 6.6 pixels
    per step, automatic layout 24), seeded random projections: each within
    the tolerance of the FP64 oracle, and with per-projection centring
    bit-identical to each other (every voxel sums the same float32 terms in
    the same order whatever the layout)."""
    api = native()
    from paper_1104_5243_gb300 import _native as N
    if case == "tiny":
        scan, vol = synth.SCANS["tiny"], synth.Volume(64)
        auto = 8 if dtype == "f32" else 108
    else:
        half = synth.SCANS["half"]
        scan, vol = synth.Scan(n=24, isx=half.isx, isy=half.isy, pitch=half.pitch), synth.Volume(96)
        auto = 24
    A = oracle.carm_matrices(scan)
    q = np.random.default_rng(11).random((scan.n, scan.isy, scan.isx), dtype=np.float32)
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    qt = torch.from_numpy(q).cuda()
    plain = []
    for lanes in LAYOUTS:
        for centre in ((1, 0) if dtype == "f32" else (None,)):
            with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=dtype) as bp:
                bp.set_option(N.BP_OPT_PATH, 1)
                bp.set_option(N.BP_OPT_LANES_X, lanes)
                if centre is not None:
                    bp.set_option(N.BP_OPT_BLOCK_CENTRE, centre)
                bp.add_projections(qt, A)
                got = bp.finalize().cpu()
                assert bp.query(N.BP_QUERY_LAST_LANES_X) == (lanes or auto)
            assert rel_l2(got.numpy(), ref) <= tol, (lanes, centre)
            if centre != 1:
                plain.append(got)
    assert all(torch.equal(plain[0], o) for o in plain[1:])


def test_reciprocal_modes_accuracy_table():
    """Sect. 7.2 compares divps, rcpps and rcpps + Newton-Raphson by PSNR.
    Here: the IEEE reciprocal against the hardware approximate one (about
    1 ulp), both against the FP64 oracle on the ramp-filtered phantom; both
    must stay far above the paper's GPU figures (63-65 dB)."""
    scan, vol, A, ell, q, ref = tiny_phantom_case()
    approx = run_gpu(vol, scan, A, q, ieee=False)
    ieee = run_gpu(vol, scan, A, q, ieee=True)
    p_a, p_i = oracle.psnr(approx, ref), oracle.psnr(ieee, ref)
    print(f"PSNR approx rcp {p_a:.1f} dB, IEEE rcp {p_i:.1f} dB")
    assert min(p_a, p_i) > 110.0
    assert abs(p_a - p_i) < 3.0


@pytest.mark.parametrize("block_centre", [1, 0])
@pytest.mark.parametrize("L,name", [(64, "tiny"), (37, None), (96, "half")])
def test_culling_is_bit_exact(L, name, block_centre):
    """Skipping (block, projection) pairs whose footprint misses the detector
    must not change a single bit (those terms are exactly zero)."""
    api = native()
    from paper_1104_5243_gb300 import _native as N
    scan = synth.SCANS[name] if name else synth.Scan(n=70, isx=53, isy=41, pitch=384 / 53)
    if name == "half":
        scan = synth.Scan(n=40, isx=scan.isx, isy=scan.isy, pitch=scan.pitch)
    vol = synth.Volume(L)
    A = oracle.carm_matrices(scan)
    q = torch.from_numpy(np.random.default_rng(L).standard_normal((scan.n, scan.isy, scan.isx)).astype(np.float32)).cuda()
    outs = []
    for cull in (0, 1):
        bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy)
        bp.set_option(N.BP_OPT_PATH, 1)
        bp.set_option(N.BP_OPT_CULL, cull)
        bp.set_option(N.BP_OPT_BLOCK_CENTRE, block_centre)
        bp.add_projections(q, A)
        outs.append(bp.finalize().cpu())
        bp.close()
    assert torch.equal(outs[0], outs[1])


def test_detector_that_sees_part_of_the_volume_culls_and_matches_oracle():
    scan = synth.Scan(n=20, isx=24, isy=10, pitch=4.0)
    vol = synth.Volume(48)
    A = oracle.carm_matrices(scan)
    q = np.random.default_rng(4).random((scan.n, scan.isy, scan.isx), dtype=np.float32)
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    for path in (1, 2):
        got, _ = run_path(vol, scan, A, q, path)
        assert rel_l2(got.numpy(), ref) <= FP32_TOL


def _scaled_run(vol, scan, A, q, dtype, path, scale, batch=None):
    api = native()
    from paper_1104_5243_gb300 import _native as N
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=dtype) as bp:
        bp.set_option(N.BP_OPT_PATH, path)
        bp.set_option(N.BP_OPT_PROJ_SCALE, scale)
        if batch is not None:
            bp.set_option(N.BP_OPT_BATCH, batch)
        bp.add_projections(torch.from_numpy(np.ascontiguousarray(q)).cuda(), A)
        assert bp.last_path == ("texture" if path == 1 else "tma")
        return bp.finalize().cpu()


@pytest.mark.parametrize("path", [1, 2])
def test_projection_scale_is_exact_for_values_in_float16_range(path):
    """The power-of-four scale of float16 storage (BP_OPT_PROJ_SCALE, one per
    batch) changes the stored values and the batch's sums only by powers of
    two: on integer-valued projections (0..1000, exact in float16 with and
    without the scale, as are their pair differences) the volume is
    bit-identical to the unscaled one, on both data paths, with batches of
    8 projections whose maxima differ (the projections scaled by 2^-2 ..
    2^3, still exact)."""
    scan, vol = synth.SCANS["tiny"], synth.Volume(64)
    A = oracle.carm_matrices(scan)
    q = np.random.default_rng(21).integers(0, 1001, (scan.n, scan.isy, scan.isx)).astype(np.float32)
    q *= (2.0 ** (np.arange(scan.n) % 6 - 2)).astype(np.float32)[:, None, None]   # 0.25 .. 8 per projection
    off = _scaled_run(vol, scan, A, q, "f16", path, 0, batch=8)
    on = _scaled_run(vol, scan, A, q, "f16", path, 1, batch=8)
    assert torch.equal(off, on)


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("magnitude", [1e6, 1e-7])
def test_projection_scale_keeps_float16_accuracy_outside_its_range(path, magnitude):
    """Projections of magnitude 1e6 overflow float16 (65504) and of 1e-7 fall
    into its subnormals (below 6.1e-5; the smallest is 6e-8): stored as they
    are, the volume is infinite or far off; with the power-of-four scale it
    is within the float16 tolerance of the FP64 oracle, and both sides are
    compared relative to the reference's own magnitude."""
    scan, vol = synth.SCANS["tiny"], synth.Volume(64)
    A = oracle.carm_matrices(scan)
    q = (np.random.default_rng(22).random((scan.n, scan.isy, scan.isx)) * magnitude).astype(np.float32)
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    on = _scaled_run(vol, scan, A, q, "f16", path, 1).numpy()
    e_on = rel_l2(on, ref)
    off = _scaled_run(vol, scan, A, q, "f16", path, 0).numpy()
    e_off = rel_l2(off, ref) if np.all(np.isfinite(off)) else np.inf
    print(f"magnitude {magnitude:g} path {path}: scaled {e_on:.2e}, unscaled {e_off:.2e}")
    assert e_on <= FP16_TOL
    assert e_off > 10 * FP16_TOL


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_projection_scale_applies_to_float16_only(dtype):
    scan, vol = synth.SCANS["tiny"], synth.Volume(64)
    A = oracle.carm_matrices(scan)
    q = np.random.default_rng(23).random((scan.n, scan.isy, scan.isx), dtype=np.float32)
    for path in (1, 2):
        assert torch.equal(_scaled_run(vol, scan, A, q, dtype, path, 0), _scaled_run(vol, scan, A, q, dtype, path, 1))


def test_projection_scale_with_host_inputs_and_the_fused_call():
    """The scaled float16 path through the other input routes: host images
    (staged on the copy stream, their maximum taken there) and the fused
    add_projections_finalize into pinned host memory give the same volume,
    bit for bit, as device images with separate calls; ragged batches."""
    api = native()
    from paper_1104_5243_gb300 import _native as N
    scan, vol = synth.SCANS["tiny"], synth.Volume(64)
    A = oracle.carm_matrices(scan)
    q = (np.random.default_rng(24).random((scan.n, scan.isy, scan.isx)) * 3e5).astype(np.float32)
    outs = []
    for route in ("device", "host", "fused"):
        with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype="f16") as bp:
            bp.set_option(N.BP_OPT_PROJ_SCALE, 1)
            bp.set_option(N.BP_OPT_BATCH, 10)
            qt = torch.from_numpy(q)
            if route == "device":
                bp.add_projections(qt.cuda(), A)
                outs.append(bp.finalize().cpu())
            elif route == "host":
                bp.add_projections(qt.pin_memory(), A)
                outs.append(bp.finalize().cpu())
            else:
                host = torch.empty(bp.shape, dtype=torch.float32).pin_memory()
                bp.add_projections_finalize(qt.cuda(), A, host)
                outs.append(host.clone())
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    assert np.all(np.isfinite(outs[0].numpy())) and rel_l2(outs[0].numpy(), ref) <= FP16_TOL
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
