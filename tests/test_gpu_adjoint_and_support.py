"""GPU parity of the adjoint scatter and of the support kernels (FP64
matrices, phantom projection/voxelisation, FDK pre-weights, ramp filter,
learned row filter and its gradients) against the FP64 oracle, through the
C ABI."""
import numpy as np
import pytest

import oracle
from paper_1104_5243_gb300 import synth

from gpu_common import native, rel_l2, torch

pytestmark = pytest.mark.gpu


def make_bp(vol, scan):
    return native().Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy)


@pytest.mark.parametrize("L,scan", [
    (32, synth.SCANS["grad"]),                                  # 32^3, 12 x 64x48
    (37, synth.Scan(n=70, isx=53, isy=41, pitch=384 / 53)),     # ragged, > one batch
])
def test_adjoint_matches_oracle(L, scan):
    vol = synth.Volume(L)
    A = oracle.carm_matrices(scan)
    f = synth.uniform_volume(L, seed=L) - 0.5
    ref = oracle.adjoint(vol.L, vol.R, vol.O, f.astype(np.float64), A, scan.isx, scan.isy)
    with make_bp(vol, scan) as bp:
        got = bp.adjoint(torch.from_numpy(f).cuda(), A).cpu().numpy()
        # host in / host out through the same entry point
        got_h = bp.adjoint(torch.from_numpy(f), A, out=torch.empty(ref.shape, dtype=torch.float32)).numpy()
    assert rel_l2(got, ref) <= 1e-5
    assert rel_l2(got_h, ref) <= 1e-5


@pytest.mark.parametrize("signed", [False, True])
def test_adjoint_dot_product_on_gpu(signed):
    """<B p, f> = <p, B^T f> with both operators on the GPU (FP32).  With
    nonnegative data the two sides agree to 5e-6 relative.  With zero-mean
    data the sums cancel, and float32 rounding scales with the sum of
    magnitudes <|p|, B^T |f|>, the bound used then."""
    scan, vol = synth.SCANS["tiny"], synth.Volume(64)
    A = oracle.carm_matrices(scan)
    rng = np.random.default_rng(21)
    draw = rng.standard_normal if signed else rng.random
    p = torch.from_numpy(draw((scan.n, scan.isy, scan.isx)).astype(np.float32)).cuda()
    f = torch.from_numpy(draw((vol.L,) * 3).astype(np.float32)).cuda()
    with make_bp(vol, scan) as bp:
        bp.add_projections(p, A)
        Bp = bp.finalize()
        Btf = bp.adjoint(f, A)
        Bt_abs = bp.adjoint(f.abs(), A)
    lhs = float((Bp.double() * f.double()).sum())
    rhs = float((p.double() * Btf.double()).sum())
    magnitude = float((p.double().abs() * Bt_abs.double()).sum())
    print(f"dot product ({'signed' if signed else 'nonnegative'}): |lhs - rhs| / |lhs| {abs(lhs - rhs) / abs(lhs):.2e}, "
          f"/ <|p|, B^T|f|> {abs(lhs - rhs) / magnitude:.2e}")
    if signed:
        assert abs(lhs - rhs) <= 1e-5 * magnitude
    else:
        assert abs(lhs - rhs) <= 5e-6 * abs(lhs)


def test_adjoint_of_half_detector_workload_sampled():
    """256^3 -> 248 x 624x480 (the differentiation workload) on sampled
    projections, compared with the oracle's adjoint restricted to them."""
    scan, vol = synth.SCANS["half"], synth.Volume(256)
    A = oracle.carm_matrices(scan)
    f = synth.uniform_volume(vol.L, seed=5)
    with make_bp(vol, scan) as bp:
        got = bp.adjoint(torch.from_numpy(f).cuda(), A)
    sel = [0, 61, 123, 247]
    ref = oracle.adjoint(vol.L, vol.R, vol.O, f.astype(np.float64), A[sel], scan.isx, scan.isy)
    assert rel_l2(got[sel].cpu().numpy(), ref) <= 1e-5


def test_ellipsoid_projection_matches_oracle():
    api = native()
    scan = synth.SCANS["tiny"]
    A = oracle.carm_matrices(scan)
    ell = synth.ellipsoids(10, seed=1, scan=scan)
    ref = oracle.ellipsoid_project(A, scan.isx, scan.isy, ell)
    got = api.ellipsoid_project(A, scan.isx, scan.isy, ell).cpu().numpy()
    # A ray grazing an ellipsoid has chord 2 a sqrt(h / |sd|^2) with h = 1 - |m|^2
    # near 0: a float32 error of ~1e-7 in h moves the chord by up to
    # 2 a sqrt(1e-7) (~0.04 mm at a = 64 mm).  Hence a max-abs bound of
    # rho * 0.1 mm per ray next to the rel-L2 bound over all rays.
    assert np.abs(got - ref).max() <= 0.1 * ell[:, 15].sum()
    assert rel_l2(got, ref) <= 1e-5


def test_ellipsoid_projection_full_detector_sampled():
    api = native()
    scan = synth.SCANS["full"]
    A = oracle.carm_matrices(scan)[::97]
    ell = synth.ellipsoids(50, seed=2, scan=scan)
    got = api.ellipsoid_project(A, scan.isx, scan.isy, ell).cpu().numpy()
    ref = oracle.ellipsoid_project(A, scan.isx, scan.isy, ell)
    assert rel_l2(got, ref) <= 1e-5


def test_voxelize_matches_oracle_up_to_boundary_ties():
    api = native()
    vol = synth.Volume(64)
    ell = synth.ellipsoids(10, seed=1, scan=synth.SCANS["tiny"])
    ref = oracle.ellipsoid_voxelize(vol.L, vol.R, vol.O, ell)
    got = api.ellipsoid_voxelize(vol.L, vol.R, vol.O, ell).cpu().numpy()
    bad = np.abs(got - ref) > 1e-6
    # a voxel centre within float32 rounding of an ellipsoid surface may fall
    # on either side; allow at most a handful of such voxels
    assert bad.sum() <= 5


@pytest.mark.parametrize("name,parker", [("train", True), ("tiny", False), ("full", True)])
def test_fdk_preweight_matches_oracle(name, parker):
    api = native()
    scan = synth.SCANS[name]
    if name == "full":
        scan = synth.Scan(n=9, isx=scan.isx, isy=scan.isy, pitch=scan.pitch)
    x = np.random.default_rng(2).random((scan.n, scan.isy, scan.isx), dtype=np.float32)
    ref = oracle.fdk_preweight(scan, x, parker=parker, scale=0.37)
    got = api.fdk_preweight(scan, torch.from_numpy(x).cuda(), parker=parker, scale=0.37).cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-6


@pytest.mark.parametrize("isx", [1, 2, 7, 160, 312, 1248])
def test_ramp_filter_matches_oracle(isx):
    api = native()
    rows = 6
    x = np.random.default_rng(isx).standard_normal((rows, isx)).astype(np.float32)
    tau = 0.2013
    ref = oracle.ramp_filter(x, tau)
    got = api.ramp_filter(torch.from_numpy(x).cuda(), tau).cpu().numpy()
    assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("T,isx,rows", [(64, 312, 37), (8, 29, 5), (1, 16, 3), (128, 100, 9), (63, 1248, 4)])
def test_row_filter_fwd_bwd_match_oracle(T, isx, rows):
    api = native()
    rng = np.random.default_rng(T + isx)
    x = rng.standard_normal((rows, isx)).astype(np.float32)
    h = rng.standard_normal(T).astype(np.float32)
    g = rng.standard_normal((rows, isx)).astype(np.float32)
    ref = oracle.row_filter_fwd(x, h)
    gin_ref, gh_ref = oracle.row_filter_bwd(x, h, g)
    xt, ht, gt = (torch.from_numpy(a).cuda() for a in (x, h, g))
    got = api.row_filter_fwd(xt, ht).cpu().numpy()
    gin, gh = api.row_filter_bwd(xt, ht, gt)
    assert rel_l2(got, ref) <= 1e-5
    assert rel_l2(gin.cpu().numpy(), gin_ref) <= 1e-5
    assert rel_l2(gh.cpu().numpy(), gh_ref) <= 1e-5
    # deterministic reduction: repeated calls agree bit for bit
    assert torch.equal(gh, api.row_filter_bwd(xt, ht, gt)[1])


def test_gpu_fdk_chain_matches_oracle_chain():
    """GPU preprocessing + backprojection vs the oracle's whole FDK chain on
    the 10-ellipsoid tiny phantom (each side computes its own line integrals,
    weights, ramp and backprojection)."""
    api = native()
    scan, vol = synth.SCANS["tiny"], synth.Volume(64)
    ell = synth.ellipsoids(10, seed=1, scan=scan)
    A_ref = oracle.carm_matrices(scan)
    ref = oracle.backproject(vol.L, vol.R, vol.O,
                             oracle.fdk_filter(scan, oracle.ellipsoid_project(A_ref, scan.isx, scan.isy, ell),
                                               parker=False).astype(np.float32), A_ref)
    A = api.carm_matrices(scan)
    q = api.fdk_filter(scan, api.ellipsoid_project(A, scan.isx, scan.isy, ell), parker=False)
    with make_bp(vol, scan) as bp:
        bp.add_projections(q, A)
        got = bp.finalize().cpu().numpy()
    assert rel_l2(got, ref) <= 1e-4


@pytest.mark.parametrize("L,scan", [
    (32, synth.SCANS["grad"]),
    (37, synth.Scan(n=70, isx=53, isy=41, pitch=384 / 53)),
    (48, synth.Scan(n=20, isx=24, isy=10, pitch=4.0)),      # detector sees part of the volume
])
def test_shared_memory_adjoint_matches_direct_and_oracle(L, scan):
    """The shared-memory adjoint (default) and the direct-atomic one agree
    to 5e-6 and both match the oracle to 1e-5.  The direct kernel's images
    differ from the oracle by float32 summation order.  The tile kernel's
    also differ by its fixed-point quantisation: a term is rounded to 2^-31
    of the block's bound sum(|f|) max(r^2), about 1e-6 relative on these
    coarse detectors."""
    api = native()
    from paper_1104_5243_gb300 import _native as N
    vol = synth.Volume(L)
    A = oracle.carm_matrices(scan)
    f = synth.uniform_volume(L, seed=L + 1) - 0.25
    ref = oracle.adjoint(vol.L, vol.R, vol.O, f.astype(np.float64), A, scan.isx, scan.isy)
    outs = []
    for cull in (0, 1):
        with make_bp(vol, scan) as bp:
            bp.set_option(N.BP_OPT_CULL, cull)
            outs.append(bp.adjoint(torch.from_numpy(f).cuda(), A).cpu().numpy())
    assert rel_l2(outs[1], outs[0]) <= 5e-6
    for o in outs:
        assert rel_l2(o, ref) <= 1e-5


@pytest.mark.parametrize("kind", ["phantom", "zero_mean"])
def test_adjoint_full_detector_512(kind):
    """512^3 -> 4 projections of the full 1248x960 detector (the coordinate
    range where float32 centring matters), against the oracle's adjoint:
    the voxelised 50-ellipsoid phantom, and a zero-mean random volume (the
    gradient-like input of the autograd backward)."""
    scan = synth.SCANS["full"]
    vol = synth.Volume(512)
    A = oracle.carm_matrices(scan)[[0, 124, 248, 371]]
    if kind == "phantom":
        f = oracle.ellipsoid_voxelize(vol.L, vol.R, vol.O, synth.ellipsoids(50, seed=2, scan=scan)).astype(np.float32)
    else:
        f = (synth.uniform_volume(vol.L, seed=9) - 0.5).astype(np.float32)
    ref = oracle.adjoint(vol.L, vol.R, vol.O, f.astype(np.float64), A, scan.isx, scan.isy)
    with make_bp(vol, scan) as bp:
        got = bp.adjoint(torch.from_numpy(f).cuda(), A).cpu().numpy()
    err = rel_l2(got, ref)
    # A pixel of B^T f sums thousands of voxel terms; with mixed signs the
    # sum is far smaller than the sum of magnitudes, and float32 rounding of
    # the terms and of the accumulation scales with the latter.  The error
    # is therefore measured against B^T |f| (equal to B^T f for the
    # nonnegative phantom).
    scale = np.linalg.norm(oracle.adjoint(vol.L, vol.R, vol.O, np.abs(f).astype(np.float64), A, scan.isx,
                                          scan.isy)) if kind == "zero_mean" else np.linalg.norm(ref)
    err_abs = np.linalg.norm(got - ref) / scale
    print(f"adjoint 512^3 -> 4 x 1248x960 {kind}: rel-L2 {err:.3e}, against B^T|f| {err_abs:.3e}")
    assert err_abs <= 1e-5


def test_adjoint_oversized_footprints_use_global_atomics():
    """256^3 (1 mm voxels, about 5 detector pixels each) onto the full
    1248x960 detector: a 32 x 32 x 4-voxel block's footprint spans 3700-5200
    pixels, more than the shared tile holds, so the tile kernel takes its
    global-atomic branch (with per-block centring)."""
    scan = synth.Scan(n=6, isx=1248, isy=960, pitch=0.308)
    vol = synth.Volume(256)
    A = oracle.carm_matrices(scan)
    f = synth.uniform_volume(vol.L, seed=33) - 0.25
    ref = oracle.adjoint(vol.L, vol.R, vol.O, f.astype(np.float64), A, scan.isx, scan.isy)
    with make_bp(vol, scan) as bp:
        got = bp.adjoint(torch.from_numpy(f).cuda(), A).cpu().numpy()
    assert rel_l2(got, ref) <= 1e-5
