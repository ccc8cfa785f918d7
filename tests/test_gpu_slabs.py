"""z-slab contexts (bp_create_slab): a volume reconstructed slab by slab
into host memory (the paper's split of the z loop, Sect. 6; volumes larger
than one context), and the adjoint of a slab, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1104_5243_gb300 import synth

from gpu_common import native, rel_l2, torch

pytestmark = pytest.mark.gpu


def case(L=37):
    scan = synth.Scan(n=70, isx=53, isy=41, pitch=384.0 / 53)
    vol = synth.Volume(L)
    A = oracle.carm_matrices(scan)
    q = np.random.default_rng(L).standard_normal((scan.n, scan.isy, scan.isx)).astype(np.float32)
    return scan, vol, A, q


@pytest.mark.parametrize("dtype,path", [("f32", 0), ("f32", 1), ("f16", 0), ("bf16", 1)])
def test_slab_by_slab_reconstruction_matches_the_oracle(dtype, path):
    """37^3 in slabs of 10 slices (10, 10, 10, 7), host output, against the
    oracle and against one context holding the whole cube (bit for bit for
    the 16-bit forms)."""
    api = native()
    from paper_1104_5243_gb300 import _native as N
    scan, vol, A, q = case()
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    qt = torch.from_numpy(q).cuda()
    if path == 0:
        got = api.backproject_slabs(vol.L, vol.R, vol.O, qt, A, slab=10, dtype=dtype).numpy()
    else:
        got = np.zeros((vol.L,) * 3, dtype=np.float32)
        for z0 in range(0, vol.L, 10):
            nz = min(10, vol.L - z0)
            with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=dtype, nz=nz, z0=z0) as bp:
                bp.set_option(N.BP_OPT_PATH, path)
                bp.add_projections(qt, A)
                got[z0:z0 + nz] = bp.finalize().cpu().numpy()
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, dtype=dtype) as bp:
        bp.set_option(N.BP_OPT_PATH, path)   # the same path (and centring tiles) as the slabs
        bp.add_projections(qt, A)
        whole = bp.finalize().cpu().numpy()
    tol = {"f32": 1e-5, "f16": 1e-3, "bf16": 1e-2}[dtype]
    print(f"{dtype} path {path}: slabs against the oracle {rel_l2(got, ref):.3e}, against the whole cube "
          f"{rel_l2(got, whole):.3e}")
    assert rel_l2(got, ref) <= tol
    if dtype == "f32":
        # per-block centring: slabs whose bricks cut the cube's differently
        # agree to float32 rounding
        assert rel_l2(got, whole) <= 1e-6
    else:
        # per-projection centring and z coordinates from the global slice
        # index: every slab computes the cube's values bit for bit
        assert np.array_equal(got, whole)


def test_slab_adjoint_equals_the_adjoint_of_the_zero_padded_volume():
    api = native()
    scan, vol, A, _ = case(40)
    f = synth.uniform_volume(vol.L, seed=3) - 0.25
    z0, nz = 13, 9
    padded = np.zeros_like(f)
    padded[z0:z0 + nz] = f[z0:z0 + nz]
    ref = oracle.adjoint(vol.L, vol.R, vol.O, padded.astype(np.float64), A, scan.isx, scan.isy)
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, nz=nz, z0=z0) as bp:
        got = bp.adjoint(torch.from_numpy(np.ascontiguousarray(f[z0:z0 + nz])).cuda(), A).cpu().numpy()
        with pytest.raises(ValueError):
            bp.adjoint(torch.from_numpy(f).cuda(), A)   # the whole cube is not this slab
    assert rel_l2(got, ref) <= 1e-5


def test_single_slice_slab_and_state_roundtrip():
    api = native()
    scan, vol, A, q = case(16)
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, nz=1, z0=15) as bp:
        bp.add_projections(torch.from_numpy(q[:30]).cuda(), A[:30])
        state, n = bp.get_state()
        assert state.shape == (1, 16, 16) and n == 30
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, nz=1, z0=15) as bp:
        bp.set_state(state, n)
        bp.add_projections(torch.from_numpy(q[30:]).cuda(), A[30:])
        got = bp.finalize().cpu().numpy()
    assert rel_l2(got[0], ref[15]) <= 1e-5


def _slab_rank(rank, world, port, L, out_dir):
    """One rank of the z-split (bench.py --split z): its slab of the L^3
    volume from every projection, on cuda:0, gathered to rank 0 over gloo."""
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import bench
    from paper_1104_5243_gb300 import _native as N
    from paper_1104_5243_gb300 import api, build
    build.build()
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    scan, vol, A, q = case(L)
    z0, nz = bench.slab_of_rank(L, world, rank)
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, nz=nz, z0=z0) as bp:
        bp.set_option(N.BP_OPT_PATH, 2)
        bp.set_option(N.BP_OPT_BRICK_DEPTH, 8)
        bp.add_projections(torch.from_numpy(q).cuda(), A)
        mine = bp.finalize().cpu()
    parts = [None] * world
    dist.all_gather_object(parts, (z0, nz, mine.numpy()))
    if rank == 0:
        np.save(os.path.join(out_dir, "stitched.npy"),
                np.concatenate([p[2] for p in sorted(parts, key=lambda t: t[0])], axis=0))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("L", [72, 64])
def test_two_ranks_split_z_stitch_to_the_whole_volume(tmp_path, L):
    """Two processes on one GPU, each reconstructing the z-slab that
    bench.slab_of_rank gives it (as bench.py --split z does on two GPUs),
    gathered over gloo: the stitched volume equals, bit for bit, one context
    holding the whole cube.  The slabs are whole 8-slice granules and the
    bricks 8 deep, so every slab brick is a brick of the cube; a slab takes
    its centring offsets and records from the whole grid, so its float32
    arithmetic is the cube's."""
    import socket
    import torch.multiprocessing as mp
    from paper_1104_5243_gb300 import _native as N
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_slab_rank, args=(2, port, L, str(tmp_path)), nprocs=2, join=True)
    stitched = np.load(tmp_path / "stitched.npy")
    api = native()
    scan, vol, A, q = case(L)
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy) as bp:
        bp.set_option(N.BP_OPT_PATH, 2)
        bp.set_option(N.BP_OPT_BRICK_DEPTH, 8)
        bp.add_projections(torch.from_numpy(q).cuda(), A)
        whole = bp.finalize().cpu().numpy()
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    assert stitched.shape == whole.shape
    np.testing.assert_array_equal(stitched, whole)
    assert rel_l2(stitched, ref) <= 1e-5


def test_moved_slab_context_equals_fresh_slab_contexts():
    """bp_move_slab re-targets one context over the volume (its allocations
    kept): every slab equals, bit for bit, the slab a fresh context of that
    slab computes, and a slab deeper than the context's allocation, or one
    outside the volume, is refused."""
    api = native()
    from paper_1104_5243_gb300 import _native as N
    scan, vol, A, q = case(40)
    qt = torch.from_numpy(q).cuda()
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, nz=16, z0=0) as moved:
        for z0, nz in [(0, 16), (16, 16), (32, 8), (5, 11)]:
            moved.move_slab(z0, nz)
            moved.add_projections(qt, A)
            got = moved.finalize().cpu()
            with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy, nz=nz, z0=z0) as fresh:
                fresh.add_projections(qt, A)
                assert torch.equal(got, fresh.finalize().cpu()), (z0, nz)
        for z0, nz in [(0, 17), (30, 16), (-1, 4), (0, 0)]:
            with pytest.raises(N.BpError) as e:
                moved.move_slab(z0, nz)
            assert e.value.status == N.BP_EINVAL


@pytest.mark.parametrize("contexts", [1, 2])
def test_threaded_slab_reconstruction_matches_the_oracle(contexts):
    """api.backproject_slabs with one or two moved contexts (two: each on its
    own stream and host thread) into pinned host memory, 56^3 in slabs of 16
    (the last one 8 slices), host and device images."""
    api = native()
    scan, vol, A, q = case(56)
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    for images in (torch.from_numpy(q).cuda(), torch.from_numpy(q).pin_memory()):
        got = api.backproject_slabs(vol.L, vol.R, vol.O, images, A, slab=16, contexts=contexts).numpy()
        assert rel_l2(got, ref) <= 1e-5
    # a pool of contexts kept across reconstructions gives the same volumes
    pool = api.slab_contexts(vol.L, vol.R, vol.O, scan.isx, scan.isy, 16, count=contexts)
    try:
        first = api.backproject_slabs(vol.L, vol.R, vol.O, torch.from_numpy(q).cuda(), A, slab=16, pool=pool)
        again = api.backproject_slabs(vol.L, vol.R, vol.O, torch.from_numpy(q).cuda(), A, slab=16, pool=pool)
        assert torch.equal(first, again) and rel_l2(first.numpy(), ref) <= 1e-5
        with pytest.raises(ValueError):
            api.backproject_slabs(vol.L, vol.R, vol.O, torch.from_numpy(q).cuda(), A, slab=32, pool=pool)
    finally:
        for bp in pool:
            bp.close()
