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
    oracle and against one context holding the whole cube."""
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
    assert rel_l2(got, ref) <= tol
    assert rel_l2(got, whole) <= (1e-6 if dtype == "f32" else 1e-5)


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
