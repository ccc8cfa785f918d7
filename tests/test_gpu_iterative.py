"""Iterative reconstruction (CGLS) on the library's operator pair: the
forward model is bp_adjoint, its transpose bp_add_projections.  CGLS from
zero converges to the minimum-norm least-squares solution, which a dense
solve of the oracle-built system matrix gives independently."""
import numpy as np
import pytest

import oracle
from paper_1104_5243_gb300 import synth

from gpu_common import native, rel_l2, torch

pytestmark = pytest.mark.gpu


def test_cgls_converges_to_dense_least_squares_solution():
    native()
    from paper_1104_5243_gb300 import api, iterative
    scan, vol = synth.Scan(n=8, isx=24, isy=18, pitch=16.0), synth.Volume(8)
    A = oracle.carm_matrices(scan)
    n_vox = vol.L ** 3
    # dense forward matrix from the oracle's adjoint of unit voxels
    P = np.zeros((scan.n * scan.isy * scan.isx, n_vox))
    for j in range(n_vox):
        e = np.zeros(n_vox)
        e[j] = 1.0
        P[:, j] = oracle.adjoint(vol.L, vol.R, vol.O, e.reshape((vol.L,) * 3), A, scan.isx, scan.isy).ravel()
    rng = np.random.default_rng(0)
    f_true = rng.random(n_vox)
    p = P @ f_true + 1e-3 * rng.standard_normal(P.shape[0])
    f_ls = np.linalg.lstsq(P, p, rcond=None)[0]
    bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy)
    ops = iterative.Operators(bp, A, scale=1.0)
    pt = torch.from_numpy(p.reshape(scan.n, scan.isy, scan.isx).astype(np.float32)).cuda()
    f, norms = iterative.cgls(ops, pt, iters=150)
    bp.close()
    assert all(b <= a * (1 + 1e-4) for a, b in zip(norms, norms[1:]))   # CGLS: residual never grows
    assert rel_l2(f.cpu().numpy().ravel(), f_ls) <= 2e-3


def test_cgls_improves_on_the_phantom_and_reduces_the_residual():
    native()
    from paper_1104_5243_gb300 import api, iterative
    scan, vol = synth.SCANS["tiny"], synth.Volume(64)
    A = oracle.carm_matrices(scan)
    ell = synth.ellipsoids(10, seed=1, scan=scan)
    lines = api.ellipsoid_project(A, scan.isx, scan.isy, ell)
    target = api.ellipsoid_voxelize(vol.L, vol.R, vol.O, ell)
    bp = api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy)
    ops = iterative.Operators(bp, A, scale=iterative.model_scale(vol.R, api.iso_pitch(scan)))
    f, norms = iterative.cgls(ops, lines, iters=20)
    bp.close()
    assert norms[-1] < 0.2 * norms[0]
    mse0 = float(torch.mean(target ** 2))
    mse = float(torch.mean((f - target) ** 2))
    print(f"CGLS 20 it: residual {norms[0]:.3e} -> {norms[-1]:.3e}, MSE {mse:.3e} (zero image {mse0:.3e})")
    assert mse < 0.25 * mse0
