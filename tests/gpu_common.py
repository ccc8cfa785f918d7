"""Shared helpers for the GPU tests: build/load the CUDA library, make the
seeded workloads, error measures.  Inputs come from the seeded generators
(paper_1104_5243_gb300.synth) or from the oracle; expected values come only
from the oracle."""
import functools

import numpy as np
import pytest

import oracle
from paper_1104_5243_gb300 import synth

torch = pytest.importorskip("torch")


@functools.lru_cache(maxsize=None)
def native():
    from paper_1104_5243_gb300 import build
    build.build()
    from paper_1104_5243_gb300 import _native
    _native.lib()
    from paper_1104_5243_gb300 import api
    return api


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@functools.lru_cache(maxsize=None)
def tiny_phantom_case():
    """Tiny workload: 64^3 at 4 mm, 36 projections of 160 x 120 (7.68 mm) over
    200 degrees, 10 seeded ellipsoids (seed 1), ramp-filtered -- all by the
    oracle.  Parker weights are off: the 200-degree arc is shorter than
    180 degrees plus the 54-degree fan of this detector."""
    scan, vol = synth.SCANS["tiny"], synth.Volume(64)
    A = oracle.carm_matrices(scan)
    ell = synth.ellipsoids(10, seed=1, scan=scan)
    lines = oracle.ellipsoid_project(A, scan.isx, scan.isy, ell)
    q = oracle.fdk_filter(scan, lines, parker=False).astype(np.float32)
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    return scan, vol, A, ell, q, ref
