"""Failure detection without a GPU fault: the device-side waits of the TMA
path are bounded; when one gives up, the kernel records an error flag that
the host returns as BP_ETIMEOUT, and the device stays usable."""
import numpy as np
import pytest

import oracle
from paper_1104_5243_gb300 import synth

from gpu_common import native, rel_l2, torch

pytestmark = pytest.mark.gpu


def test_bounded_wait_completes_when_the_barrier_is_released():
    from paper_1104_5243_gb300 import _native as N
    native()
    assert N.bp_selftest_bounded_wait(True, 100) == N.BP_OK


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    """A barrier nothing completes: the wait gives up after 50 suspensions
    (at most 5 ms), the status is BP_ETIMEOUT, and a backprojection run
    afterwards still matches the oracle."""
    from paper_1104_5243_gb300 import _native as N
    api = native()
    assert N.bp_selftest_bounded_wait(False, 50) == N.BP_ETIMEOUT
    assert "gave up" in N.bp_last_error(None)
    scan, vol = synth.SCANS["grad"], synth.Volume(32)
    A = oracle.carm_matrices(scan)
    q = np.random.default_rng(5).standard_normal((scan.n, scan.isy, scan.isx)).astype(np.float32)
    ref = oracle.backproject(vol.L, vol.R, vol.O, q, A)
    with api.Backprojector(vol.L, vol.R, vol.O, scan.isx, scan.isy) as bp:
        bp.add_projections(torch.from_numpy(q).cuda(), A)
        got = bp.finalize().cpu().numpy()
    assert rel_l2(got, ref) <= 1e-5
