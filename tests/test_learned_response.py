"""The learned filter's parameterisations on the CPU (no kernels run): the
cosine-coefficient form and the small-MLP response form both start as the
plain ramp, stay symmetric, pass gradients to their parameters, and resample
to a finer detector consistently."""
import pytest
import torch

from paper_1104_5243_gb300 import learned


@pytest.mark.parametrize("response", ["cosine", "mlp"])
def test_starts_as_the_ramp_and_stays_symmetric_under_training(response):
    torch.manual_seed(0)
    T = 64
    filt = learned.LearnedRowFilter(T, tau=1.2, response=response)
    assert torch.count_nonzero(filt.delta) == 0
    assert torch.equal(filt.taps, filt.ramlak_central)
    # gradient steps towards a symmetric change with a smooth response (a
    # 3-tap sharpening stencil; a change concentrated at the lowest
    # frequencies is not what the MLP's smooth response fits quickly)
    target = torch.zeros(T)
    target[T // 2] = 0.01
    target[T // 2 - 1] = target[T // 2 + 1] = -0.004
    opt = torch.optim.Adam(filt.parameters(), lr=1e-3)
    first = None
    for _ in range(200):
        opt.zero_grad()
        loss = torch.sum((filt.delta - target) ** 2)
        loss.backward()
        assert all(p.grad is not None and torch.isfinite(p.grad).all() for p in filt.parameters())
        opt.step()
        first = loss.item() if first is None else first
    assert loss.item() < 0.1 * first
    d = filt.delta.detach()
    # symmetric about the centre tap: delta[T/2 + j] == delta[T/2 - j]
    j = torch.arange(1, T // 2)
    assert torch.allclose(d[T // 2 + j], d[T // 2 - j], atol=1e-7)


@pytest.mark.parametrize("response", ["cosine", "mlp"])
def test_resampling_at_factor_one_is_the_delta(response):
    torch.manual_seed(1)
    filt = learned.LearnedRowFilter(32, response=response)
    with torch.no_grad():
        for p in filt.parameters():
            p.add_(0.01 * torch.randn_like(p))
    assert torch.allclose(filt.delta_at_pitch(1), filt.delta.detach(), atol=1e-6)
    fine = filt.delta_at_pitch(4)
    assert fine.numel() == 4 * 32
    # every 4th fine tap sits on a coarse tap: the same series, scaled by 1/4
    assert torch.allclose(fine[::4], filt.delta.detach() / 4, atol=1e-6)


def test_unknown_response_is_rejected():
    with pytest.raises(ValueError):
        learned.LearnedRowFilter(16, response="spline")
