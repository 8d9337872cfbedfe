"""Failure detection without a GPU fault: the bounded completion waits of the tensor-core
kernels.

The environment knob ARKCOS_TEST_WITHHOLD_MMA makes the tensor-core kernels skip the issue of
their MMAs (and of the commit that would arrive on the completion barrier), so every wait runs
out after about a second with nothing in flight.  The kernel records the error, frees its
tensor memory and returns; arkcos_sync_status reports ETIMEOUT and clears the record, and the
next call without the knob computes the right result."""
import numpy as np
import pytest

from paper_1104_0672_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ark():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_1104_0672_gb300 as ark
    return ark


def _setup(ark, nside=64):
    """nside 64 for the contraction; nside 256 for the knot projection, whose tensor-core form
    needs a kernel grid of at least 1024 points (the pairs next to the poles go by FFT)."""
    import torch
    g = ark.Grid.healpix(nside)
    gmax = (3 if nside == 64 else 2) * inputs.DEG
    k = ark.Kernel(g, inputs.gaussian_knots(gmax / 3, gmax, 128), gmax)
    x = torch.from_numpy(inputs.white_noise(g.npix, 2, config=30)).to(torch.device("cuda:0"))
    return g, k, x


def test_expired_contraction_wait_reports_timeout_and_recovers(ark, monkeypatch):
    import torch
    from paper_1104_0672_gb300 import _native
    g, k, x = _setup(ark)
    ref = ark.convolve(g, k, x, ark.FLAG_3XTF32)
    ark.sync_status()
    monkeypatch.setenv("ARKCOS_TEST_WITHHOLD_MMA", "1")
    ark.convolve(g, k, x, ark.FLAG_3XTF32)
    with pytest.raises(_native.ArkcosError) as e:
        ark.sync_status()
    assert e.value.status == _native.ETIMEOUT
    monkeypatch.delenv("ARKCOS_TEST_WITHHOLD_MMA")
    ark.sync_status()  # the record was cleared by the report
    y = ark.convolve(g, k, x, ark.FLAG_3XTF32)
    ark.sync_status()
    assert torch.equal(y, ref)


def test_expired_knot_projection_wait_reports_timeout_and_recovers(ark, monkeypatch):
    import torch
    from paper_1104_0672_gb300 import _native
    g, k, x = _setup(ark, 256)
    gg = torch.flip(x, dims=[1]).contiguous()
    # the knot gradient alone: its projection is the only tensor-core kernel of the call
    _, gk0 = ark.convolve_backward(g, k, x, gg, need_map_grad=False, flags=ark.FLAG_3XTF32)
    ark.sync_status()
    monkeypatch.setenv("ARKCOS_TEST_WITHHOLD_MMA", "1")
    ark.convolve_backward(g, k, x, gg, need_map_grad=False, flags=ark.FLAG_3XTF32)
    with pytest.raises(_native.ArkcosError) as e:
        ark.sync_status()
    assert e.value.status == _native.ETIMEOUT
    monkeypatch.delenv("ARKCOS_TEST_WITHHOLD_MMA")
    _, gk = ark.convolve_backward(g, k, x, gg, need_map_grad=False, flags=ark.FLAG_3XTF32)
    ark.sync_status()
    assert torch.equal(gk, gk0)
    assert np.isfinite(gk.cpu().numpy()).all()
