"""The support radius chosen from a tolerance (Sec. 4 truncation-error estimate) on the GPU: a
kernel built by Kernel.for_tolerance convolves white noise with the truncation error the
estimate predicts.  The reference is the same Gaussian with a support of 5 FWHM (tail below
1e-29 of the peak); the measured relative difference must lie within a factor of two of the
predicted sigma / rms (a missing 2l + 1, 4 pi or a squared coefficient would put it off by
orders of magnitude)."""
import math

import numpy as np
import pytest

from paper_1104_0672_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tol", [1e-2, 1e-3])
def test_tolerance_kernel_meets_its_estimate(tol):
    import torch

    import paper_1104_0672_gb300 as ark
    g = ark.Grid.healpix(256)
    fwhm = 40 * inputs.ARCMIN
    s = fwhm / math.sqrt(8 * math.log(2))
    f = lambda gam: np.exp(-0.5 * (gam / s) ** 2) / (2 * math.pi * s * s)
    kt = ark.Kernel.for_tolerance(g, f, tol)
    gfull = 5 * fwhm
    kf = ark.Kernel(g, f(gfull * np.arange(1024) / 1023), gfull)
    x = torch.from_numpy(inputs.white_noise(g.npix, 2, config=34)).to(torch.device("cuda:0"))
    yt = ark.convolve(g, kt, x).double()
    yf = ark.convolve(g, kf, x).double()
    ark.sync_status()
    measured = float((yt - yf).norm() / yf.norm())
    assert kt.gamma_max < gfull and kt.rel_error <= tol * (1 + 1e-9)
    assert 0.5 * kt.rel_error <= measured <= 2.0 * kt.rel_error, (measured, kt.rel_error, kt.gamma_max)
