"""Several radial kernels on the same input (the Sec. 5 route to asymmetric beams: O(10)
symmetric convolutions of one map), arkcos_convolve_multi, against the FP64 oracle and against
one arkcos_convolve call per kernel.  Tolerance: frac RMS <= 1e-5 (Sec. 1, Sec. 4.3)."""
import numpy as np
import pytest

import oracle
from paper_1104_0672_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ark():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_1104_0672_gb300 as ark
    return ark


def _frac(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _kernels(ark, g, fwhms_deg):
    kn = []
    for f in fwhms_deg:
        gmax = 3 * f * inputs.DEG
        kn.append((inputs.gaussian_knots(f * inputs.DEG, gmax, 128), gmax))
    return [ark.Kernel(g, k, gm) for k, gm in kn], kn


@pytest.mark.parametrize("form", ["fp32", "tf32"])
def test_multi_outputs_and_weighted_sum_vs_oracle(ark, form):
    import torch
    spec = ("healpix", 64)
    g = ark.Grid.healpix(64)
    ks, kn = _kernels(ark, g, (1.0, 1.6, 2.3))
    fl = ark.FLAG_3XTF32 if form == "tf32" else 0
    x = inputs.white_noise(g.npix, 2, config=31)
    xt = torch.from_numpy(x).to(torch.device("cuda:0"))
    y = ark.convolve_multi(g, ks, xt, flags=fl)  # [2, 3, npix]
    w = np.array([0.5, -1.25, 2.0])
    s = ark.convolve_multi(g, ks, xt, weights=w, flags=fl)  # [2, npix]
    ark.sync_status()
    y, s = y.cpu().numpy(), s.cpu().numpy()
    for b in range(2):
        refs = [oracle.convolve(spec, k, gm, x[b].astype(np.float64)) for k, gm in kn]
        for k in range(3):
            assert _frac(y[b, k], refs[k]) < TOL, (b, k)
        assert _frac(s[b], sum(wk * r for wk, r in zip(w, refs))) < TOL, b


def test_multi_equals_single_calls(ark):
    """One output per kernel equals the per-kernel convolve calls (same FP32 arithmetic, the
    input transformed once instead of once per kernel); 40 outputs exercise two launch groups
    of the per-map contraction and of the pole fix."""
    import torch
    g = ark.Grid.healpix(32)
    ks, _ = _kernels(ark, g, [1.5 + 0.2 * i for i in range(8)])
    xt = torch.from_numpy(inputs.white_noise(g.npix, 5, config=32)).to(torch.device("cuda:0"))
    for fl in (0, ark.FLAG_3XTF32):
        y = ark.convolve_multi(g, ks, xt, flags=fl)
        for k, kern in enumerate(ks):
            ref = ark.convolve(g, kern, xt, fl)
            d = (y[:, k] - ref).double().norm(dim=1) / ref.double().norm(dim=1)
            assert float(d.max()) < 1e-6, (fl, k, float(d.max()))
    ark.sync_status()


def test_multi_nside2048_ten_kernels_weighted(ark):
    """Ten Gaussian components of 4.5'-5.22' FWHM (support 3 FWHM) on one nside-2048 map, summed
    with weights (an O(10) decomposition at the headline resolution): against the weighted sum
    of the per-kernel convolve calls on every pixel and against the oracle on a ring subset."""
    import torch
    ns = 2048
    spec = ("healpix", ns)
    g = ark.Grid.healpix(ns)
    fw = 4.5 + 0.08 * np.arange(10)
    kn = [(inputs.gaussian_knots(f * inputs.ARCMIN, 3 * f * inputs.ARCMIN, 256), 3 * f * inputs.ARCMIN) for f in fw]
    ks = [ark.Kernel(g, k, gm) for k, gm in kn]
    w = inputs.rng(33).uniform(0.2, 1.0, 10)
    x = inputs.white_noise(g.npix, 1, config=33)
    xt = torch.from_numpy(x).to(torch.device("cuda:0"))
    s = ark.convolve_multi(g, ks, xt, weights=w, flags=ark.FLAG_3XTF32)
    ref = torch.zeros_like(s, dtype=torch.float64)
    for wk, kern in zip(w, ks):
        ref += wk * ark.convolve(g, kern, xt, ark.FLAG_3XTF32).double()
    ark.sync_status()
    assert float((s.double() - ref).norm() / ref.norm()) < 1e-6
    R = 4 * ns - 1
    rings = [0, 1, 700, ns - 1, ns, 2 * ns - 1, R - 1]
    th, ph, wr, n, off = oracle.geometry(spec)
    pix = np.concatenate([np.arange(off[i], off[i] + n[i]) for i in rings])
    orc = sum(wk * oracle.convolve(spec, k, gm, x[0].astype(np.float64), rings=rings) for wk, (k, gm) in zip(w, kn))
    assert _frac(s[0].cpu().numpy()[pix], orc[pix]) < TOL
