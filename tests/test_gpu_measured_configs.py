"""Parity of the exact configurations the benchmark times, through the C ABI.

* The headline step: 16 HEALPix nside-2048 maps with one shared 5' Gaussian beam (15' support,
  256 knots), after `autotune()` has installed its launch shape on these buffers exactly as
  `bench.py` does, in the 3xTF32 tensor-core form and in the plain FP32 form.  Maps 0, 7 and 15
  (first, middle and last of the contraction's map loop) are compared with the FP64 oracle on a
  ring subset covering both poles, the first rings of each Bluestein buffer class, the cap/belt
  boundaries and the equator.
* The backward pass of the nside-2048 configuration (map and knot gradients) in both forms:
  the map gradient against the oracle's transposed operator on a ring subset; the knot gradient
  against central differences of J = <g, L(f) x> (exact for any step, since L is linear in the
  knots) and against the Euler identity sum_t f_t dJ/df_t = J.

Tolerance: fractional RMS <= 1e-5 against the oracle (the accuracy the paper states, Sec. 1
and Sec. 4.3).  The finite-difference bounds follow from that bar by Cauchy-Schwarz: a forward
map within frac RMS eps of the exact one gives |J_computed - J| <= eps ||g|| ||y||."""
import numpy as np
import pytest

import oracle
from paper_1104_0672_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5
NSIDE = 2048


@pytest.fixture(scope="module")
def ark():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need CUDA")
    import paper_1104_0672_gb300 as ark
    return ark


def _frac(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _rings():
    """Output rings that exercise every code path of the transforms and the contraction at
    nside 2048: pole rings (pole fix), short cap rings (staged fold), the first ring of each
    FFT buffer class (n = 1028: M 4096 Bluestein; 2052: M 8192; 4100: M 16384), the last cap
    ring, the first belt rings (shifted and unshifted), the equator and their mirrors."""
    ns = NSIDE
    R = 4 * ns - 1
    north = [0, 1, 2, 9, 256, 257, 512, 513, 1024, 1025, ns - 2, ns - 1, ns, ns + 1, 2 * ns - 1]
    south = [R - 1 - i for i in (0, 1, 257, 1025, ns - 1, ns)]
    return sorted(set(north + south))


def _pix(rings):
    th, ph, w, n, off = oracle.geometry(("healpix", NSIDE))
    return np.concatenate([np.arange(off[i], off[i] + n[i]) for i in rings])


@pytest.fixture(scope="module")
def headline(ark):
    """The bench's maps and beam, and the oracle on maps 0, 7, 15 (shared by both forms)."""
    import torch
    g = ark.Grid.healpix(NSIDE)
    gmax = 15 * inputs.ARCMIN
    knots = inputs.gaussian_knots(5 * inputs.ARCMIN, gmax, 256)
    k = ark.Kernel(g, knots, gmax)
    xh = inputs.white_noise(g.npix, 16, config=3)  # the bench's maps (rank 0)
    rings = _rings()
    refs = {b: oracle.convolve(("healpix", NSIDE), knots, gmax, xh[b].astype(np.float64), rings=rings)
            for b in (0, 7, 15)}
    x = torch.from_numpy(xh).to(torch.device("cuda:0"))
    return g, k, x, rings, refs


@pytest.mark.parametrize("form", ["tf32", "fp32"])
def test_headline_batch_autotuned(ark, headline, form):
    import torch
    g, k, x, rings, refs = headline
    flags = ark.FLAG_3XTF32 if form == "tf32" else 0
    y = torch.empty_like(x)
    ws = torch.empty(ark.workspace_size(g, k, 16), dtype=torch.uint8, device=x.device)
    shape = ark.autotune(g, k, x, flags=flags, out=y, workspace=ws)
    y.fill_(float("nan"))
    ark.convolve(g, k, x, out=y, workspace=ws, flags=flags)
    ark.sync_status()
    pix = _pix(rings)
    for b, ref in refs.items():
        got = y[b].cpu().numpy()
        assert np.isfinite(got).all(), b
        err = _frac(got[pix], ref[pix])
        assert err < TOL, (form, shape, b, err)
    # the shape the tuner chose is the one later calls keep using: a second call is identical
    y2 = ark.convolve(g, k, x, workspace=ws, flags=flags)
    assert torch.equal(y, y2)


@pytest.mark.parametrize("form", ["tf32", "fp32"])
def test_backward_nside2048_full_size(ark, form):
    import torch
    dev = torch.device("cuda:0")
    spec = ("healpix", NSIDE)
    g = ark.Grid.healpix(NSIDE)
    gmax = 15 * inputs.ARCMIN
    knots = inputs.gaussian_knots(5 * inputs.ARCMIN, gmax, 256)
    k = ark.Kernel(g, knots, gmax)
    flags = ark.FLAG_3XTF32 if form == "tf32" else 0
    x = torch.from_numpy(inputs.white_noise(g.npix, 1, config=3)).to(dev)
    # g correlated with the output, so that J and its knot derivatives are far above the
    # roundoff of a dot product over 50M pixels
    y0 = ark.convolve(g, k, x, flags)
    gg = (y0 + 0.1 * y0.std() * torch.from_numpy(inputs.white_noise(g.npix, 1, config=3, salt=5)).to(dev))
    gin, gk = ark.convolve_backward(g, k, x, gg, flags=flags)
    ark.sync_status()
    # map gradient: the transposed operator (oracle) on a ring subset
    rings = _rings()
    pix = _pix(rings)
    refa = oracle.adjoint(spec, knots, gmax, gg[0].cpu().numpy().astype(np.float64), rings=rings)
    assert _frac(gin[0].cpu().numpy()[pix], refa[pix]) < TOL
    # knot gradient: central differences (exact up to the forward's error bar, L linear in f)
    gk = gk[0].cpu().numpy()
    gnorm = float(gg.double().norm())
    h = 64.0 * float(np.abs(knots).max())
    for t in (0, 40, 120, 200, 255):
        e = np.zeros_like(knots)
        e[t] = h
        k.update_knots(knots + e)
        yp = ark.convolve(g, k, x, flags).double()
        k.update_knots(knots - e)
        ym = ark.convolve(g, k, x, flags).double()
        jp, jm = float((gg.double() * yp).sum()), float((gg.double() * ym).sum())
        fd = (jp - jm) / (2 * h)
        bound = TOL * gnorm * (float(yp.norm()) + float(ym.norm())) / (2 * h) + TOL * np.abs(gk).max()
        assert abs(fd - gk[t]) <= bound, (t, fd, gk[t], bound)
    k.update_knots(knots)
    y = ark.convolve(g, k, x, flags).double()
    J = float((gg.double() * y).sum())
    assert abs(float(np.dot(knots, gk)) - J) <= TOL * (gnorm * float(y.norm()) + float(np.abs(knots * gk).sum()))
