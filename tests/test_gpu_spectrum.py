"""Accuracy of the method against the exact spherical convolution as a function of multipole
(the Sec. 4.3 power-spectrum accuracy study, 6' FWHM Gaussian, not band-limited at l = 4096).

A single Y_lm is an eigenfunction of a radial convolution (Sec. 2, s_lm = K_l r_lm), so the
exact output is b_l Y_lm, b_l the Legendre coefficient of the tabulated profile; the error per
multipole is the frac RMS of output - b_l input over the whole nside-2048 map, for 24 values of
l from 2 to 4096 (m = 2l/3: a mix of ring frequencies that the polar-cap rings represent only
down to their own Nyquist frequency).  The envelope below is the measured curve with a factor
of two of margin; the paper quotes < 1e-3 for the power spectrum.  With the 18' support a
ring's band spans 33 input rings at the equator, wider than the 32-slot tensor-core tile, so
the 3xTF32 flag runs the CUDA-core generation here (the two forms give the same maps)."""
import math

import numpy as np
import pytest

import oracle
from paper_1104_0672_gb300 import inputs

pytestmark = pytest.mark.gpu

NSIDE = 2048
FWHM = 6 * inputs.ARCMIN
GMAX = 18 * inputs.ARCMIN
ELLS = [int(round(v)) for v in np.geomspace(2, 4096, 24)]


def envelope(l):
    """Largest accepted error at multipole l (measured: 1.2e-5 - 1.5e-5 up to l = 1515, 2.5e-5
    at 2111, 9.8e-5 at 2940, 8.1e-4 at 4096)."""
    return 3e-5 if l <= 1600 else (6e-5 if l <= 2500 else (2e-4 if l <= 3500 else 2e-3))


def error_curve(ark, form, ells=ELLS):
    """[(l, m, frac RMS error)] of the GPU convolution of real Y_lm maps against b_l Y_lm."""
    import torch
    from paper_1104_0672_gb300 import support
    spec = ("healpix", NSIDE)
    g = ark.Grid.healpix(NSIDE)
    th_r, ph0, w, n, off = oracle.geometry(spec)
    _, ph = inputs.centres(spec)
    knots = inputs.gaussian_knots(FWHM, GMAX, 256)
    T = knots.size
    ut = 4 * np.sin(0.5 * GMAX * np.arange(T) / (T - 1)) ** 2
    # the profile as the library tabulates it: linear in u between the knots, zero past u_max
    prof = lambda gam: np.where(4 * np.sin(0.5 * gam) ** 2 <= ut[-1],
                                np.interp(4 * np.sin(0.5 * gam) ** 2, ut, knots), 0.0)
    b = support.legendre_coefficients(prof, max(ells), 0.0, GMAX)
    ringid = np.repeat(np.arange(len(n)), n)
    cases = [(l, (2 * l) // 3) for l in ells]
    x = np.empty((len(cases), int(n.sum())), dtype=np.float32)
    for c, (l, m) in enumerate(cases):
        x[c] = inputs._legendre_norm(l, m, np.cos(th_r))[l][ringid] * np.cos(m * ph + 0.3)
    k = ark.Kernel(g, knots, GMAX)
    y = ark.convolve(g, k, torch.from_numpy(x).to(torch.device("cuda:0")), form).cpu().numpy()
    out = []
    for c, (l, m) in enumerate(cases):
        ref = b[l] * x[c].astype(np.float64)
        out.append((l, m, float(np.linalg.norm(y[c] - ref) / np.linalg.norm(ref))))
    return out


def test_error_spectrum_6arcmin():
    import paper_1104_0672_gb300 as ark
    res = error_curve(ark, ark.FLAG_3XTF32)
    bad = [(l, m, e) for l, m, e in res if not e < envelope(l)]
    assert not bad, bad
