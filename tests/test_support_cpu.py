"""Support-radius chooser (Sec. 4 truncation error, Sec. 2 Legendre convention): pins to closed
forms and identities, CPU only."""
import math

import numpy as np
import pytest

from paper_1104_0672_gb300 import support


def _legendre(lmax, z):
    p = np.zeros(lmax + 2)
    p[0] = 1.0
    if lmax + 1 >= 1:
        p[1] = z
    for l in range(2, lmax + 2):
        p[l] = ((2 * l - 1) * z * p[l - 1] - (l - 1) * p[l - 2]) / l
    return p


def test_top_hat_cap_closed_form():
    """f = 1 on the cap gamma <= a: K_0 = 2 pi (1 - cos a) (the cap's area) and, from
    int P_l = (P_{l+1} - P_{l-1}) / (2l + 1), K_l = 2 pi (P_{l-1}(c) - P_{l+1}(c)) / (2l + 1)."""
    a, lmax = 0.3, 60
    k = support.legendre_coefficients(lambda g: np.ones_like(g), lmax, 0.0, a)
    c = math.cos(a)
    p = _legendre(lmax, c)
    ref = np.empty(lmax + 1)
    ref[0] = 2 * math.pi * (1 - c)
    for l in range(1, lmax + 1):
        ref[l] = 2 * math.pi * (p[l - 1] - p[l + 1]) / (2 * l + 1)
    assert np.max(np.abs(k - ref)) < 1e-10


def test_whole_sphere_constant():
    """f = 1 everywhere: K_l = 4 pi delta_l0."""
    k = support.legendre_coefficients(lambda g: np.ones_like(g), 20)
    assert abs(k[0] - 4 * math.pi) < 1e-10 and np.max(np.abs(k[1:])) < 1e-10


def test_gaussian_beam_small_angle():
    """A normalised Gaussian of width s << 1: K_l -> exp(-l (l + 1) s^2 / 2) (flat-sky limit),
    to O(s^2)."""
    s = 5 * math.pi / (180 * 60) / math.sqrt(8 * math.log(2))  # 5' FWHM
    f = lambda g: np.exp(-0.5 * (g / s) ** 2) / (2 * math.pi * s * s)
    lmax = 2000
    k = support.legendre_coefficients(f, lmax, 0.0, 12 * s)
    ell = np.arange(lmax + 1)
    ref = np.exp(-0.5 * ell * (ell + 1) * s * s)
    assert np.max(np.abs(k - ref)) < 1e-4


def test_parseval_for_white_spectrum():
    """With C_l = 1 the variance sum is the kernel's squared norm on the sphere:
    sum_l (2l + 1) / (4 pi) K_l^2 = 2 pi int f(gamma)^2 sin gamma dgamma (addition theorem)."""
    s = 0.05
    f = lambda g: np.exp(-0.5 * (g / s) ** 2)
    lmax = 400
    var = support.output_variance(f, np.ones(lmax + 1))
    integrate = pytest.importorskip("scipy.integrate")
    norm2 = 2 * math.pi * integrate.quad(lambda g: f(g) ** 2 * math.sin(g), 0.0, math.pi,
                                         epsabs=1e-16, epsrel=1e-13, limit=400, points=[s, 5 * s])[0]
    assert abs(var - norm2) < 1e-9 * norm2


def test_truncation_error_is_the_tail():
    """sigma^2 of the truncation at gamma_max equals the variance of convolving with the
    tail alone, and vanishes for the whole sphere."""
    s = 0.04
    f = lambda g: np.exp(-0.5 * (g / s) ** 2)
    cl = 1.0 / (np.arange(301) + 1.0) ** 2
    gm = 2.5 * s
    tail = lambda g: np.where(g > gm, f(g), 0.0)
    e = support.truncation_error(f, gm, cl)
    k_tail = support.legendre_coefficients(f, 300, gm, support.support_end(f))
    w = (2 * np.arange(301) + 1) / (4 * math.pi) * cl
    assert abs(e - w @ k_tail ** 2) < 1e-15 + 1e-12 * e
    assert support.truncation_error(f, math.pi, cl) == 0.0
    assert e > 0.0 and tail(np.array([gm * 1.01]))[0] > 0.0
    k_tail_full = support.legendre_coefficients(f, 300, gm, math.pi)
    assert np.max(np.abs(k_tail - k_tail_full)) < 1e-12


@pytest.mark.parametrize("tol", [1e-3, 1e-5])
def test_choose_support_is_minimal(tol):
    s = 5 * math.pi / (180 * 60) / math.sqrt(8 * math.log(2))
    f = lambda g: np.exp(-0.5 * (g / s) ** 2) / (2 * math.pi * s * s)
    ell = np.arange(4097)
    cl = np.where(ell >= 2, 1.0 / (ell * (ell + 1.0) + 1e-300), 0.0)
    gm = support.choose_support(f, cl, tol)
    var = support.output_variance(f, cl)
    assert support.truncation_error(f, gm, cl) <= tol * tol * var * (1 + 1e-9)
    assert support.truncation_error(f, gm * 0.98, cl) > tol * tol * var
    # a tighter tolerance needs a larger support; the 5' beam needs a few FWHM
    assert 1.0 * 5 * math.pi / (180 * 60) < gm < 6 * 5 * math.pi / (180 * 60)


def test_kernel_for_tolerance_tabulates_the_chosen_support():
    """The support radius the tolerance picks meets the Sec. 4 bound, a 2% smaller one does not,
    and the knots are the profile at t gamma_max / (T - 1), as Kernel() takes them."""
    s = 40 * math.pi / (180 * 60) / math.sqrt(8 * math.log(2))
    f = lambda g: np.exp(-0.5 * (g / s) ** 2) / (2 * math.pi * s * s)
    cl = support.white_spectrum(767, 12 * 256 ** 2)
    r = support.kernel_for_tolerance(f, cl, 1e-3, nknots=64)
    gm, var = r["gamma_max"], support.output_variance(f, cl)
    assert r["rel_error"] <= 1e-3 * (1 + 1e-9)
    assert support.truncation_error(f, 0.98 * gm, cl) > 1e-6 * var
    g = gm * np.arange(64) / 63
    assert np.array_equal(r["knots"], f(g))
    assert abs(cl.sum() * 12 * 256 ** 2 / (4 * math.pi) - 768) < 1e-9


@pytest.mark.parametrize("l,m", [(40, 7), (512, 300), (2000, 700), (3500, 2000)])
def test_normalised_legendre_orthonormal(l, m):
    """The seeded Y_lm inputs use orthonormal associated Legendre functions:
    2 pi int_{-1}^{1} lambda_l^m(x)^2 dx = 1 and lambda_l^m is orthogonal to lambda_{l-2}^m, up
    to the high orders where an unscaled recurrence's start value sin^m underflows."""
    from paper_1104_0672_gb300 import inputs
    x, w = np.polynomial.legendre.leggauss(l + 64)
    lam = inputs._legendre_norm(l, m, x)
    assert abs(2 * math.pi * (w @ lam[l] ** 2) - 1.0) < 1e-10
    assert abs(2 * math.pi * (w @ (lam[l] * lam[l - 2]))) < 1e-10
