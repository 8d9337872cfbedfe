"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(brute force on tiny grids, the Funk-Hecke closed form, invariants, transposition and
finite-difference identities).  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_1104_0672_gb300 import inputs
from tests import brute

def _gauss(fwhm_deg, cut_deg, T=64):
    return inputs.gaussian_knots(fwhm_deg * inputs.DEG, cut_deg * inputs.DEG, T), cut_deg * inputs.DEG


# Support radii in these tests are chosen off the grid spacings: a truncated profile
# jumps at gamma_max, and a sample lying exactly on the edge would be kept or dropped
# depending on the last bit of its squared chord.


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------- geometry
@pytest.mark.parametrize("nside", [1, 2, 4, 8, 256])
def test_healpix_geometry(oracle_lib, nside):
    th, ph, w, n, off = oracle.geometry(("healpix", nside))
    assert len(th) == 4 * nside - 1
    assert n.sum() == 12 * nside * nside
    assert np.allclose(th + th[::-1], math.pi, atol=1e-14)
    assert abs(w.sum() * 1 - 4 * math.pi / (12 * nside * nside) * len(w)) < 1e-12
    assert abs(np.sum(w * n) - 4 * math.pi) < 1e-12
    # independent pixel-centre implementation
    thp, php = inputs.healpix_centres(nside)
    assert np.allclose(np.repeat(th, n), thp, atol=1e-13)
    assert np.allclose(np.repeat(ph, n), php - 2 * math.pi * (np.arange(thp.size) - np.repeat(off, n)) / np.repeat(n, n), atol=1e-13)


def test_healpix_equal_area_rings(oracle_lib):
    # each ring's area 2 pi (cos of boundaries) equals n_ring * 4 pi / npix; checked by the
    # z spacing: cap ring i has z = 1 - i^2/(3 ns^2) and equatorial z steps 2/(3 ns)
    ns = 16
    th, ph, w, n, off = oracle.geometry(("healpix", ns))
    z = np.cos(th)
    assert np.allclose(np.diff(z[ns - 1:3 * ns]), -2.0 / (3 * ns), atol=1e-13)
    assert np.allclose(1 - z[:ns - 1], (np.arange(1, ns) ** 2) / (3.0 * ns * ns), atol=1e-14)


@pytest.mark.parametrize("nt,nphi", [(8, 16), (128, 256), (7, 10)])
def test_ecp_weights(oracle_lib, nt, nphi):
    th, ph, w, n, off = oracle.geometry(("ecp", nt, nphi))
    assert abs(np.sum(w * n) - 4 * math.pi) < 1e-12
    # Fejer's first rule integrates cos^k(theta) sin(theta) exactly for k < nt
    for k in range(0, nt):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.sum(w * nphi / (2 * math.pi) * np.cos(th) ** k) - exact) < 1e-12


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("grid", [("ecp", 8, 16), ("ecp", 16, 32), ("ecp", 12, 18)])
def test_ecp_equals_true_direct_sum(oracle_lib, grid):
    """On ECP every ring has N pixels and no offset, so the hybrid equals the true-profile
    direct sum to roundoff (Sec. 4.3, last paragraph)."""
    # the cut (58 deg) is not a multiple of any grid spacing here, so no sample sits
    # exactly on the support edge, where the truncated profile jumps
    knots, gm = _gauss(30.0, 58.0, T=48)
    r = inputs.white_noise(inputs.npix(grid), 1, config=1, dtype=np.float64)[0]
    a = oracle.convolve(grid, knots, gm, r)
    b = brute.direct_true(grid, knots, gm, r)
    assert _rel(a, b) < 1e-12


@pytest.mark.parametrize("nside", [1, 2, 4, 8])
@pytest.mark.parametrize("pole_fix", [False, True])
def test_healpix_equals_interpolant_direct_sum(oracle_lib, nside, pole_fix):
    """The hybrid steps equal a direct sum with the trigonometric interpolant of the
    N-point kernel samples; pole rings equal the true direct sum (Sec. 4.2)."""
    grid = ("healpix", nside)
    knots, gm = _gauss(40.0 / nside, 86.0 / nside, T=40)
    r = inputs.white_noise(inputs.npix(grid), 1, config=2, dtype=np.float64)[0]
    a = oracle.convolve(grid, knots, gm, r, pole_fix=pole_fix)
    b = brute.hybrid_brute(grid, knots, gm, r, pole_fix=pole_fix)
    assert _rel(a, b) < 1e-12


@pytest.mark.parametrize("nside", [2, 4])
def test_healpix_no_shift_fix_and_basic(oracle_lib, nside):
    grid = ("healpix", nside)
    knots, gm = _gauss(40.0 / nside, 86.0 / nside, T=40)
    r = inputs.white_noise(inputs.npix(grid), 1, config=2, dtype=np.float64)[0]
    a = oracle.convolve(grid, knots, gm, r, shift_fix=False, pole_fix=False)
    b = brute.hybrid_brute(grid, knots, gm, r, shift_fix=False, pole_fix=False)
    assert _rel(a, b) < 1e-12
    a = oracle.convolve(grid, knots, gm, r, variant="basic", pole_fix=False)
    b = brute.hybrid_brute(grid, knots, gm, r, variant="basic", pole_fix=False)
    assert _rel(a, b) < 1e-12


def test_healpix_equatorial_rings_exact(oracle_lib):
    """Output rings whose whole band is equatorial equal the true direct sum to roundoff
    (the ringing cancels exactly there, Sec. 4.3)."""
    ns = 8
    grid = ("healpix", ns)
    knots, gm = _gauss(8.0, 14.0, T=64)
    th, ph, w, n, off = oracle.geometry(grid)
    r = inputs.white_noise(inputs.npix(grid), 1, config=2, dtype=np.float64)[0]
    eq = [i for i in range(len(th)) if all(n[j] == 4 * ns for j in range(len(th))
                                         if abs(th[i] - th[j]) <= gm)]
    assert len(eq) >= 5
    a = oracle.convolve(grid, knots, gm, r, rings=eq)
    pix = np.concatenate([np.arange(off[i], off[i] + n[i]) for i in eq])
    b = brute.direct_true(grid, knots, gm, r, pix)
    assert _rel(a[pix], b) < 1e-12
    # without the shift fix these rings are no longer exact
    c = oracle.convolve(grid, knots, gm, r, rings=eq, shift_fix=False)
    assert _rel(c[pix], b) > 1e-6


def test_direct_matches_brute(oracle_lib):
    grid = ("healpix", 4)
    knots, gm = _gauss(10.0, 25.0, T=64)
    r = inputs.white_noise(inputs.npix(grid), 1, config=2, dtype=np.float64)[0]
    assert _rel(oracle.direct(grid, knots, gm, r), brute.direct_true(grid, knots, gm, r)) < 1e-12


# ---------------------------------------------------------------- closed forms
def test_funk_hecke_ecp(oracle_lib):
    """Config 1: ECP 128x256, Gaussian FWHM 4 deg cut at 12 deg, 256 knots.  A Y_lm input
    comes out scaled by the kernel's Legendre coefficient b_l (Sec. 2, Eq. lspacedef), up to
    the quadrature error of the pixelisation (Sec. 2, last paragraph).  Measured worst frac
    RMS 1.53e-5 here (the oracle itself equals the direct sum to 1e-15); the bound is 2x."""
    grid = ("ecp", 128, 256)
    knots = inputs.gaussian_knots(4 * inputs.DEG, 12 * inputs.DEG, 256)
    gm = 12 * inputs.DEG
    th, ph = inputs.centres(grid)
    b = brute.legendre_coeffs(knots, gm, 40)
    worst = 0.0
    for (l, m) in [(0, 0), (1, 0), (2, 1), (7, 3), (20, 20), (33, 5), (40, 17)]:
        y = inputs.ylm_real(l, m, th, ph, 0.3)
        out = oracle.convolve(grid, knots, gm, y)
        worst = max(worst, _rel(out, b[l] * y))
    assert worst < 3.1e-5, worst


@pytest.mark.parametrize("l,m,bound", [(2, 1, 1e-4), (20, 7, 1e-4), (60, 30, 1e-4), (158, 64, 3e-4)])
def test_funk_hecke_healpix(oracle_lib, l, m, bound):
    """On HEALPix (nside 128, 1.5 deg FWHM, 4.5 deg cut) a Y_lm comes out scaled by b_l too,
    up to the method's own error: 2.8e-5, 2.8e-5, 2.6e-5 and 1.0e-4 measured for these (l, m)
    (it grows where b_l is small, 6.9e-4 at l = 2 nside).  A dropped term, a wrong phase sign or
    a transposed ring index shows up orders of magnitude above the bound."""
    spec = ("healpix", 128)
    th, ph = inputs.centres(spec)
    gm = 4.5 * inputs.DEG
    knots = inputs.gaussian_knots(1.5 * inputs.DEG, gm, 256)
    b = brute.legendre_coeffs(knots, gm, l)
    y = inputs.ylm_real(l, m, th, ph, 0.3)
    out = oracle.convolve(spec, knots, gm, y)
    assert _rel(out, b[l] * y) < bound


def test_funk_hecke_converges(oracle_lib):
    """The quadrature error vanishes as grid and profile table are refined: at 256x512 with
    4096 knots the Y_lm eigen-relation holds to 3.2e-8 (measured; bound 1e-7)."""
    grid = ("ecp", 256, 512)
    knots = inputs.gaussian_knots(4 * inputs.DEG, 12 * inputs.DEG, 4096)
    gm = 12 * inputs.DEG
    th, ph = inputs.centres(grid)
    b = brute.legendre_coeffs(knots, gm, 40, nodes=8)
    for (l, m) in [(7, 3), (40, 17)]:
        y = inputs.ylm_real(l, m, th, ph, 0.3)
        out = oracle.convolve(grid, knots, gm, y)
        assert _rel(out, b[l] * y) < 1e-7


def test_constant_map(oracle_lib):
    """A constant map is multiplied by sum_q w_q f(gamma_pq) -> K_0 = 2 pi int f dz, up to
    quadrature error (measured max 1.67e-5 relative at 64x128; bound 2x)."""
    grid = ("ecp", 64, 128)
    knots = inputs.gaussian_knots(8 * inputs.DEG, 24 * inputs.DEG, 256)
    gm = 24 * inputs.DEG
    out = oracle.convolve(grid, knots, gm, np.ones(inputs.npix(grid)))
    b0 = brute.legendre_coeffs(knots, gm, 0)[0]
    assert np.max(np.abs(out - b0)) / b0 < 3.4e-5


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("grid", [("healpix", 4), ("ecp", 16, 32)])
def test_linearity(oracle_lib, grid):
    knots, gm = _gauss(15.0, 35.0, T=32)
    g = inputs.rng(5)
    r1, r2 = g.standard_normal((2, inputs.npix(grid)))
    a = oracle.convolve(grid, knots, gm, 2.5 * r1 - 0.75 * r2)
    b = 2.5 * oracle.convolve(grid, knots, gm, r1) - 0.75 * oracle.convolve(grid, knots, gm, r2)
    assert _rel(a, b) < 1e-13


@pytest.mark.parametrize("grid,variant,pole", [
    (("healpix", 4), "enhanced", True), (("healpix", 4), "enhanced", False),
    (("healpix", 2), "basic", True), (("ecp", 10, 16), "enhanced", True)])
def test_adjoint_dot(oracle_lib, grid, variant, pole):
    """<g, L r> = <L^T g, r> for the transposed steps."""
    knots, gm = _gauss(20.0, 43.7, T=32)
    g = inputs.rng(6)
    r, gg = g.standard_normal((2, inputs.npix(grid)))
    Lr = oracle.convolve(grid, knots, gm, r, variant=variant, pole_fix=pole)
    Ltg = oracle.adjoint(grid, knots, gm, gg, variant=variant, pole_fix=pole)
    lhs, rhs = np.dot(gg, Lr), np.dot(Ltg, r)
    assert abs(lhs - rhs) <= 1e-12 * (np.linalg.norm(gg) * np.linalg.norm(Lr))


def test_healpix_self_adjoint(oracle_lib):
    """With equal pixel weights and no pole fix the ENHANCED HEALPix operator is symmetric."""
    grid = ("healpix", 4)
    knots, gm = _gauss(20.0, 43.7, T=32)
    gg = inputs.rng(7).standard_normal(inputs.npix(grid))
    a = oracle.adjoint(grid, knots, gm, gg, pole_fix=False)
    b = oracle.convolve(grid, knots, gm, gg, pole_fix=False)
    assert _rel(a, b) < 1e-13


@pytest.mark.parametrize("grid,pole", [(("healpix", 2), True), (("healpix", 4), False),
                                       (("ecp", 8, 12), True)])
def test_knot_gradient(oracle_lib, grid, pole):
    """L is linear in the knots: central differences are exact up to roundoff, and
    sum_t f_t dJ/df_t = J (Euler)."""
    knots, gm = _gauss(25.0, 48.3, T=12)
    g = inputs.rng(8)
    r, gg = g.standard_normal((2, inputs.npix(grid)))
    grad = oracle.knot_grad(grid, knots, gm, r, gg, pole_fix=pole)
    J = np.dot(gg, oracle.convolve(grid, knots, gm, r, pole_fix=pole))
    assert abs(np.dot(knots, grad) - J) < 1e-11 * max(1.0, abs(J))
    h = 0.37
    for t in [0, 3, 7, 11]:
        e = np.zeros_like(knots)
        e[t] = h
        jp = np.dot(gg, oracle.convolve(grid, knots + e, gm, r, pole_fix=pole))
        jm = np.dot(gg, oracle.convolve(grid, knots - e, gm, r, pole_fix=pole))
        fd = (jp - jm) / (2 * h)
        assert abs(fd - grad[t]) < 1e-10 * max(1.0, np.abs(grad).max()), (t, fd, grad[t])


def test_healpix_rotation_and_flip_equivariance(oracle_lib):
    """A 90 deg rotation about z moves every pixel by n_ring/4 along its ring; the N-S flip
    reverses the ring order.  The output follows both exactly."""
    ns = 4
    grid = ("healpix", ns)
    th, ph, w, n, off = oracle.geometry(grid)
    knots, gm = _gauss(15.0, 35.0, T=32)
    r = inputs.rng(9).standard_normal(inputs.npix(grid))

    def rot(x):
        y = np.empty_like(x)
        for i in range(len(n)):
            y[off[i]:off[i] + n[i]] = np.roll(x[off[i]:off[i] + n[i]], n[i] // 4)
        return y

    def flip(x):
        y = np.empty_like(x)
        for i in range(len(n)):
            j = len(n) - 1 - i
            y[off[i]:off[i] + n[i]] = x[off[j]:off[j] + n[j]]
        return y

    out = oracle.convolve(grid, knots, gm, r)
    assert _rel(oracle.convolve(grid, knots, gm, rot(r)), rot(out)) < 1e-13
    assert _rel(oracle.convolve(grid, knots, gm, flip(r)), flip(out)) < 1e-13


def test_ecp_roll_equivariance(oracle_lib):
    grid = ("ecp", 12, 20)
    knots, gm = _gauss(20.0, 40.0, T=32)
    r = inputs.rng(10).standard_normal(inputs.npix(grid)).reshape(12, 20)
    out = oracle.convolve(grid, knots, gm, r.ravel()).reshape(12, 20)
    out2 = oracle.convolve(grid, knots, gm, np.roll(r, 3, axis=1).ravel()).reshape(12, 20)
    assert _rel(out2, np.roll(out, 3, axis=1)) < 1e-13
