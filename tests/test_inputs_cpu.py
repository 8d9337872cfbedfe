"""Pins of the harness-side inverse spherical-harmonic transform that makes the seeded
C_l random fields (inputs.random_alm, inputs.synthesize_healpix).  CPU only: the same torch
code runs on the GPU for the full-size field."""
import math

import numpy as np
import pytest

from paper_1104_0672_gb300 import inputs


@pytest.mark.parametrize("l,m", [(0, 0), (1, 0), (2, 1), (7, 7), (17, 11), (33, 5), (40, 1), (40, 40)])
def test_synthesis_of_single_harmonics(l, m):
    """One coefficient a_lm = e^{i 0.7} (m > 0; its conjugate partner a_{l,-m} implied) gives
    2 Re(e^{i 0.7} Y_lm), and a real a_l0 gives a_l0 Y_l0, at every pixel centre: checked
    against the scalar per-(l, m) recurrence of inputs.ylm_real.  l_max = 40 > 2 nside, so
    the cap rings fold modes above their own Nyquist frequency."""
    ns, lmax = 16, 40
    th, ph = inputs.healpix_centres(ns)
    alm = np.zeros((lmax + 1, lmax + 1), complex)
    alm[m, l] = np.exp(0.7j) if m > 0 else 1.3
    got = inputs.synthesize_healpix(ns, alm)
    ref = 2 * inputs.ylm_real(l, m, th, ph, 0.7) if m > 0 else 1.3 * inputs.ylm_real(l, 0, th, ph)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_synthesis_is_linear_in_the_coefficients():
    ns, lmax = 8, 24
    a1 = inputs.random_alm(lmax, np.ones(lmax + 1), config=30, salt=1)
    a2 = inputs.random_alm(lmax, np.ones(lmax + 1), config=30, salt=2)
    t1, t2 = inputs.synthesize_healpix(ns, a1), inputs.synthesize_healpix(ns, a2)
    t12 = inputs.synthesize_healpix(ns, 2.0 * a1 - 0.5 * a2)
    assert np.abs(t12 - (2.0 * t1 - 0.5 * t2)).max() < 1e-12 * np.abs(t12).max()


def test_random_alm_statistics():
    """E|a_lm|^2 = C_l (m > 0 complex, m = 0 real), zero below the diagonal, seeded."""
    lmax = 512
    ell = np.arange(lmax + 1, dtype=np.float64)
    cl = np.zeros(lmax + 1)
    cl[1:] = 1.0 / (ell[1:] * (ell[1:] + 1.0))
    a = inputs.random_alm(lmax, cl, config=31)
    assert np.array_equal(a, inputs.random_alm(lmax, cl, config=31))
    assert np.all(a[np.tril_indices(lmax + 1, -1)] == 0)
    assert np.all(a[0].imag == 0) and np.all(a[:, 0][1:] == 0)
    r = np.array([np.mean(np.abs(a[1:l + 1, l]) ** 2) / cl[l] for l in range(256, lmax + 1)])
    assert abs(r.mean() - 1.0) < 0.01
    r0 = np.mean(a[0, 256:].real ** 2 / cl[256:])
    assert abs(r0 - 1.0) < 0.15


def test_cl_field_pixel_variance():
    """The map variance of a field with C_l = 1/(l(l+1)) at nside 32 (l <= 64) against the
    expectation sum_l (2l+1) C_l / 4 pi, averaged over four seeds (cosmic variance of the low
    multipoles dominates the spread)."""
    ns, lmax = 32, 64
    ell = np.arange(lmax + 1, dtype=np.float64)
    cl = np.zeros(lmax + 1)
    cl[1:] = 1.0 / (ell[1:] * (ell[1:] + 1.0))
    expect = np.sum((2 * ell + 1) * cl) / (4 * math.pi)
    v = np.mean([np.mean(inputs.cl_field_healpix(ns, lmax, cl, config=32, salt=s) ** 2) for s in range(4)])
    assert 0.6 * expect < v < 1.5 * expect
