"""Seeded synthetic inputs for the ring convolution: maps and radial profiles.

This module holds no step of the convolution itself.  It makes the inputs that both the
CUDA path and the FP64 oracle consume: white-noise maps, point sources, real spherical
harmonics sampled at pixel centres, and tabulated radial profiles (Gaussian beams and a
spherical Mexican-hat wavelet).  Pixel centres are computed here from the published
HEALPix RING definition (Gorski et al. 2005) and the ECP definition, independently of
both the library and the oracle.

Seeds follow ``seed = 11040672 + config`` (numpy PCG64).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 11040672
ARCMIN = math.pi / (180.0 * 60.0)
DEG = math.pi / 180.0


def rng(config: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(config) + 1000 * int(salt)))


# --------------------------------------------------------------------- pixel centres
def healpix_npix(nside: int) -> int:
    return 12 * nside * nside


def healpix_centres(nside: int):
    """(theta, phi) of every pixel in RING order."""
    ns = int(nside)
    th, ph = [], []
    for r in range(1, 4 * ns):
        if r < ns:
            n, z, s = 4 * r, 1.0 - r * r / (3.0 * ns * ns), 1
            t = 2.0 * math.asin(r / (math.sqrt(6.0) * ns))
        elif r <= 3 * ns:
            n, z = 4 * ns, 4.0 / 3.0 - 2.0 * r / (3.0 * ns)
            s = 1 if (r - ns) % 2 == 0 else 0
            t = math.acos(z)
        else:
            i = 4 * ns - r
            n, s = 4 * i, 1
            t = math.pi - 2.0 * math.asin(i / (math.sqrt(6.0) * ns))
        q = np.arange(n, dtype=np.float64)
        th.append(np.full(n, t))
        ph.append((2.0 * q + s) * math.pi / n)
    return np.concatenate(th), np.concatenate(ph)


def ecp_centres(ntheta: int, nphi: int):
    t = (np.arange(ntheta) + 0.5) * math.pi / ntheta
    p = 2.0 * math.pi * np.arange(nphi) / nphi
    return np.repeat(t, nphi), np.tile(p, ntheta)


def centres(grid):
    if grid[0] == "healpix":
        return healpix_centres(grid[1])
    return ecp_centres(grid[1], grid[2])


def npix(grid) -> int:
    return healpix_npix(grid[1]) if grid[0] == "healpix" else int(grid[1]) * int(grid[2])


# --------------------------------------------------------------------- maps
def white_noise(npix: int, nmaps: int = 1, config: int = 0, salt: int = 0, dtype=np.float32):
    return rng(config, salt).standard_normal((nmaps, npix)).astype(dtype)


def point_sources(npix: int, count: int, config: int = 0, salt: int = 7):
    m = np.zeros(npix)
    idx = rng(config, salt).choice(npix, size=count, replace=False)
    m[idx] = 1.0
    return m, idx


def _legendre_norm(lmax: int, m: int, x: np.ndarray) -> np.ndarray:
    """Orthonormal associated Legendre functions lambda_l^m(x) for l = m..lmax
    (so that Y_lm = lambda_l^m(cos theta) e^{i m phi}), by the standard three-term recurrence
    in l run on scaled values: lambda_m^m = (-1)^m sqrt(1/4pi) prod_k sqrt((2k+1)/2k) sin^m
    is carried as a per-point logarithm (for large m it underflows long before the functions
    it starts do) and the recurrence renormalises whenever it grows past 1e150."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    out = np.zeros((lmax + 1, x.size))
    if m > lmax:
        return out
    logc = 0.5 * math.log(1.0 / (4.0 * math.pi)) + 0.5 * sum(math.log((2.0 * k + 1.0) / (2.0 * k))
                                                             for k in range(1, m + 1))
    with np.errstate(divide="ignore"):
        scale = logc + m * np.log(s) if m > 0 else np.full_like(x, logc)
    live = np.isfinite(scale)  # points where sin theta = 0 and m > 0 are exactly zero
    scale = np.where(live, scale, 0.0)
    sign = -1.0 if m % 2 else 1.0
    big, logbig = 1e150, math.log(1e150)

    def emit(l, v):
        with np.errstate(under="ignore"):
            out[l] = np.where(live, sign * v * np.exp(scale), 0.0)

    p_prev = np.zeros_like(x)
    p = np.ones_like(x)
    emit(m, p)
    if m + 1 <= lmax:
        p_prev, p = p, x * math.sqrt(2.0 * m + 3.0) * p
        emit(m + 1, p)
    for l in range(m + 2, lmax + 1):
        a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
        b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
        p_prev, p = p, a * (x * p - b * p_prev)
        grow = np.abs(p) > big
        if grow.any():
            p = np.where(grow, p / big, p)
            p_prev = np.where(grow, p_prev / big, p_prev)
            scale = scale + np.where(grow, logbig, 0.0)
        emit(l, p)
    return out


def ylm_real(l: int, m: int, theta: np.ndarray, phi: np.ndarray, phase: float = 0.0):
    """Re[e^{i phase} Y_lm(theta, phi)] for m >= 0 (orthonormal convention)."""
    lam = _legendre_norm(l, m, np.cos(theta))[l]
    return lam * np.cos(m * phi + phase)


def ylm_mix(grid, count: int, lmax: int, config: int = 0, salt: int = 3):
    """Sum of ``count`` real parts of unit-modulus random-phase a_lm Y_lm, l <= lmax."""
    th, ph = centres(grid)
    g = rng(config, salt)
    out = np.zeros(th.size)
    for _ in range(count):
        l = int(g.integers(0, lmax + 1))
        m = int(g.integers(0, l + 1))
        out += ylm_real(l, m, th, ph, float(g.uniform(0, 2 * math.pi)))
    return out


# --------------------------------------------------------------------- radial profiles
def knot_angles(gamma_max: float, T: int) -> np.ndarray:
    return gamma_max * np.arange(T, dtype=np.float64) / (T - 1)


def gaussian_knots(fwhm: float, gamma_max: float, T: int = 256) -> np.ndarray:
    """Gaussian beam exp(-gamma^2 / 2 sigma^2) / (2 pi sigma^2), sigma = FWHM / sqrt(8 ln 2),
    tabulated at gamma_t = t gamma_max / (T-1)."""
    sig = fwhm / math.sqrt(8.0 * math.log(2.0))
    g = knot_angles(gamma_max, T)
    return np.exp(-0.5 * (g / sig) ** 2) / (2.0 * math.pi * sig * sig)


def mexican_hat_knots(scale: float, gamma_max: float, T: int = 256) -> np.ndarray:
    """Spherical Mexican-hat wavelet (Martinez-Gonzalez et al. 2002) through the
    stereographic distance y = 2 tan(gamma/2): (1 + y^2/4)^2 (2 - y^2/R^2) e^{-y^2/2R^2},
    normalised to a unit peak.  The last knot is set to zero when the truncation jump
    exceeds 1e-8 of the peak, so the tabulated profile is continuous at the support edge."""
    g = knot_angles(gamma_max, T)
    y = 2.0 * np.tan(0.5 * g)
    r2 = (y / scale) ** 2
    f = (1.0 + 0.25 * y * y) ** 2 * (2.0 - r2) * np.exp(-0.5 * r2)
    f = f / f[0]
    if abs(f[-1]) > 1e-8:
        f[-1] = 0.0
    return f
