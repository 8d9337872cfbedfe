"""Support radius of a truncated radial kernel from the truncation-error estimate of Sec. 4.

A radial kernel f(gamma) has the Legendre coefficients of Sec. 2,
    K_l = 2 pi int_{-1}^{1} f(acos z) P_l(z) dz = 2 pi int_0^pi f(gamma) P_l(cos gamma) sin gamma dgamma.
Truncating it at gamma_max changes them by Delta K_l, the same integral over (gamma_max, pi], and
convolving an isotropic map of power spectrum C_l then errs by (Sec. 4)
    sigma^2 = sum_{l <= lmax} (2l + 1) / (4 pi) Delta K_l^2 C_l,
against the variance sum_l (2l + 1) / (4 pi) K_l^2 C_l of the convolved map itself.
choose_support() returns the smallest gamma_max whose relative error sigma / rms stays within a
tolerance; kernel_for_tolerance() also tabulates the profile at the knots of that support,
the arguments of Kernel(grid, knots, gamma_max) (api.Kernel.for_tolerance does both).

Host-side numerics on numpy only; nothing on the convolution path calls this module.
"""
from __future__ import annotations

import math

import numpy as np


_GL_X, _GL_W = np.polynomial.legendre.leggauss(16)


def legendre_coefficients(profile, lmax: int, gamma_lo: float = 0.0, gamma_hi: float = math.pi) -> np.ndarray:
    """K_l = 2 pi int_{gamma_lo}^{gamma_hi} f(gamma) P_l(cos gamma) sin gamma dgamma for
    l = 0..lmax (Sec. 2 convention), by a composite 16-point Gauss-Legendre rule in gamma with
    panels narrower than a quarter period of P_lmax; P_l by the three-term recurrence.
    profile: a vectorised callable f(gamma) (radians)."""
    if lmax < 0:
        raise ValueError("lmax must be >= 0")
    if not 0.0 <= gamma_lo <= gamma_hi <= math.pi:
        raise ValueError("need 0 <= gamma_lo <= gamma_hi <= pi")
    out = np.zeros(lmax + 1)
    if gamma_hi == gamma_lo:
        return out
    panels = max(1, math.ceil(2.0 * (gamma_hi - gamma_lo) * (lmax + 1) / math.pi))
    edges = np.linspace(gamma_lo, gamma_hi, panels + 1)
    half = 0.5 * (edges[1:] - edges[:-1])
    g = (half[:, None] * _GL_X[None, :] + (edges[:-1] + half)[:, None]).ravel()
    w = (half[:, None] * _GL_W[None, :]).ravel()
    wz = 2.0 * math.pi * w * np.sin(g) * np.asarray(profile(g), dtype=np.float64)
    z = np.cos(g)
    p_prev, p = np.ones_like(z), z
    out[0] = wz.sum()
    if lmax >= 1:
        out[1] = wz @ p
    for l in range(2, lmax + 1):
        p_prev, p = p, ((2 * l - 1) * z * p - (l - 1) * p_prev) / l
        out[l] = wz @ p
    return out


def support_end(profile, samples: int = 200001) -> float:
    """The angle past which the profile vanishes on a fine grid of [0, pi] (pi if it never
    does): the upper limit of every integral below."""
    g = np.linspace(0.0, math.pi, samples)
    nz = np.nonzero(np.asarray(profile(g)) != 0.0)[0]
    if nz.size == 0:
        return 0.0
    return float(min(math.pi, g[nz[-1]] + math.pi / (samples - 1)))


def _weights(cl) -> np.ndarray:
    cl = np.asarray(cl, dtype=np.float64)
    ell = np.arange(cl.size)
    return (2 * ell + 1) / (4 * math.pi) * cl


def truncation_error(profile, gamma_max: float, cl) -> float:
    """sigma^2 of Sec. 4: the mean quadratic error of convolving a map of power spectrum cl
    (l = 0..len(cl)-1) with the kernel truncated at gamma_max."""
    end = support_end(profile)
    if gamma_max >= end:
        return 0.0
    dk = legendre_coefficients(profile, len(cl) - 1, gamma_max, end)
    return float(_weights(cl) @ (dk * dk))


def output_variance(profile, cl) -> float:
    """Variance of the map convolved with the untruncated kernel."""
    k = legendre_coefficients(profile, len(cl) - 1, 0.0, support_end(profile))
    return float(_weights(cl) @ (k * k))


def choose_support(profile, cl, rel_tol: float, gamma_min: float = 1e-4, iters: int = 40) -> float:
    """Smallest gamma_max in [gamma_min, support end] with sqrt(sigma^2 / variance) <= rel_tol,
    by bisection (the relative error is taken to fall with gamma_max, as it does for
    kernels whose tail decays monotonically)."""
    end = support_end(profile)
    var = output_variance(profile, cl)
    if var <= 0.0:
        raise ValueError("the kernel convolves this spectrum to zero")
    tol2 = rel_tol * rel_tol * var
    if truncation_error(profile, gamma_min, cl) <= tol2:
        return gamma_min
    lo, hi = gamma_min, end
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if truncation_error(profile, mid, cl) <= tol2:
            hi = mid
        else:
            lo = mid
    return hi


def white_spectrum(lmax: int, npix: int) -> np.ndarray:
    """C_l of a map of unit-variance uncorrelated pixels on an equal-area grid of npix pixels,
    up to lmax: 4 pi / npix for every l (the default spectrum of kernel_for_tolerance)."""
    return np.full(lmax + 1, 4.0 * math.pi / npix)


def kernel_for_tolerance(profile, cl, rel_tol: float, nknots: int = 256) -> dict:
    """The support radius choose_support() gives for (profile, cl, rel_tol) and the profile
    tabulated there: knots f(gamma_t), gamma_t = t gamma_max / (nknots - 1), as
    Kernel(grid, knots, gamma_max) takes them.  Returns {"knots", "gamma_max", "rel_error"},
    rel_error = sqrt(sigma^2 / variance) at that radius (Sec. 4)."""
    if nknots < 2:
        raise ValueError("nknots must be >= 2")
    gm = choose_support(profile, cl, rel_tol)
    g = gm * np.arange(nknots) / (nknots - 1)
    knots = np.asarray(profile(g), dtype=np.float64)
    err = math.sqrt(truncation_error(profile, gm, cl) / output_variance(profile, cl))
    return {"knots": knots, "gamma_max": gm, "rel_error": err}
