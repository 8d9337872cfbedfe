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


def healpix_rings(nside: int):
    """Per RING-order ring: colatitude, pixel count and first-pixel longitude (HEALPix RING
    definition, Gorski et al. 2005)."""
    ns = int(nside)
    th, n, p0 = [], [], []
    for r in range(1, 4 * ns):
        i = min(r, 4 * ns - r)
        if i < ns:
            t = 2.0 * math.asin(i / (math.sqrt(6.0) * ns))
            th.append(t if r < ns else math.pi - t)
            n.append(4 * i)
            p0.append(math.pi / (4 * i))
        else:
            th.append(math.acos(4.0 / 3.0 - 2.0 * r / (3.0 * ns)))
            n.append(4 * ns)
            p0.append(math.pi / (4 * ns) if (r - ns) % 2 == 0 else 0.0)
    return np.array(th), np.array(n, dtype=np.int64), np.array(p0)


def random_alm(lmax: int, cl, config: int = 0, salt: int = 0) -> np.ndarray:
    """Seeded harmonic coefficients of a Gaussian random field with angular power spectrum
    cl[l] (l = 0..lmax): alm[m, l] (zero for l < m), a_l0 ~ N(0, C_l) real, a_lm ~ complex
    normal with E|a_lm|^2 = C_l for m > 0."""
    g = rng(config, salt)
    re = g.standard_normal((lmax + 1, lmax + 1))
    im = g.standard_normal((lmax + 1, lmax + 1))
    c = np.sqrt(np.asarray(cl, dtype=np.float64)[: lmax + 1])
    a = (re + 1j * im) * (c / math.sqrt(2.0))[None, :]
    a[0] = re[0] * c
    a[np.tril_indices(lmax + 1, -1)] = 0.0  # entries [m, l] with l < m
    return a


def synthesize_healpix(nside: int, alm: np.ndarray, device="cpu") -> np.ndarray:
    """The real field T = sum_{l, |m| <= l} a_lm Y_lm (a_{l,-m} = (-1)^m conj a_lm) at the
    HEALPix RING pixel centres, FP64, from alm[m, l] (m, l = 0..lmax).

    Inverse spherical-harmonic transform in two steps: per ring and m, F_m(theta) = sum_l a_lm
    lambda_l^m(cos theta) with the orthonormal Legendre recurrence of _legendre_norm (scaled
    values with a per-point log scale), run in torch over all m and all northern rings at once
    on `device` and split into the parts of even and odd l + m, which give the mirrored
    southern ring (lambda_l^m(-x) = (-1)^(l+m) lambda_l^m(x)); then per ring
    T_q = Re sum_m c_m F_m exp(i m (phi0 + 2 pi q / n)) (c_0 = 1, c_m = 2) by folding m modulo
    n and one inverse DFT."""
    import torch

    lmax = alm.shape[1] - 1
    ns = int(nside)
    dev = torch.device(device)
    f64 = torch.float64
    th, nr, p0 = healpix_rings(ns)
    J = 2 * ns  # northern rings and the equator (ring index 0..2 ns - 1)
    x = torch.tensor(np.cos(th[:J]), dtype=f64, device=dev)
    s = torch.sqrt(torch.clamp(1.0 - x * x, min=0.0))
    logs = torch.log(s)
    M = lmax + 1
    A = torch.tensor(alm.T.copy(), dtype=torch.complex128, device=dev)  # [l][m]
    P = torch.zeros((M, J), dtype=f64, device=dev)
    Pp = torch.zeros_like(P)
    S = torch.zeros_like(P)
    Er, Ei, Or, Oi = (torch.zeros_like(P) for _ in range(4))
    ms = torch.arange(M, dtype=f64, device=dev)
    # log of lambda_m^m's constant (-1)^m sqrt(1/4pi) prod_k sqrt((2k+1)/2k), sign kept apart
    lk = torch.log((2.0 * ms[1:] + 1.0) / (2.0 * ms[1:])) * 0.5
    logc = 0.5 * math.log(1.0 / (4.0 * math.pi)) + torch.cat([torch.zeros(1, dtype=f64, device=dev),
                                                              torch.cumsum(lk, 0)])
    sign = torch.where(torch.arange(M, device=dev) % 2 == 1, -1.0, 1.0).to(f64)
    big, logbig = 1e150, math.log(1e150)
    for l in range(M):
        if l > 0:
            m = ms[:l]
            a = torch.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = torch.sqrt(torch.clamp(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0), min=0.0))
            pn = a[:, None] * (x[None, :] * P[:l] - b[:, None] * Pp[:l])
            Pp[:l] = P[:l]
            P[:l] = pn
            grow = pn.abs() > big
            if bool(grow.any()):
                P[:l] = torch.where(grow, P[:l] / big, P[:l])
                Pp[:l] = torch.where(grow, Pp[:l] / big, Pp[:l])
                S[:l] = S[:l] + grow.to(f64) * logbig
        P[l] = 1.0
        Pp[l] = 0.0
        S[l] = logc[l] + l * logs
        val = sign[: l + 1, None] * P[: l + 1] * torch.exp(S[: l + 1])
        c = A[l, : l + 1]
        even = ((torch.arange(l + 1, device=dev) + l) % 2 == 0).to(f64)[:, None]
        tr, ti = c.real[:, None] * val, c.imag[:, None] * val
        Er[: l + 1] += even * tr
        Ei[: l + 1] += even * ti
        Or[: l + 1] += (1.0 - even) * tr
        Oi[: l + 1] += (1.0 - even) * ti
    Fn = torch.complex(Er + Or, Ei + Oi)   # [m][ring], northern rings
    Fs = torch.complex(Er - Or, Ei - Oi)   # their southern mirrors
    cm = torch.full((M,), 2.0, dtype=f64, device=dev)
    cm[0] = 1.0
    R = 4 * ns - 1
    offs = np.concatenate([[0], np.cumsum(nr)])
    out = np.empty(int(offs[-1]))
    mi = torch.arange(M, device=dev)
    for r in range(R):
        j = r if r < J else R - 1 - r
        F = (Fn if r < J else Fs)[:, j]
        n = int(nr[r])
        ph = torch.exp(1j * mi.to(f64) * float(p0[r]))
        G = torch.zeros(n, dtype=torch.complex128, device=dev)
        G.index_add_(0, mi % n, cm * F * ph)
        out[offs[r]:offs[r + 1]] = (torch.fft.ifft(G) * n).real.cpu().numpy()
    return out


def cl_field_healpix(nside: int, lmax: int, cl, config: int = 0, salt: int = 0, device="cpu") -> np.ndarray:
    """Seeded Gaussian random field with power spectrum cl[l] (l <= lmax) at the HEALPix
    RING pixel centres (FP64): random_alm, then synthesize_healpix."""
    return synthesize_healpix(nside, random_alm(lmax, cl, config, salt), device)


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
