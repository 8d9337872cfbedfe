"""Independent brute-force restatements used to pin the oracle (CPU, numpy, FP64).

These share nothing with ``oracle/``: pixel centres come from the input module's own
HEALPix/ECP definitions, angular distances from 3-D unit vectors (squared chord
|n_p - n_q|^2), the profile lookup from ``np.interp`` on the u-knots, and the
trigonometric interpolant from its Dirichlet-kernel form instead of a DFT.
"""
from __future__ import annotations

import math

import numpy as np

from paper_1104_0672_gb300 import inputs


def unit_vectors(theta, phi):
    st = np.sin(theta)
    return np.stack([st * np.cos(phi), st * np.sin(phi), np.cos(theta)], axis=-1)


def profile_u(knots, gamma_max, u):
    """K(u): linear in u = 2(1 - cos gamma) between knot u_t = 4 sin^2(gamma_t/2), 0 beyond."""
    T = len(knots)
    ut = 4.0 * np.sin(0.5 * gamma_max * np.arange(T) / (T - 1)) ** 2
    v = np.interp(u, ut, knots)
    return np.where(u <= ut[-1], v, 0.0)


def ring_table(grid):
    """Ring (theta, phi0, n, weight) from pixel centres: rings are runs of equal theta."""
    th, ph = inputs.centres(grid)
    brk = np.flatnonzero(np.diff(th) != 0) + 1
    starts = np.concatenate([[0], brk])
    ends = np.concatenate([brk, [th.size]])
    thr = th[starts]
    phi0 = ph[starts]
    n = ends - starts
    if grid[0] == "healpix":
        w = np.full(len(starts), 4 * math.pi / th.size)
    else:
        nt, nphi = grid[1], grid[2]
        # Fejer first-rule weights: exact integration of polynomials in cos(theta)
        # of degree < nt on the nodes (k+1/2) pi / nt (Waldvogel 2006, Eq. 2.4).
        k = np.arange(1, nt // 2 + 1)
        w = np.array([(2.0 / nt) * (1 - 2 * np.sum(np.cos(2 * k * t) / (4 * k * k - 1)))
                      for t in thr]) * (2 * math.pi / nphi)
    return thr, phi0, n, starts, w


def direct_true(grid, knots, gamma_max, r, out_pix=None):
    """s_p = sum_q w_q f(gamma_pq) r_q with the squared chord from Cartesian vectors."""
    th, ph = inputs.centres(grid)
    thr, phi0, n, starts, w = ring_table(grid)
    wq = np.repeat(w, n)
    v = unit_vectors(th, ph)
    pix = np.arange(th.size) if out_pix is None else np.asarray(out_pix)
    out = np.empty(len(pix))
    for z, p in enumerate(pix):
        u = np.sum((v - v[p]) ** 2, axis=1)
        out[z] = np.sum(wq * profile_u(knots, gamma_max, u) * r)
    return out


def _dirichlet(N, y, window=None):
    """sum'_{|m|<=N/2} e^{i m y} (halved Nyquist) = 1 + 2 sum_{m<N/2} cos(m y) + cos(N y/2),
    or sum_m W(m) cos(m y) for an explicit symmetric window W over m = 0..N/2."""
    m = np.arange(0, N // 2 + 1)
    if window is None:
        c = np.full(m.size, 2.0)
        c[0] = 1.0
        c[-1] = 1.0
    else:
        c = 2.0 * window
        c[0] = window[0]
    return np.cos(np.multiply.outer(y, m)) @ c


def hybrid_brute(grid, knots, gamma_max, r, variant="enhanced", shift_fix=True,
                 pole_fix=True):
    """The hybrid operator written as a direct sum with the trigonometric interpolant of the
    kernel samples:  s_ip = sum_j w_j sum_q r_jq (1/N) sum_k K_k D(phi_ip - phi_jq - delta_ij
    - 2 pi k / N), D the (windowed) Dirichlet kernel.  Pole rings (HEALPix) use the true
    direct sum when pole_fix is set."""
    thr, phi0, n, starts, w = ring_table(grid)
    R = len(thr)
    N = 4 * grid[1] if grid[0] == "healpix" else grid[2]
    th, ph = inputs.centres(grid)
    out = np.zeros(th.size)
    kk = np.arange(N)
    for i in range(R):
        pi_ = ph[starts[i]:starts[i] + n[i]]
        if grid[0] == "healpix" and pole_fix and i in (0, R - 1):
            out[starts[i]:starts[i] + n[i]] = direct_true(grid, knots, gamma_max, r,
                                                          np.arange(starts[i], starts[i] + n[i]))
            continue
        acc = np.zeros(n[i])
        for j in range(R):
            if abs(thr[i] - thr[j]) > gamma_max:
                continue
            delta = (phi0[i] - phi0[j]) if (shift_fix and n[i] == n[j]) else 0.0
            x = delta + 2 * math.pi * kk / N
            u = 4 * (np.sin(0.5 * (thr[i] - thr[j])) ** 2 * np.cos(0.5 * x) ** 2
                     + np.sin(0.5 * (thr[i] + thr[j])) ** 2 * np.sin(0.5 * x) ** 2)
            K = profile_u(knots, gamma_max, u)
            nz = np.flatnonzero(K)
            if nz.size == 0:
                continue
            pj = ph[starts[j]:starts[j] + n[j]]
            window = None
            if variant == "basic":
                mm = np.arange(0, N // 2 + 1).astype(float)

                def win(nr):
                    h = np.where(2 * mm < nr, 1.0, 0.0)
                    h[2 * mm == nr] = 0.5 if nr < N else 1.0
                    return h
                wi = np.where(2 * mm < n[i], 1.0, 0.0)
                wi[2 * mm == n[i]] = 0.5
                window = wi * win(n[j])
                if n[i] == N and n[j] == N:
                    window = None
            y = (pi_[:, None, None] - pj[None, :, None] - delta
                 - 2 * math.pi * kk[nz][None, None, :] / N)
            D = _dirichlet(N, y.reshape(-1), window).reshape(y.shape)
            acc += w[j] * np.einsum("pqk,q,k->p", D, r[starts[j]:starts[j] + n[j]], K[nz]) / N
        out[starts[i]:starts[i] + n[i]] = acc
    return out


def legendre_coeffs(knots, gamma_max, lmax, nodes=24):
    """b_l = 2 pi int_{cos gamma_max}^1 K(z) P_l(z) dz for the tabulated profile, which is
    linear in z on every knot segment, by per-segment Gauss-Legendre quadrature
    (Sec. 2, Legendre convention)."""
    T = len(knots)
    zt = np.cos(gamma_max * np.arange(T) / (T - 1))
    x, wg = np.polynomial.legendre.leggauss(nodes)
    b = np.zeros(lmax + 1)
    for t in range(T - 1):
        z0, z1 = zt[t + 1], zt[t]
        z = 0.5 * (z1 - z0) * x + 0.5 * (z1 + z0)
        lam = (z1 - z) / (z1 - z0)  # 0 at z1 (knot t), 1 at z0 (knot t+1)
        K = knots[t] * (1 - lam) + knots[t + 1] * lam
        P = np.polynomial.legendre.legvander(z, lmax)
        b += 0.5 * (z1 - z0) * (wg * K) @ P
    return 2 * math.pi * b
