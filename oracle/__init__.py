"""FP64 CPU oracle for the ARKCoS hybrid ring convolution (Elsner & Wandelt 2011).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it; the product path never imports it.  It shares no code with
the CUDA library (its own geometry, kernel lookup and naive DFTs live in
``arkcos_oracle.c``).  Each function cites the paper passage it follows.

Parity status per function:
  * convolve (ENHANCED, both grids), direct, adjoint, knot_grad: pinned by the CPU
    tests (brute-force direct sums, Funk-Hecke closed form, invariants, dot-product and
    finite-difference identities).
  * convolve with variant="basic" on HEALPix polar caps: parity unpinned (no closed
    form exists for the truncation operator; only its brute-force restatement checks it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "arkcos_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

HEALPIX = 0
ECP = 1
_OPT_BASIC = 1
_OPT_NO_SHIFT = 2
_OPT_NO_POLE = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            L, I, D, U = ctypes.c_long, ctypes.c_int, ctypes.c_double, ctypes.c_uint
            P = ctypes.c_void_p
            lib.oracle_nrings.argtypes = [I, L, L]
            lib.oracle_nrings.restype = L
            lib.oracle_geometry.argtypes = [I, L, L, P, P, P, P, P]
            lib.oracle_geometry.restype = I
            lib.oracle_convolve.argtypes = [I, L, L, P, L, D, U, P, P, P, L, I]
            lib.oracle_convolve.restype = I
            lib.oracle_direct.argtypes = [I, L, L, P, L, D, P, P, P, L, I]
            lib.oracle_direct.restype = I
            lib.oracle_adjoint.argtypes = [I, L, L, P, L, D, U, P, P, P, L, I]
            lib.oracle_adjoint.restype = I
            lib.oracle_knot_grad.argtypes = [I, L, L, P, L, D, U, P, P, P, I]
            lib.oracle_knot_grad.restype = I
            _lib = lib
    return _lib


def _grid_args(grid):
    kind = grid[0]
    if kind == "healpix":
        return HEALPIX, int(grid[1]), 0
    if kind == "ecp":
        return ECP, int(grid[1]), int(grid[2])
    raise ValueError(f"unknown grid {grid!r}")


def _opts(variant="enhanced", shift_fix=True, pole_fix=True):
    o = 0
    if variant == "basic":
        o |= _OPT_BASIC
    elif variant != "enhanced":
        raise ValueError(variant)
    if not shift_fix:
        o |= _OPT_NO_SHIFT
    if not pole_fix:
        o |= _OPT_NO_POLE
    return o


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def geometry(grid):
    """Ring table (theta, phi0, weight, npix_ring, offset) -- HEALPix per Gorski et al.
    2005 (the ring structure of Sec. 4.1), ECP with Fejer first-rule weights."""
    lib = _load()
    kind, a, b = _grid_args(grid)
    R = lib.oracle_nrings(kind, a, b)
    if R < 0:
        raise ValueError(f"bad grid {grid!r}")
    th, ph, w = (np.zeros(R) for _ in range(3))
    n, off = np.zeros(R, np.int64), np.zeros(R, np.int64)
    assert lib.oracle_geometry(kind, a, b, _ptr(th), _ptr(ph), _ptr(w), _ptr(n), _ptr(off)) == 0
    return th, ph, w, n, off


def npix(grid):
    th, ph, w, n, off = geometry(grid)
    return int(n.sum())


def _rings_arg(rings):
    if rings is None:
        return None, 0, None
    r = np.ascontiguousarray(np.asarray(rings, dtype=np.int64))
    return _ptr(r), len(r), r


def convolve(grid, knots, gamma_max, map_in, rings=None, variant="enhanced",
             shift_fix=True, pole_fix=True, nthreads=0):
    """Hybrid forward convolution (Sec. 4.1 steps, Sec. 4.3 enhancements, Sec. 4.2 pole fix)
    of one FP64 map.  With ``rings`` given only those output rings are computed (other
    entries of the result are NaN)."""
    lib = _load()
    kind, a, b = _grid_args(grid)
    x = np.ascontiguousarray(map_in, dtype=np.float64)
    k = np.ascontiguousarray(knots, dtype=np.float64)
    out = np.full_like(x, np.nan)
    rp, nr, keep = _rings_arg(rings)
    rc = lib.oracle_convolve(kind, a, b, _ptr(k), len(k), float(gamma_max),
                             _opts(variant, shift_fix, pole_fix), _ptr(x), _ptr(out), rp, nr,
                             int(nthreads))
    if rc:
        raise ValueError("oracle_convolve rejected its arguments")
    return out


def direct(grid, knots, gamma_max, map_in, rings=None, nthreads=0):
    """True-profile weighted direct sum s_p = sum_q w_q f(gamma_pq) r_q (Sec. 3.1 Eq. direct)."""
    lib = _load()
    kind, a, b = _grid_args(grid)
    x = np.ascontiguousarray(map_in, dtype=np.float64)
    k = np.ascontiguousarray(knots, dtype=np.float64)
    out = np.full_like(x, np.nan)
    rp, nr, keep = _rings_arg(rings)
    rc = lib.oracle_direct(kind, a, b, _ptr(k), len(k), float(gamma_max), _ptr(x), _ptr(out),
                           rp, nr, int(nthreads))
    if rc:
        raise ValueError("oracle_direct rejected its arguments")
    return out


def adjoint(grid, knots, gamma_max, gmap, rings=None, variant="enhanced", shift_fix=True,
            pole_fix=True, nthreads=0):
    """Transpose of ``convolve`` applied to ``gmap`` (gradient with respect to the map)."""
    lib = _load()
    kind, a, b = _grid_args(grid)
    g = np.ascontiguousarray(gmap, dtype=np.float64)
    k = np.ascontiguousarray(knots, dtype=np.float64)
    out = np.full_like(g, np.nan)
    rp, nr, keep = _rings_arg(rings)
    rc = lib.oracle_adjoint(kind, a, b, _ptr(k), len(k), float(gamma_max),
                            _opts(variant, shift_fix, pole_fix), _ptr(g), _ptr(out), rp, nr,
                            int(nthreads))
    if rc:
        raise ValueError("oracle_adjoint rejected its arguments")
    return out


def knot_grad(grid, knots, gamma_max, map_in, gmap, variant="enhanced", shift_fix=True,
              pole_fix=True, nthreads=0):
    """d<g, L(f) r>/d f_t for every profile knot t (all ring pairs)."""
    lib = _load()
    kind, a, b = _grid_args(grid)
    x = np.ascontiguousarray(map_in, dtype=np.float64)
    g = np.ascontiguousarray(gmap, dtype=np.float64)
    k = np.ascontiguousarray(knots, dtype=np.float64)
    out = np.zeros(len(k))
    rc = lib.oracle_knot_grad(kind, a, b, _ptr(k), len(k), float(gamma_max),
                              _opts(variant, shift_fix, pole_fix), _ptr(x), _ptr(g), _ptr(out),
                              int(nthreads))
    if rc:
        raise ValueError("oracle_knot_grad rejected its arguments")
    return out
