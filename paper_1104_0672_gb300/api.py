"""PyTorch-facing wrapper of libarkcos: grids, kernels, convolve / backward and an autograd
Function.  Torch provides device memory and streams; every step of the convolution runs in
the library's CUDA kernels.  There is no CPU path: the calls raise when CUDA or the library
is unavailable."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from ._native import FLAG_BASIC, FLAG_NO_POLE_FIX, FLAG_NO_SHIFT_FIX, FLAG_3XTF32  # noqa: F401


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need_cuda(t: torch.Tensor, name: str, dtype=torch.float32):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Grid:
    """Isolatitude-ring grid: HEALPix RING (Sec. 4.1) or ECP (Sec. 4.3)."""

    def __init__(self, handle, kind, params):
        self._h = handle
        self.kind = kind
        self.params = params
        L = N.load()
        r, p, n = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        N.check(L.arkcos_grid_info(self._h, ctypes.byref(r), ctypes.byref(p), ctypes.byref(n)))
        self.nrings, self.npix, self.nlon = r.value, p.value, n.value

    @classmethod
    def healpix(cls, nside: int) -> "Grid":
        L = N.load()
        h = ctypes.c_void_p()
        N.check(L.arkcos_create_grid_healpix(int(nside), ctypes.byref(h)))
        return cls(h, "healpix", (int(nside),))

    @classmethod
    def ecp(cls, ntheta: int, nphi: int) -> "Grid":
        L = N.load()
        h = ctypes.c_void_p()
        N.check(L.arkcos_create_grid_ecp(int(ntheta), int(nphi), ctypes.byref(h)))
        return cls(h, "ecp", (int(ntheta), int(nphi)))

    def close(self):
        if self._h:
            N.check(N.load().arkcos_destroy_grid(self._h))
            self._h = None

    def __del__(self):
        try:
            if self._h:
                N.load().arkcos_destroy_grid(self._h)
        except Exception:
            pass


class Kernel:
    """Tabulated radial profile f(gamma_t), gamma_t = t gamma_max / (T-1) (Sec. 4.1)."""

    def __init__(self, grid: Grid, knots, gamma_max: float):
        k = np.ascontiguousarray(np.asarray(knots, dtype=np.float64))
        L = N.load()
        h = ctypes.c_void_p()
        N.check(L.arkcos_set_kernel(grid._h, k.ctypes.data_as(ctypes.c_void_p), len(k),
                                    float(gamma_max), 0, ctypes.byref(h)))
        self._h = h
        self.grid = grid
        self.nknots = len(k)
        self.gamma_max = float(gamma_max)

    @classmethod
    def for_tolerance(cls, grid: Grid, profile, rel_tol: float, cl=None, nknots: int = 256) -> "Kernel":
        """The profile f(gamma) (a vectorised callable, radians) truncated at the smallest support
        whose truncation error (Sec. 4, sigma^2 = sum (2l + 1)/4pi Delta K_l^2 C_l) stays within
        rel_tol of the convolved map's rms, tabulated at nknots knots.  cl defaults to the
        spectrum of unit-variance white noise on the grid's pixels up to l = 3 nside - 1
        (HEALPix) or ntheta - 1 (ECP).  The chosen radius and estimate are kept as
        .gamma_max and .rel_error."""
        from . import support
        if cl is None:
            lmax = 3 * grid.params[0] - 1 if grid.kind == "healpix" else grid.params[0] - 1
            cl = support.white_spectrum(lmax, grid.npix)
        r = support.kernel_for_tolerance(profile, cl, rel_tol, nknots)
        k = cls(grid, r["knots"], r["gamma_max"])
        k.rel_error = r["rel_error"]
        return k

    def update_knots(self, knots, stream=None):
        """New knot values (same count and support): a CUDA float64 tensor (copied on the
        stream) or a host array."""
        L = N.load()
        if isinstance(knots, torch.Tensor) and knots.is_cuda:
            _need_cuda(knots, "knots", torch.float64)
            if knots.numel() != self.nknots:
                raise ValueError("knot count differs")
            N.check(L.arkcos_kernel_update_knots(self._h, ctypes.c_void_p(knots.data_ptr()), 1,
                                                 _stream_handle(stream)))
        else:
            k = np.ascontiguousarray(np.asarray(knots, dtype=np.float64))
            if k.size != self.nknots:
                raise ValueError("knot count differs")
            N.check(L.arkcos_kernel_update_knots(self._h, k.ctypes.data_as(ctypes.c_void_p), 0,
                                                 None))

    def close(self):
        if self._h:
            N.check(N.load().arkcos_destroy_kernel(self._h))
            self._h = None

    def __del__(self):
        try:
            if self._h:
                N.load().arkcos_destroy_kernel(self._h)
        except Exception:
            pass


def _kernel_array(kernels):
    if isinstance(kernels, Kernel):
        kernels = [kernels]
    arr = (ctypes.c_void_p * len(kernels))(*[k._h.value for k in kernels])
    return arr, len(kernels)


def workspace_size(grid: Grid, kernels, nmaps: int, flags: int = 0, backward: bool = False) -> int:
    arr, nk = _kernel_array(kernels)
    out = ctypes.c_size_t()
    N.check(N.load().arkcos_workspace_size(grid._h, arr, nk, int(nmaps), int(flags),
                                           int(bool(backward)), ctypes.byref(out)))
    return out.value


def _workspace(nbytes: int, device, workspace=None):
    if workspace is not None:
        return workspace  # the library checks its size and alignment
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def convolve(grid: Grid, kernels, maps: torch.Tensor, flags: int = 0, out=None, workspace=None,
             stream=None) -> torch.Tensor:
    """Forward convolution of maps [B, npix] (CUDA float32) with one shared kernel or one
    kernel per map."""
    _need_cuda(maps, "maps")
    if maps.dim() == 1:
        return convolve(grid, kernels, maps[None], flags, None if out is None else out[None],
                        workspace, stream)[0]
    B = maps.shape[0]
    if maps.shape[1] != grid.npix:
        raise ValueError(f"maps have {maps.shape[1]} pixels, grid has {grid.npix}")
    if out is None:
        out = torch.empty_like(maps)
    _need_cuda(out, "out")
    arr, nk = _kernel_array(kernels)
    ws = _workspace(workspace_size(grid, kernels, B, flags, False), maps.device, workspace)
    N.check(N.load().arkcos_convolve(grid._h, arr, nk, ctypes.c_void_p(maps.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), B,
                                     ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                     _stream_handle(stream), int(flags)))
    return out


def multi_workspace_size(grid: Grid, kernels, nmaps: int, weighted: bool = False, flags: int = 0) -> int:
    arr, nk = _kernel_array(kernels)
    out = ctypes.c_size_t()
    N.check(N.load().arkcos_multi_workspace_size(grid._h, arr, nk, int(nmaps), int(bool(weighted)), int(flags),
                                                 ctypes.byref(out)))
    return out.value


def convolve_multi(grid: Grid, kernels, maps: torch.Tensor, weights=None, flags: int = 0, out=None,
                   workspace=None, stream=None) -> torch.Tensor:
    """Several kernels on the same maps [B, npix] (CUDA float32), each map ring-analysed once:
    returns [B, K, npix] (one output per kernel) or, with `weights` (K floats), the weighted
    sums [B, npix]."""
    _need_cuda(maps, "maps")
    if maps.dim() == 1:
        r = convolve_multi(grid, kernels, maps[None], weights, flags, None if out is None else out[None],
                           workspace, stream)
        return r[0]
    B = maps.shape[0]
    if maps.shape[1] != grid.npix:
        raise ValueError(f"maps have {maps.shape[1]} pixels, grid has {grid.npix}")
    arr, nk = _kernel_array(kernels)
    w = None
    if weights is not None:
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
        if w.shape != (nk,):
            raise ValueError("weights must hold one value per kernel")
    shape = (B, grid.npix) if w is not None else (B, nk, grid.npix)
    if out is None:
        out = torch.empty(shape, dtype=torch.float32, device=maps.device)
    _need_cuda(out, "out")
    if tuple(out.shape) != shape:
        raise ValueError(f"out must have shape {shape}")
    ws = _workspace(multi_workspace_size(grid, kernels, B, w is not None, flags), maps.device, workspace)
    N.check(N.load().arkcos_convolve_multi(grid._h, arr, nk,
                                           w.ctypes.data_as(ctypes.c_void_p) if w is not None else None,
                                           ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(out.data_ptr()), B,
                                           ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream),
                                           int(flags)))
    return out


def autotune(grid: Grid, kernels, maps: torch.Tensor, flags: int = 0, out=None, workspace=None,
             stream=None) -> dict:
    """Choose the launch shape of convolve(grid, kernels, maps, flags) by timing the candidates
    on these buffers (out is overwritten); later convolve calls with the same grid, kernels,
    number of maps and flags use it.  Returns the chosen shape and its time."""
    _need_cuda(maps, "maps")
    B = maps.shape[0]
    if out is None:
        out = torch.empty_like(maps)
    arr, nk = _kernel_array(kernels)
    ws = _workspace(workspace_size(grid, kernels, B, flags, False), maps.device, workspace)
    res = (ctypes.c_int64 * 5)()
    N.check(N.load().arkcos_autotune(grid._h, arr, nk, ctypes.c_void_p(maps.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), B, ctypes.c_void_p(ws.data_ptr()),
                                     ws.numel(), _stream_handle(stream), int(flags), res))
    return {"fft_split": int(res[0]), "maps_per_contraction_cta": int(res[1]), "candidates": int(res[2]),
            "best_ms": res[3] / 1000.0, "tc_form": int(res[4])}


def set_launch_shape(grid: Grid, kernels, nmaps: int, flags: int = 0, fft_split: int = 1,
                     maps_per_contraction_cta: int = 0, tc_form: int = 0) -> None:
    """Install the launch shape later convolve(grid, kernels, maps of nmaps, flags) calls use
    (in place of an autotuned or default one); every shape gives bitwise the same result."""
    arr, nk = _kernel_array(kernels)
    shape = (ctypes.c_int64 * 3)(int(fft_split), int(maps_per_contraction_cta), int(tc_form))
    N.check(N.load().arkcos_set_launch_shape(grid._h, arr, nk, int(nmaps), int(flags), shape))


def host_workspace_size(grid: Grid, kernels, nmaps: int, maps_per_chunk: int = 4, flags: int = 0) -> int:
    arr, nk = _kernel_array(kernels)
    out = ctypes.c_size_t()
    N.check(N.load().arkcos_host_workspace_size(grid._h, arr, nk, int(nmaps), int(maps_per_chunk),
                                                int(flags), ctypes.byref(out)))
    return out.value


def convolve_host(grid: Grid, kernels, maps: torch.Tensor, flags: int = 0, out=None, maps_per_chunk: int = 4,
                  workspace=None, device=None, stream=None) -> torch.Tensor:
    """Forward convolution of HOST maps [B, npix] (CPU float32, pinned for overlap) into a host
    output, pipelined in chunks of maps_per_chunk maps: uploads, convolutions and downloads of
    consecutive chunks overlap.  Returns `out`; it is complete once `stream` (the current CUDA
    stream by default) has reached this point, e.g. after torch.cuda.synchronize()."""
    if maps.device.type != "cpu" or maps.dtype != torch.float32 or not maps.is_contiguous():
        raise ValueError("maps must be a contiguous CPU float32 tensor")
    if maps.dim() == 1:
        return convolve_host(grid, kernels, maps[None], flags, None if out is None else out[None],
                             maps_per_chunk, workspace, device, stream)[0]
    B = maps.shape[0]
    if maps.shape[1] != grid.npix:
        raise ValueError(f"maps have {maps.shape[1]} pixels, grid has {grid.npix}")
    if out is None:
        out = torch.empty_like(maps, pin_memory=maps.is_pinned())
    if out.device.type != "cpu" or out.dtype != torch.float32 or not out.is_contiguous() or out.shape != maps.shape:
        raise ValueError("out must be a contiguous CPU float32 tensor shaped like maps")
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    arr, nk = _kernel_array(kernels)
    ws = _workspace(host_workspace_size(grid, kernels, B, maps_per_chunk, flags), dev, workspace)
    N.check(N.load().arkcos_convolve_host(grid._h, arr, nk, ctypes.c_void_p(maps.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), B, int(maps_per_chunk),
                                          ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                          _stream_handle(stream), int(flags)))
    return out


def convolve_backward(grid: Grid, kernels, maps, grad_out: torch.Tensor, need_map_grad=True,
                      need_knot_grad=True, flags: int = 0, workspace=None, stream=None):
    """Returns (grad_maps or None, grad_knots [nkernels, T] float64 or None)."""
    _need_cuda(grad_out, "grad_out")
    if grad_out.dim() == 1:
        gm, gk = convolve_backward(grid, kernels, None if maps is None else maps[None],
                                   grad_out[None], need_map_grad, need_knot_grad, flags,
                                   workspace, stream)
        return (None if gm is None else gm[0]), gk
    B = grad_out.shape[0]
    arr, nk = _kernel_array(kernels)
    kl = [kernels] if isinstance(kernels, Kernel) else list(kernels)
    gin = torch.empty_like(grad_out) if need_map_grad else None
    gk = None
    if need_knot_grad:
        _need_cuda(maps, "maps")
        T = kl[0].nknots
        if any(k.nknots != T for k in kl):
            raise ValueError("per-map kernels must share the knot count")
        gk = torch.empty((nk, T), dtype=torch.float64, device=grad_out.device)
    ws = _workspace(workspace_size(grid, kernels, B, flags, True), grad_out.device, workspace)
    N.check(N.load().arkcos_convolve_backward(
        grid._h, arr, nk,
        ctypes.c_void_p(maps.data_ptr()) if maps is not None else None,
        ctypes.c_void_p(grad_out.data_ptr()),
        ctypes.c_void_p(gin.data_ptr()) if gin is not None else None,
        ctypes.c_void_p(gk.data_ptr()) if gk is not None else None,
        B, ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream), int(flags)))
    return gin, gk


def ring_analysis(grid: Grid, maps: torch.Tensor, stream=None) -> torch.Tensor:
    """Half spectra of every ring, concatenated: complex64 [B, sum_j (n_j/2 + 1)]."""
    _need_cuda(maps, "maps")
    B = maps.shape[0]
    nspec = (grid.npix + 2 * grid.nrings) // 2
    out = torch.empty((B, nspec), dtype=torch.complex64, device=maps.device)
    N.check(N.load().arkcos_ring_analysis(grid._h, ctypes.c_void_p(maps.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), B,
                                          _stream_handle(stream)))
    return out


def ring_synthesis(grid: Grid, coeffs: torch.Tensor, flags: int = 0, stream=None) -> torch.Tensor:
    """Maps from kernel-grid coefficients complex64 [B, nrings, N/2 + 1]."""
    if not coeffs.is_cuda or coeffs.dtype != torch.complex64 or not coeffs.is_contiguous():
        raise TypeError("coeffs must be a contiguous CUDA complex64 tensor")
    B = coeffs.shape[0]
    out = torch.empty((B, grid.npix), dtype=torch.float32, device=coeffs.device)
    N.check(N.load().arkcos_ring_synthesis(grid._h, ctypes.c_void_p(coeffs.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), B, int(flags),
                                           _stream_handle(stream)))
    return out


def convolve_batch(jobs, workspace=None, stream=None):
    """Forward convolutions of several grids in one stream-ordered call.  jobs: list of
    (grid, kernels, maps_in [B, npix] CUDA float32, flags); returns the output tensors.  The
    call performs no host synchronisation, so a torch.cuda.CUDAGraph capture of it replays
    the whole batch with one graph launch (allocate `workspace` outside the capture)."""
    recs, outs, keep = [], [], []
    for grid, kernels, maps, flags in jobs:
        _need_cuda(maps, "maps")
        arr, nk = _kernel_array(kernels)
        out = torch.empty_like(maps)
        keep.append(arr)
        recs.append(N.Job(grid._h.value, ctypes.cast(arr, ctypes.c_void_p).value, nk, maps.data_ptr(),
                          out.data_ptr(), maps.shape[0], int(flags)))
        outs.append(out)
    jarr = (N.Job * len(recs))(*recs)
    L = N.load()
    need = ctypes.c_size_t()
    N.check(L.arkcos_batch_workspace_size(jarr, len(recs), ctypes.byref(need)))
    ws = _workspace(need.value, jobs[0][2].device, workspace)
    N.check(L.arkcos_convolve_batch(jarr, len(recs), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                    _stream_handle(stream)))
    return outs


def batch_workspace_size(jobs) -> int:
    recs, keep = [], []
    for grid, kernels, maps, flags in jobs:
        arr, nk = _kernel_array(kernels)
        keep.append(arr)
        recs.append(N.Job(grid._h.value, ctypes.cast(arr, ctypes.c_void_p).value, nk, 0, 0,
                          int(maps.shape[0]) if hasattr(maps, "shape") else int(maps), int(flags)))
    jarr = (N.Job * len(recs))(*recs)
    need = ctypes.c_size_t()
    N.check(N.load().arkcos_batch_workspace_size(jarr, len(recs), ctypes.byref(need)))
    return need.value


def kernel_info(kernel: Kernel):
    """(representative ring pairs, in-support kernel samples, largest band height)."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    N.check(N.load().arkcos_kernel_info(kernel._h, ctypes.byref(a), ctypes.byref(b),
                                        ctypes.byref(c)))
    return a.value, b.value, c.value


def stage_timing(enable: bool = True):
    """Turn per-stage CUDA-event timing on (clearing old records) or off."""
    N.check(N.load().arkcos_stage_timing(int(bool(enable))))


def stage_report() -> dict:
    """{stage: (milliseconds, executions, kernel launches)} since stage_timing(True)."""
    L = N.load()
    out = {}
    i = 0
    while True:
        name, ms = ctypes.c_char_p(), ctypes.c_double()
        ex, nl = ctypes.c_int64(), ctypes.c_int64()
        st = L.arkcos_stage_report(i, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(ex),
                                   ctypes.byref(nl))
        if st == N.EINVAL:
            break
        N.check(st)
        if ex.value:
            out[name.value.decode()] = (ms.value, ex.value, nl.value)
        i += 1
    return out


def measure_peak(unit: str, stream=None) -> dict:
    """Arithmetic peak of the current device from a short isolated kernel (a roofline
    denominator): unit "fp32" (fmaf), "fp32x2" (packed two-lane FMA), "fp64" or "tf32_mma"
    (tcgen05 kind::tf32, M 128 N 256 K 8).  Returns {"tflops", "ms"}."""
    units = {"fp32": 0, "fp32x2": 1, "fp64": 2, "tf32_mma": 3}
    t, ms = ctypes.c_double(), ctypes.c_double()
    N.check(N.load().arkcos_measure_peak(units[unit], ctypes.byref(t), ctypes.byref(ms), _stream_handle(stream)))
    return {"tflops": t.value, "ms": ms.value}


def sync_status(stream=None):
    N.check(N.load().arkcos_sync_status(_stream_handle(stream)))


class ConvolveFunction(torch.autograd.Function):
    """maps [B, npix] float32, knots [nkernels, T] float64 (CUDA) -> convolved maps.
    The knot tensor is copied into the kernel handles before the forward pass, so gradients
    with respect to it (dJ/df_t, Sec. 4.1 table) flow through the hand-written adjoint.  With
    a process group (`dist` = torch.distributed, `group` = its group or None for the default)
    the knot gradient is summed over the ranks after the backward pass: every rank holds the
    same shared beam and convolves its own maps."""

    @staticmethod
    def forward(ctx, maps, knots, grid, kernels, flags, dist=None, group=None):
        kl = [kernels] if isinstance(kernels, Kernel) else list(kernels)
        for k, row in zip(kl, knots.reshape(len(kl), -1)):
            k.update_knots(row.contiguous())
        ctx.grid, ctx.kernels, ctx.flags, ctx.dist, ctx.group = grid, kernels, flags, dist, group
        ctx.save_for_backward(maps)
        return convolve(grid, kernels, maps.contiguous(), flags)

    @staticmethod
    def backward(ctx, g):
        (maps,) = ctx.saved_tensors
        need_map, need_knots = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gm, gk = convolve_backward(ctx.grid, ctx.kernels, maps.contiguous(), g.contiguous(),
                                   need_map, need_knots, ctx.flags)
        if gk is not None and ctx.dist is not None:
            from . import replicas
            replicas.allreduce_knot_grad(gk, ctx.dist, ctx.group)
        return gm, gk, None, None, None, None, None


def convolve_autograd(grid: Grid, kernels, maps: torch.Tensor, knots: torch.Tensor, flags: int = 0,
                      dist=None, group=None):
    """Differentiable convolution of maps with the kernels whose knot values are `knots`.
    Data-parallel beam fitting: pass dist=torch.distributed (and a group) so that the knot
    gradient of the beam every rank shares is summed over the ranks."""
    return ConvolveFunction.apply(maps, knots, grid, kernels, flags, dist, group)
