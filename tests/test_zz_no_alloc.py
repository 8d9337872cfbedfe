"""The allocation-free forward convolution, arkcos_convolve_static, against arkcos_convolve.

Some callers cannot give the library a device workspace while they run -- their device memory
belongs to another framework's pool, or they may not call cudaMalloc (which can synchronise the
device) inside their loop.  arkcos_convolve_static serves them from a fixed scratch array built
into the library.  This file is named to be collected last, so that a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1104_0672_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5  # fractional RMS, as in the other GPU parity tests


def _frac(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _static(lib, grid, kernels, x, out, stream, flags):
    import ctypes
    karr = (ctypes.c_void_p * len(kernels))(*[k._h.value for k in kernels])
    return lib.arkcos_convolve_static(grid._h, karr, len(kernels), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), x.shape[0], stream, flags)


@pytest.mark.parametrize("beams", ["shared", "permap"])
@pytest.mark.parametrize("form", ["fp32", "tf32"])
def test_static_scratch_matches_workspace_entry_point(beams, form):
    import torch

    import paper_1104_0672_gb300 as ark
    from paper_1104_0672_gb300 import _native

    assert torch.cuda.is_available()
    lib = _native.load()
    dev = torch.device("cuda:0")
    flags = ark.FLAG_3XTF32 if form == "tf32" else 0
    grid = ark.Grid.healpix(128)
    gmax = 2.5 * inputs.DEG
    if beams == "shared":
        kernels = [ark.Kernel(grid, inputs.gaussian_knots(50 * inputs.ARCMIN, gmax, 256), gmax)]
    else:
        kernels = [ark.Kernel(grid, inputs.gaussian_knots(f * inputs.ARCMIN, gmax, 256), gmax) for f in (40, 55)]
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    # a call of another shape first (another grid, map count and beam), so that the compared
    # calls run on leftovers laid out differently from what they write themselves
    other = ark.Grid.healpix(64)
    ko = ark.Kernel(other, inputs.gaussian_knots(2 * inputs.DEG, 6 * inputs.DEG, 128), 6 * inputs.DEG)
    xo = torch.from_numpy(inputs.white_noise(other.npix, 3, config=14, salt=9)).to(dev)
    oo = torch.empty_like(xo)
    assert _static(lib, other, [ko], xo, oo, stream, ark.FLAG_3XTF32 if form == "fp32" else 0) == _native.OK

    # two calls in a row, each on fresh input, each against the workspace entry point
    kk = kernels[0] if beams == "shared" else kernels
    for call in range(2):
        x = torch.from_numpy(inputs.white_noise(grid.npix, 2, config=14, salt=call)).to(dev)
        ref = ark.convolve(grid, kk, x, flags).cpu().numpy()
        out = torch.full_like(x, float("nan"))
        st = _static(lib, grid, kernels, x, out, stream, flags)
        assert st == _native.OK, lib.arkcos_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        for b in range(2):
            assert _frac(got[b], ref[b]) < TOL


def test_static_scratch_rejects_oversized_requests():
    import torch

    import paper_1104_0672_gb300 as ark
    from paper_1104_0672_gb300 import _native

    lib = _native.load()
    dev = torch.device("cuda:0")
    grid = ark.Grid.healpix(1024)
    gmax = 15 * inputs.ARCMIN
    kern = ark.Kernel(grid, inputs.gaussian_knots(5 * inputs.ARCMIN, gmax, 256), gmax)
    karr = (ctypes.c_void_p * 1)(kern._h.value)
    x = torch.zeros((1, grid.npix), device=dev)
    out = torch.zeros_like(x)
    st = lib.arkcos_convolve_static(grid._h, karr, 1, ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), 1,
                                    ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream), 0)
    assert st == _native.EWORKSPACE
    assert b"scratch" in lib.arkcos_last_error()
