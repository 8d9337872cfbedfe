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


def test_static_scratch_matches_workspace_entry_point():
    import torch

    import paper_1104_0672_gb300 as ark
    from paper_1104_0672_gb300 import _native

    assert torch.cuda.is_available()
    lib = _native.load()
    dev = torch.device("cuda:0")
    grid = ark.Grid.healpix(128)
    gmax = 2.5 * inputs.DEG
    kern = ark.Kernel(grid, inputs.gaussian_knots(50 * inputs.ARCMIN, gmax, 256), gmax)
    karr = (ctypes.c_void_p * 1)(kern._h.value)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    # two calls in a row, each on fresh input, each against the workspace entry point
    for call in range(2):
        x = torch.from_numpy(inputs.white_noise(grid.npix, 2, config=14, salt=call)).to(dev)
        ref = ark.convolve(grid, kern, x).cpu().numpy()
        out = torch.full_like(x, float("nan"))
        st = lib.arkcos_convolve_static(grid._h, karr, 1, ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), 2, stream, 0)
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
