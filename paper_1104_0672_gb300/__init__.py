"""GB300 ring-band sphere convolution (the hybrid method of Elsner & Wandelt 2011, ARKCoS).

The compute path is the CUDA library libarkcos.so (C ABI in include/arkcos.h); this package
is its thin PyTorch binding.  Public names (imported lazily so that ``inputs`` can be used
without torch or a GPU):

    Grid.healpix(nside), Grid.ecp(ntheta, nphi), Kernel(grid, knots, gamma_max),
    convolve(grid, kernels, maps), convolve_host(grid, kernels, host_maps),
    convolve_backward(...), convolve_autograd(...), convolve_batch(jobs),
    workspace_size(...), autotune(...), set_launch_shape(...), FLAG_BASIC, FLAG_NO_SHIFT_FIX,
    FLAG_NO_POLE_FIX, FLAG_3XTF32

Submodules: ``inputs`` (seeded synthetic maps and beams), ``support`` (support radius of a
truncated kernel from the truncation-error estimate), ``replicas`` (one process per GPU).
"""

_API = {"Grid", "Kernel", "convolve", "convolve_backward", "convolve_autograd",
        "ConvolveFunction", "workspace_size", "sync_status", "ring_analysis", "ring_synthesis",
        "kernel_info", "stage_timing", "stage_report", "convolve_batch", "batch_workspace_size",
        "convolve_host", "host_workspace_size", "autotune", "set_launch_shape", "measure_peak", "convolve_multi",
        "multi_workspace_size", "FLAG_BASIC",
        "FLAG_NO_SHIFT_FIX", "FLAG_NO_POLE_FIX", "FLAG_3XTF32"}


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
