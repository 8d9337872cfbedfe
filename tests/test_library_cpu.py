"""CPU-side checks of the C-ABI library: it builds, loads, exports every symbol the header
declares, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

from paper_1104_0672_gb300 import _native, build

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _native.load(build_if_missing=False)


def header_functions():
    names = set()
    for h in sorted(os.listdir(INCLUDE)):
        if h.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(INCLUDE, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(arkcos_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_expected_entry_points():
    fns = header_functions()
    assert set(fns) == set(_native.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name
    assert lib.arkcos_version().decode().startswith("arkcos")


def test_argument_validation_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.arkcos_create_grid_healpix(0, ctypes.byref(h)) == _native.EINVAL
    assert b"nside" in lib.arkcos_last_error()
    assert lib.arkcos_create_grid_ecp(8, 15, ctypes.byref(h)) == _native.EINVAL
    assert lib.arkcos_create_grid_healpix(4, None) == _native.EINVAL
    assert lib.arkcos_grid_info(None, None, None, None) == _native.EINVAL
    assert lib.arkcos_destroy_grid(None) == _native.OK
    assert lib.arkcos_destroy_kernel(None) == _native.OK
    assert lib.arkcos_convolve(None, None, 1, None, None, 1, None, 0, None, 0) == _native.EINVAL
    assert lib.arkcos_convolve_host(None, None, 1, None, None, 1, 1, None, 0, None, 0) == _native.EINVAL
    assert lib.arkcos_host_workspace_size(None, None, 1, 1, 1, 0, None) == _native.EINVAL
    assert lib.arkcos_autotune(None, None, 1, None, None, 1, None, 0, None, 0, None) == _native.EINVAL
    assert lib.arkcos_set_launch_shape(None, None, 1, 1, 0, None) == _native.EINVAL
    assert lib.arkcos_ring_analysis(None, None, None, 1, None) == _native.EINVAL
    assert lib.arkcos_convolve_multi(None, None, 2, None, None, None, 1, None, 0, None, 0) == _native.EINVAL
    assert lib.arkcos_multi_workspace_size(None, None, 2, 1, 0, 0, None) == _native.EINVAL
    t, ms = ctypes.c_double(), ctypes.c_double()
    assert lib.arkcos_measure_peak(7, ctypes.byref(t), ctypes.byref(ms), None) == _native.EINVAL


def test_product_path_does_not_reference_the_oracle():
    pkg = os.path.dirname(build.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(root, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert not re.search(r"\boracle\.[A-Za-z_]+\(", src), f
                assert "liboracle" not in src and "arkcos_oracle" not in src, f


def test_binding_refuses_host_tensors():
    """No CPU fallback: the device entry points take CUDA tensors only (host maps go through
    convolve_host, which copies them to the device itself)."""
    torch = pytest.importorskip("torch")
    from paper_1104_0672_gb300 import api
    with pytest.raises(TypeError):
        api._need_cuda(torch.zeros(4), "maps")
    with pytest.raises(TypeError):
        api._need_cuda(torch.zeros(4, dtype=torch.float64), "maps")
    with pytest.raises(TypeError):
        api._need_cuda(None, "maps")
