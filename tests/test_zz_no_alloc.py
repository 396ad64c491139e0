"""The allocation-free field sampler against the allocating one.

dfp2s_sample_zernike_fields_noalloc serves callers that cannot allocate device
memory while drawing frames (a fixed memory plan, a host framework that owns
the allocator, latency-bound loops).  It must give the same fields as
dfp2s_sample_zernike_fields, call after call, although its scratch is one
static array that keeps the previous call's contents.  This file is collected
last so a failure here never hides the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the FP32 tolerance of the other field tests


def _rel_l2(x, y):
    x = x.double().cpu().numpy()
    y = y.double().cpu().numpy()
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


@pytest.fixture(scope="module")
def d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_06713_gb300 as lib
    lib.load()
    return lib


def test_noalloc_matches_allocating_entry_point_twice(d):
    lib = d.load()
    J, N, H, W = 36, 256, 200, 180
    f = d.SpectralFactor(J, N, 8.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for frame, dr in ((3, 2.0), (4, 4.0)):  # two calls in a row on the shared static scratch
        ref = d.sample_zernike_fields(f, dr, 7, frame, H, W)
        out = torch.full((J, H, W), float("nan"), device="cuda")
        rc = lib.dfp2s_sample_zernike_fields_noalloc(f.handle, dr, 7, frame, H, W, ctypes.c_void_p(out.data_ptr()),
                                                     stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel_l2(out, ref) <= TOL


def test_noalloc_rejects_factors_beyond_the_static_scratch(d):
    lib = d.load()
    f = d.SpectralFactor(16, 1024, 8.0)  # 16 * 513 * 1024 * 8 bytes > 48 MiB
    out = torch.empty(16, 64, 64, device="cuda")
    rc = lib.dfp2s_sample_zernike_fields_noalloc(f.handle, 1.0, 0, 0, 64, 64, ctypes.c_void_p(out.data_ptr()),
                                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    buf = ctypes.create_string_buffer(512)
    lib.dfp2s_last_error(buf, 512)
    assert b"static scratch" in buf.value


def test_noalloc_call_takes_no_device_memory(d):
    # the property the entry point exists for: once the first call on the device has looked up the static
    # array (and the kernels are loaded), further calls leave the device's free memory unchanged
    lib = d.load()
    J, N, H, W = 36, 256, 256, 256
    f = d.SpectralFactor(J, N, 8.0)
    out = torch.empty((J, H, W), device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.dfp2s_sample_zernike_fields_noalloc(f.handle, 3.0, 5, 0, H, W, ctypes.c_void_p(out.data_ptr()),
                                                   stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for frame in range(1, 4):
        assert lib.dfp2s_sample_zernike_fields_noalloc(f.handle, 3.0, 5, frame, H, W,
                                                       ctypes.c_void_p(out.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs a second GPU to make another device current")
def test_noalloc_rejects_a_factor_of_another_device(d):
    lib = d.load()
    with torch.cuda.device(0):
        f = d.SpectralFactor(6, 64, 8.0)
    with torch.cuda.device(1):
        out = torch.empty(6, 32, 32, device="cuda")
        rc = lib.dfp2s_sample_zernike_fields_noalloc(f.handle, 1.0, 0, 0, 32, 32, ctypes.c_void_p(out.data_ptr()),
                                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
