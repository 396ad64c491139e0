"""Failure paths, made to fail without faulting the GPU.

* A bounded wait on a barrier that nothing completes runs out and the host reads
  DFP2S_ETIMEOUT; the kernel has let its bulk copy land and released its tensor
  memory, so a tensor-core blur launched afterwards still matches the oracle.
* A simulated device-allocation failure (the library's own test hook, a fake of
  the failing cudaMalloc) makes every creating entry point return DFP2S_ENOMEM,
  creates no handle and leaks no device memory.
"""
import ctypes

import numpy as np
import pytest
import torch

from inputs import synthetic
from oracle import image

pytestmark = pytest.mark.gpu

ETIMEOUT, ENOMEM = -4, -2


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_06713_gb300 as d
    d.load()
    return d


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _message(L):
    buf = ctypes.create_string_buffer(512)
    L.dfp2s_last_error(buf, 512)
    return buf.value.decode()


def _bf16(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def test_bounded_wait_runs_out_and_the_context_stays_usable(lib):
    L = lib.load()
    for limit_ns in (1_000_000, 20_000_000):
        assert L.dfp2s_check_bounded_wait(limit_ns, _stream()) == ETIMEOUT
        assert "ran out" in _message(L)
    assert L.dfp2s_check_bounded_wait(10, _stream()) == -1  # limit below 1 us
    # tensor memory was released and the context works: a tensor-core blur against the oracle
    C, H, W, K = 3, 40, 160, 100
    img = synthetic.blobs(H, W, C, n=6, seed=1)
    basis = synthetic.random_orthonormal_rows(K, 33 * 33, seed=2).reshape(K, 33, 33)
    w = np.random.default_rng(3).standard_normal((H, W, K)).astype(np.float32)
    P = lib.P2S(36, torch.as_tensor(basis, dtype=torch.float32, device="cuda"))
    g = lib.basis_blur_tc(P, torch.as_tensor(img, device="cuda"), torch.as_tensor(w, device="cuda")).cpu().numpy()
    P.check()
    o = image.basis_blur(_bf16(img - 0.5) + 0.5, w, _bf16(basis))
    assert float(np.linalg.norm(g - o) / np.linalg.norm(o)) < 1e-5


def _create_factor(L):
    from paper_2210_06713_gb300 import FactorParams
    h = ctypes.c_void_p()
    p = FactorParams(12, 64, 8.0, 0)
    rc = L.dfp2s_build_spectral_factor(ctypes.byref(p), ctypes.byref(h), _stream())
    return rc, h


def _create_p2s(L, basis):
    h = ctypes.c_void_p()
    rc = L.dfp2s_p2s_create(12, basis.shape[0], ctypes.c_void_p(basis.data_ptr()), ctypes.byref(h))
    return rc, h


def test_simulated_allocation_failures_return_enomem_without_leaks(lib):
    L = lib.load()
    basis = torch.as_tensor(synthetic.random_orthonormal_rows(16, 33 * 33, seed=4).reshape(16, 33, 33),
                            dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    try:
        for create, destroy in ((_create_factor, L.dfp2s_factor_destroy),
                                (lambda L: _create_p2s(L, basis), L.dfp2s_p2s_destroy)):
            failed = 0
            for n in range(1, 40):
                assert L.dfp2s_debug_fail_allocation(n) == 0
                rc, h = create(L)
                L.dfp2s_debug_fail_allocation(0)
                if rc == 0:  # fewer than n allocations: created
                    assert h.value
                    destroy(h)
                    break
                assert rc == ENOMEM, (n, rc, _message(L))
                assert not h.value  # no handle on failure
                failed += 1
            assert failed >= 2  # the failures happened at different allocations
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 >= free0 - (2 << 20)  # nothing leaked (allocation granularity aside)
    finally:
        L.dfp2s_debug_fail_allocation(0)
    assert L.dfp2s_debug_fail_allocation(-1) == -1
