"""The dense-root form of the field sampler on the GPU (DFP2S_FACTOR_DENSE, dfp2s_sample_zernike_fields_dense):
the per-frequency symmetric root of L diag(lambda) L^T (FP64 Jacobi on the device) against numpy's eigh of the
oracle's matrices, and whole fields against the oracle (sampler.sample_fields_dense, reading R6)."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import sampler, spectrum, zernike

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_06713_gb300 as d
    d.load()
    return d


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("J,H,W,N,dr", [
    (6, 12, 10, 16, 1.0),
    (15, 40, 33, 64, 2.5),    # odd J: the Jacobi matrix padded with a zero row and column
    (36, 200, 150, 256, 3.0),
    (48, 30, 30, 64, 1.0),    # the largest J of the dense form
])
def test_dense_fields_match_oracle(lib, J, H, W, N, dr):
    f = lib.SpectralFactor(J, N, 8.0, kind=lib.FACTOR_DENSE)
    g = lib.sample_zernike_fields_dense(f, dr, 6, 2, H, W).cpu().numpy()
    o = sampler.sample_fields_dense(6, 2, J, H, W, dr, 8.0, N)
    assert _rel(g, o) < TOL


def test_dense_root_at_full_size(lib):
    # the 512 x 512 frame's grid: F at sampled bins against eigh of L diag(lambda) L^T; symmetry and F F^T
    J, N = 36, 1024
    f = lib.SpectralFactor(J, N, 8.0, kind=lib.FACTOR_DENSE)
    rng = np.random.default_rng(0)
    kx = np.concatenate([[0, 0, N // 2, N // 2, 1, 3], rng.integers(0, N // 2 + 1, 40)])
    ky = np.concatenate([[1, N // 2, 0, 7, N - 1, 0], rng.integers(0, N, 40)])
    Fg = lib.dense_root(f)[:, :, torch.as_tensor(kx, device="cuda"), torch.as_tensor(ky, device="cuda")]
    Fg = Fg.permute(2, 0, 1).double().cpu().numpy()  # (bins, J, J)
    lam = spectrum.lambdas(J, N, 8.0)[:, ky, kx].T     # lambda[j, ky, kx] at the bins
    L = zernike.noll_cholesky(J, 1.0)
    S = np.einsum("ik,bk,jk->bij", L, lam, L)
    ev, U = np.linalg.eigh(S)
    Fo = np.einsum("bik,bk,bjk->bij", U, np.sqrt(np.clip(ev, 0, None)), U)
    for b in range(len(kx)):
        if kx[b] == 0 and ky[b] == 0:
            assert np.abs(Fg[b]).max() == 0.0  # DC
            continue
        scale = np.abs(Fo[b]).max()
        assert np.abs(Fg[b] - Fo[b]).max() < 2e-6 * scale, (kx[b], ky[b])
        assert np.abs(Fg[b] - Fg[b].T).max() < 1e-6 * scale
        assert np.abs(Fg[b] @ Fg[b].T - S[b]).max() < 1e-5 * np.abs(S[b]).max()


def test_dense_form_is_refused_where_it_is_not_built(lib):
    L = lib.load()
    h = ctypes.c_void_p()
    p = lib.FactorParams(50, 64, 8.0, lib.FACTOR_DENSE, 0)
    assert L.dfp2s_build_spectral_factor(ctypes.byref(p), ctypes.byref(h), None) == -5  # J > 48
    p = lib.FactorParams(12, 64, 8.0, lib.FACTOR_DENSE, 3)
    assert L.dfp2s_build_spectral_factor(ctypes.byref(p), ctypes.byref(h), None) == -5  # with subharmonics
    f = lib.SpectralFactor(12, 64, 8.0)
    out = torch.empty(12, 8, 8, device="cuda")
    assert L.dfp2s_sample_zernike_fields_dense(f.handle, 1.0, 1, 0, 8, 8, ctypes.c_void_p(out.data_ptr()), None) == -1
    # a dense factor serves the factored sampler unchanged
    fd = lib.SpectralFactor(12, 64, 8.0, kind=lib.FACTOR_DENSE)
    assert torch.equal(lib.sample_zernike_fields(fd, 2.0, 3, 1, 20, 20), lib.sample_zernike_fields(f, 2.0, 3, 1, 20, 20))
