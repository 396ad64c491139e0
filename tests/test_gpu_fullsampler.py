"""The exact sampler of the full cross-spectral density on the GPU (dfp2s_sample_zernike_fields_full) against the
oracle (oracle/fullsampler.py, Sec. III-B, reading R29): element by element on whole fields, from tiny grids to
the 512 x 512 frame's N = 1024 grid, and by its statistics where the oracle cannot follow (3840 x 2160)."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import fullsampler as fs
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
    (3, 1, 1, 16, 1.0),       # minimal J, one pixel
    (6, 12, 10, 16, 1.0),     # every bin of the grid is a Nyquist line, a corner or next to one
    (15, 40, 33, 128, 2.5),   # odd width, five radial orders
    (36, 64, 64, 128, 4.0),   # eight orders
    (36, 200, 150, 256, 3.0),
    (64, 30, 30, 64, 1.0),    # the largest J: ten orders
])
def test_full_fields_match_oracle(lib, J, H, W, N, dr):
    f = lib.SpectralFactor(J, N, 8.0, kind=lib.FACTOR_FULL)
    g = lib.sample_zernike_fields_full(f, dr, 7, 2, H, W).cpu().numpy()
    o = fs.sample_fields_full(7, 2, J, H, W, dr, 8.0, N)
    assert _rel(g, o) < TOL


def test_full_fields_full_size_512(lib):
    # the 512 x 512 frame's grid, every element
    J, H, W, N = 36, 512, 512, 1024
    f = lib.SpectralFactor(J, N, 8.0, kind=lib.FACTOR_FULL)
    g = lib.sample_zernike_fields_full(f, 2.0, 3, 1, H, W).cpu().numpy()
    o = fs.sample_fields_full(3, 1, J, H, W, 2.0, 8.0, N)
    assert _rel(g, o) < TOL
    for j in (0, 2, 9, 35):  # per mode as well (the high orders are small)
        assert _rel(g[j], o[j]) < 3 * TOL, j


def test_full_fields_4k_statistics(lib):
    # 3840 x 2160 (N = 4096): per-mode variance A0_jj (D/r0)^{5/3} and the sign structure of the zero-lag
    # covariance, from the fields of a few frames
    J, H, W, N, dr = 36, 2160, 3840, 4096, 4.0
    f = lib.SpectralFactor(J, N, 8.0, kind=lib.FACTOR_FULL)
    A0 = zernike.noll_matrix(J, dr)
    acc = np.zeros((J, J))
    frames = 3
    for fr in range(frames):
        a = lib.sample_zernike_fields_full(f, dr, 11, fr, H, W).double().reshape(J, -1)
        acc += (a @ a.T / a.shape[1]).cpu().numpy()
    C = acc / frames
    var_ratio = np.diag(C) / np.diag(A0)
    assert np.all(np.abs(var_ratio[2:] - 1) < 0.08), var_ratio  # tilts (large-scale) sampled less often
    assert np.all(np.abs(var_ratio[:2] - 1) < 0.5), var_ratio[:2]
    # Noll's strongest off-diagonal couplings keep their sign: (2, 8), (3, 7), (4, 11)
    for i, j in ((0, 6), (1, 5), (2, 9)):
        assert C[i, j] * A0[i, j] > 0 and abs(C[i, j]) > 0.3 * abs(A0[i, j]), (i, j, C[i, j], A0[i, j])


def test_cross_correlation_the_approximation_drops(lib):
    # Sec. III-D: the approximation has no tilt-defocus cross-covariance at any lag (different m), the full
    # tensor an odd one; the GPU fields, averaged over frames, follow the full tensor
    J, H, W, N, dr = 3, 224, 224, 256, 1.0
    f = lib.SpectralFactor(J, N, 8.0, kind=lib.FACTOR_FULL)
    A0 = zernike.noll_matrix(J, 1.0)
    S = spectrum.cross_spectrum_torus(J, N, 8.0, A0)
    Cs = np.real(np.fft.ifft2(S, axes=(0, 1)))  # E[a_i(x) a_j(x + s)] = Cs[sy, sx, i, j]
    lag = 12
    want = Cs[0, lag, 0, 2]
    assert abs(want) > 0.02 * np.sqrt(A0[0, 0] * A0[2, 2])  # a real correlation, not rounding
    vals = []
    for fr in range(48):
        a = lib.sample_zernike_fields_full(f, dr, 5, fr, H, W).double()
        vals.append(float((a[0, :, : W - lag] * a[2, :, lag:]).mean()))
    m, se = np.mean(vals), np.std(vals) / np.sqrt(len(vals))
    assert abs(m - want) < 4 * se + 0.1 * abs(want), (m, se, want)
    assert abs(m) > 4 * se  # and not the approximation's zero


def test_full_sampler_needs_a_full_factor(lib):
    L = lib.load()
    f = lib.SpectralFactor(6, 32, 8.0)
    out = torch.empty(6, 8, 8, device="cuda")
    rc = L.dfp2s_sample_zernike_fields_full(f.handle, 1.0, 1, 0, 8, 8, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
    ff = lib.SpectralFactor(6, 32, 8.0, kind=lib.FACTOR_FULL)
    rc = L.dfp2s_sample_zernike_fields_full(ff.handle, 1.0, 1, 0, 33, 8, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1  # does not fit the grid
    # the full factor still serves the factored sampler, unchanged
    a = lib.sample_zernike_fields(ff, 1.5, 4, 0, 20, 20).cpu().numpy()
    b = lib.sample_zernike_fields(lib.SpectralFactor(6, 32, 8.0), 1.5, 4, 0, 20, 20).cpu().numpy()
    assert np.array_equal(a, b)
    assert sampler.grid_size(20, 20) == 64
