"""Subharmonic levels of the factored sampler on the GPU (dfp2s_factor_params.subharmonic_levels) against the oracle
(oracle/subharmonics.py, Sec. IV-B, reading R31)."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import sampler, spectrum, zernike
from oracle import subharmonics as sh

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


@pytest.mark.parametrize("J,H,W,levels,dr", [
    (10, 40, 33, 3, 2.0),
    (36, 100, 90, 6, 3.0),
    (15, 1, 7, 12, 1.0),   # the most levels, one row
])
def test_subharmonic_fields_match_oracle(lib, J, H, W, levels, dr):
    N = sampler.grid_size(H, W)
    f = lib.SpectralFactor(J, N, 8.0, subharmonics=levels)
    g = lib.sample_zernike_fields(f, dr, 4, 3, H, W).cpu().numpy()
    o = sh.sample_fields(4, 3, J, H, W, dr, levels, 8.0, N)
    assert _rel(g, o) < TOL
    # the tilt fields, where the subharmonics carry most of their power, on their own
    assert _rel(g[:2], o[:2]) < TOL


def test_subharmonic_fields_full_size(lib):
    J, H, W, levels = 36, 512, 512, 9
    f = lib.SpectralFactor(J, 1024, 8.0, subharmonics=levels)
    g = lib.sample_zernike_fields(f, 2.0, 8, 1, H, W).cpu().numpy()
    o = sh.sample_fields(8, 1, J, H, W, 2.0, levels, 8.0, 1024)
    assert _rel(g, o) < TOL


def test_zero_levels_is_the_paper_sampler_and_full_is_refused(lib):
    a = lib.sample_zernike_fields(lib.SpectralFactor(12, 64, 8.0, subharmonics=0), 2.0, 1, 0, 30, 30)
    b = lib.sample_zernike_fields(lib.SpectralFactor(12, 64, 8.0), 2.0, 1, 0, 30, 30)
    assert torch.equal(a, b)
    L = lib.load()
    h = ctypes.c_void_p()
    p = lib.FactorParams(12, 64, 8.0, lib.FACTOR_FULL, 3)
    assert L.dfp2s_build_spectral_factor(ctypes.byref(p), ctypes.byref(h), None) == -5
    p = lib.FactorParams(12, 64, 8.0, lib.FACTOR_FACTORED, 13)
    assert L.dfp2s_build_spectral_factor(ctypes.byref(p), ctypes.byref(h), None) == -1


def test_tilt_dtv_follows_the_subharmonic_expectation(lib):
    # over many frames the x-tilt differential variance of the CUDA fields reaches 2 A0_00 (D/r0)^{5/3} (1 - rho(d))
    # of the subharmonic sampler, far below the plain torus sampler's (whose missing low frequencies decorrelate
    # the tilt too fast); the DTV is free of each frame's near-constant subharmonic offset
    J, H, W, N, levels, dr, frames = 3, 120, 120, 256, 9, 1.0, 64
    lags = [8, 16, 32, 60]
    lam, s = sh.lambdas_and_amplitudes(J, N, 8.0, levels)
    want = np.array([2 * (1 - sh.unit_autocorrelation(lam[0], s[0], 0, d)) for d in lags])
    lam0 = spectrum.lambdas(1, N, 8.0)[0]
    plain = np.array([2 * (1 - sh.unit_autocorrelation(lam0, np.zeros((0, 8)), 0, d)) for d in lags])
    f = lib.SpectralFactor(J, N, 8.0, subharmonics=levels)
    a00 = zernike.noll_matrix(J, dr)[0, 0]
    per = []
    for fr in range(frames):
        t = lib.tilt_statistics(lib.sample_zernike_fields(f, dr, 21, fr, H, W), max(lags)).cpu().numpy()
        per.append(t[0, lags, 2] / a00)
    per = np.array(per)
    m, se = per.mean(axis=0), per.std(axis=0) / np.sqrt(frames)
    assert np.all(np.abs(m - want) < 4 * se + 0.005), (m, se, want)
    assert np.all(plain - want > 10 * se)
