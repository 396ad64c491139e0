"""Sec. IV-B statistics on the GPU (dfp2s_aperture_statistics, dfp2s_tilt_statistics) against the oracle
(oracle/aperture.py) on the same fields, and the CUDA sampler's fields against the statistics' expectations.

Tolerances: the phase is formed in FP32 (J products of |a Z| <= ~3, error ~6e-6 rad), so the structure function at
one sample's offset (differences of ~0.3 rad) carries ~1e-4 relative error and the OTFs ~1e-5 absolute."""
import numpy as np
import pytest
import torch

from oracle import aperture, sampler, zernike

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_06713_gb300 as d
    d.load()
    return d


def _fields(lib, J, H, W, dr, seed=1, frame=0):
    f = lib.SpectralFactor(J, sampler.grid_size(H, W), 8.0)
    return lib.sample_zernike_fields(f, dr, seed, frame, H, W)


def _check(g, o):
    Dx, Dy, He, Hs = o
    gx, gy = g["D_x"].cpu().numpy(), g["D_y"].cpu().numpy()
    assert gx[0] == 0 and gy[0] == 0
    assert np.abs(gx[1:] - Dx[1:]).max() <= 2e-4 * Dx[1:].max() and np.allclose(gx[1:], Dx[1:], rtol=2e-4)
    assert np.allclose(gy[1:], Dy[1:], rtol=2e-4)
    assert np.abs(g["H_LE"].cpu().numpy() - He).max() < 5e-5
    assert np.abs(g["H_SE"].cpu().numpy() - Hs).max() < 5e-5


@pytest.mark.parametrize("J,H,W,step,dr", [
    (36, 96, 80, 4, 2.0),   # 480 realisations: several per CTA
    (15, 33, 47, 1, 4.0),   # every pixel, odd sizes
    (36, 1, 1, 1, 1.0),     # one realisation
])
def test_aperture_statistics_match_oracle(lib, J, H, W, step, dr):
    a = _fields(lib, J, H, W, dr)
    g = lib.aperture_statistics(a, step)
    _check(g, aperture.aperture_statistics(a.cpu().numpy(), step))


def test_aperture_statistics_full_size(lib):
    # the 512 x 512 frame's fields, every fourth pixel (16384 realisations)
    a = _fields(lib, 36, 512, 512, 2.0, seed=5)
    g = lib.aperture_statistics(a, 4)
    _check(g, aperture.aperture_statistics(a.cpu().numpy(), 4))


def test_tilts_only_short_exposure_is_diffraction_limited(lib):
    # J = 2: the phase is a plane, which the short-exposure OTF removes completely
    a = _fields(lib, 3, 40, 40, 3.0)[:2].contiguous()  # the two tilt fields
    g = lib.aperture_statistics(a, 2)
    H0 = aperture.otf(np.zeros((1, 64, 64)))
    assert np.abs(g["H_SE"].cpu().numpy() - H0).max() < 5e-5
    assert g["H_LE"][0, 8].item() < H0[0, 8] - 0.05  # the tilt jitter lowers the long-exposure OTF
    _check(g, aperture.aperture_statistics(a.cpu().numpy(), 2))


def test_sampler_meets_the_aperture_statistics_expectations(lib):
    # the simulator's own validation (Sec. IV-B): every pixel's vector is N(0, A_0(D/r0)), so the statistics of
    # the CUDA sampler's fields approach the Gaussian expectations (Fig. struct_fun, Fig. SELE); the tilts are
    # large-scale (a frame holds few independent tilt samples), so the bound is four frame-to-frame standard errors
    J, dr, frames = 36, 2.0, 16
    per = []
    for fr in range(frames):
        g = lib.aperture_statistics(_fields(lib, J, 512, 512, dr, seed=9, frame=fr), 4)
        per.append(np.concatenate([g["D_x"].cpu().numpy(), g["D_y"].cpu().numpy(),
                                   g["H_LE"][0, :24].cpu().numpy(), g["H_SE"][0, :24].cpu().numpy()]))
    per = np.array(per)
    m, se = per.mean(axis=0), per.std(axis=0) / np.sqrt(frames)
    A = zernike.noll_matrix(J, dr)
    Ex, Ey = aperture.expected_structure_function(A)
    nus = [(0, v) for v in range(24)]
    E = aperture.expected_otf(A, nus=nus)[0, :24]
    Es = aperture.expected_otf(A, tilt_removed=True, nus=nus)[0, :24]
    want = np.concatenate([Ex, Ey, E, Es])
    assert np.all(np.abs(m - want) <= 4 * se + 1e-9), np.max(np.abs(m - want) / (se + 1e-12))
    assert np.all(se[1:33] < 0.1 * Ex[1:])  # and the bound is informative


@pytest.mark.parametrize("H,W,max_lag", [(96, 80, 20), (512, 512, 64), (7, 300, 6)])
def test_tilt_statistics_match_oracle(lib, H, W, max_lag):
    a = _fields(lib, 6, H, W, 2.0)
    g = lib.tilt_statistics(a, max_lag).cpu().numpy()
    o = aperture.tilt_statistics(a.cpu().numpy(), max_lag)
    assert np.allclose(g, o, rtol=1e-5, atol=1e-7 * np.abs(o).max())
    # the paper's identity on the GPU's own sums
    assert np.allclose(g[..., 2], g[..., 4] + g[..., 5] - 2 * g[..., 0], rtol=1e-5, atol=1e-6 * g[..., 4].max())
    assert np.allclose(g[..., 3], g[..., 6] + g[..., 7] - 2 * g[..., 1], rtol=1e-5, atol=1e-6 * g[..., 6].max())


def test_statistics_reject_bad_arguments(lib):
    import ctypes
    L = lib.load()
    a = torch.zeros(2, 8, 8, device="cuda")
    out = torch.empty(8192 + 66, device="cuda", dtype=torch.float64)
    p = ctypes.c_void_p
    assert L.dfp2s_aperture_statistics(p(a.data_ptr()), 1, 8, 8, 1, p(out.data_ptr()), None) == -1  # J < 2
    assert L.dfp2s_aperture_statistics(p(a.data_ptr()), 2, 8, 8, 0, p(out.data_ptr()), None) == -1  # step 0
    assert L.dfp2s_tilt_statistics(p(a.data_ptr()), 8, 8, 8, p(out.data_ptr()), None) == -1       # lag >= side
