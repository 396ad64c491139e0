"""Pins of the oracle's aperture and spatial statistics (Sec. IV-B; reading R30)."""
import numpy as np
import pytest

from oracle import aperture, sampler, stats, zernike


def _draws(J, dr, n, seed):
    rng = np.random.default_rng(seed)
    L = zernike.noll_cholesky(J, dr)
    return rng.standard_normal((n, J)) @ L.T  # a ~ N(0, A_0(D/r0))


def test_diffraction_limited_otf():
    H = aperture.otf(np.zeros((1, 64, 64)))
    E = aperture.expected_otf(np.zeros((3, 3)))
    assert np.abs(H - E).max() < 1e-12  # both the discrete autocorrelation of the aperture
    assert H[0, 0] == pytest.approx(1.0)
    nu = np.arange(33)
    ref = aperture.diffraction_otf_analytic(nu / 32.0)
    assert np.abs(H[0, :33] - ref).max() < 0.03  # 797 samples against the continuous disk
    assert np.abs(H[:33, 0] - ref).max() < 0.03
    assert np.allclose(H[0, 1:], H[0, :0:-1])  # symmetric


def test_otf_of_a_sample_exact_shift():
    # a phase ramp 2 pi (k x_idx)/64 moves the PSF by k bins: |F|^2 shifted, its OTF H_diff e^{2 pi i k nu/64}
    J = 3
    a = np.zeros((1, J))
    a[0, 0] = 1.0
    phi = aperture.phases(a)  # a_2 Z_2 = 2 a_2 x, x = (i - 32)/16
    k = 2
    ramp = 2 * np.pi * k * (np.arange(64) - 32)[None, None, :] / 64.0 * np.ones((1, 64, 1))
    H = aperture.otf(ramp)
    H0 = aperture.otf(np.zeros((1, 64, 64)))
    nu = np.arange(64)
    assert np.allclose(H, H0 * np.cos(2 * np.pi * k * nu / 64.0)[None, :], atol=1e-12)
    # the plane removal takes it out completely
    assert np.allclose(aperture.otf(aperture.remove_plane(ramp)), H0, atol=1e-12)
    assert np.allclose(aperture.otf(aperture.remove_plane(phi)), H0, atol=1e-12)


def test_plane_removal_is_the_least_squares_residual():
    phi = aperture.phases(_draws(10, 2.0, 3, 1))
    r = aperture.remove_plane(phi)
    P, xx, yy = aperture._aperture()
    m = P > 0
    for basis in (np.ones(m.sum()), xx[m], yy[m]):
        assert np.abs(r[:, m] @ basis).max() < 1e-9
    assert np.all(r[:, ~m] == 0)
    # and only a plane was removed
    d = (phi - r)[:, m]
    X = np.stack([np.ones(m.sum()), xx[m], yy[m]], axis=1)
    coef, *_ = np.linalg.lstsq(X, d.T, rcond=None)
    assert np.abs(X @ coef - d.T).max() < 1e-9


def test_structure_function_with_many_modes_is_kolmogorov():
    # Eq. (fried_struct): D(r) = 6.88 (r / r0)^{5/3}; Noll's A_0 is the expansion of exactly that phase (R21), so
    # the expectation over enough modes reaches it; r = delta / 32 aperture diameters
    dr = 2.0
    Dx, Dy = aperture.expected_structure_function(zernike.noll_matrix(135, dr))  # n <= 15
    for d in (8, 16, 24, 32):
        ref = 6.88 * (d / 32.0 * dr) ** (5 / 3)
        assert Dx[d] == pytest.approx(ref, rel=0.04), d
        assert Dy[d] == pytest.approx(ref, rel=0.04), d
    # fewer modes miss the small scales first
    Dx36, _ = aperture.expected_structure_function(zernike.noll_matrix(36, dr))
    assert Dx36[2] < 0.9 * Dx[2] and Dx36[32] == pytest.approx(Dx[32], rel=0.12)


def test_long_exposure_otf_with_many_modes_is_frieds():
    # E[e^{-j dphi}] = exp(-D/2) for Gaussian phase: H_LE = H_diff exp(-3.44 (nu / r0)^{5/3})
    dr = 2.0
    nus = [(0, v) for v in range(20)]
    E = aperture.expected_otf(zernike.noll_matrix(135, dr), nus=nus)
    H0 = aperture.otf(np.zeros((1, 64, 64)))
    for v in (2, 4, 8, 12):
        ref = H0[0, v] * np.exp(-3.44 * (v / 32.0 * dr) ** (5 / 3))
        assert E[0, v] == pytest.approx(ref, rel=0.05, abs=2e-4), v
    Es = aperture.expected_otf(zernike.noll_matrix(135, dr), tilt_removed=True, nus=nus)
    assert np.all(Es[0, 1:20] > E[0, 1:20])  # removing the tilt raises the OTF


@pytest.mark.parametrize("J,dr", [(15, 1.0), (36, 3.0)])
def test_empirical_statistics_reach_their_expectation(J, dr):
    a = _draws(J, dr, 3000, 2)
    phi = aperture.phases(a)
    Dx, Dy = aperture.structure_function(phi)
    A = zernike.noll_matrix(J, dr)
    Ex, Ey = aperture.expected_structure_function(A)
    assert np.allclose(Dx[1:], Ex[1:], rtol=0.08) and np.allclose(Dy[1:], Ey[1:], rtol=0.08)
    H = aperture.otf(phi)
    E = aperture.expected_otf(A)
    assert np.abs(H[0, :24] - E[0, :24]).max() < 0.03
    Hs = aperture.otf(aperture.remove_plane(phi))
    Es = aperture.expected_otf(A, tilt_removed=True)
    assert np.abs(Hs[0, :24] - Es[0, :24]).max() < 0.03
    # a planted error (the SE expectation without the plane removal) is caught
    assert np.abs(Hs[0, :24] - E[0, :24]).max() > 0.05


def test_realisations_follow_the_subgrid():
    f = np.arange(2 * 5 * 7, dtype=np.float64).reshape(2, 5, 7)
    r = aperture.realisations(f, 3)
    assert r.shape == (2 * 3, 2)
    assert np.array_equal(r[:, 0], f[0, ::3, ::3].ravel()) and np.array_equal(r[:, 1], f[1, ::3, ::3].ravel())


def test_tilt_statistics_identity_and_expectation():
    J, H, W, dr = 6, 96, 96, 2.0
    N = sampler.grid_size(H, W)
    per = []
    frames = 24
    for fr in range(frames):
        out = aperture.tilt_statistics(sampler.sample_fields(3, fr, J, H, W, dr, 8.0, N), 16)
        # the paper's identity, exactly, for the window means
        assert np.allclose(out[..., 2], out[..., 4] + out[..., 5] - 2 * out[..., 0], rtol=0, atol=1e-12)
        assert np.allclose(out[..., 3], out[..., 6] + out[..., 7] - 2 * out[..., 1], rtol=0, atol=1e-12)
        assert np.all(out[:, 0, 2:4] == 0) and np.allclose(out[:, 0, 0], out[:, 0, 4])
        per.append(out)
    per = np.array(per)
    acc, se = per.mean(axis=0), per.std(axis=0) / np.sqrt(frames)
    # the expectation: A~(d) of the sampler (the tilt rows of L have one entry, so A~_00(d) = A0_00 rho_0(d))
    lags = [(0, d) for d in range(17)] + [(d, 0) for d in range(17)]
    C = stats.approx_covariance(J, N, 8.0, dr, lags)
    want_x = np.array([C[l][0, 0] for l in range(17)])
    want_y = np.array([C[17 + l][1, 1] for l in range(17)])
    assert np.all(np.abs(acc[0, :, 0] - want_x) < 4 * se[0, :, 0] + 0.02 * want_x[0])
    assert np.all(np.abs(acc[1, :, 1] - want_y) < 4 * se[1, :, 1] + 0.02 * want_y[0])
    # the DTV grows with the lag (Sec. IV-B: monotonically increasing)
    assert np.all(np.diff(acc[0, :, 2]) > 0) and np.all(np.diff(acc[1, :, 3]) > 0)
