"""Pins of the full (non-approximated) cross-spectral sampler of the oracle (Sec. III-B; reading R29).

* The rank-R root R(k) = D(k) P chol(Gamma) reproduces the cross spectrum built term by term
  (spectrum.cross_spectrum_torus) at every bin.
* The sampler as a linear map M of its Gaussians has M M^T equal to the dense full tensor
  (spectrum.full_tensor_torus) on whole small tori: every cross-covariance at every lag, not a statistic.
* The Philox-driven draw equals that linear map applied to the same Gaussians.
* Theta_j, whose phase sets the sign of every cross-spectrum term, is Noll's aperture transform of Z_j
  (numerical transform over the unit disk).
"""
import math

import numpy as np
import pytest
from scipy.special import jv

from oracle import fullsampler as fs
from oracle import noise, spectrum, zernike


def test_radial_orders_and_rank():
    orders, of = fs.radial_orders(36)
    assert orders == [1, 2, 3, 4, 5, 6, 7, 8]          # Noll 2..37
    assert of[0] == 0 and of[2] == 1 and of[-1] == 7     # Z2 n=1, Z4 n=2, Z37 n=8
    assert fs.radial_orders(15)[0] == [1, 2, 3, 4, 5]   # Noll 2..16
    # the Gram matrix of the orders is positive definite off DC (so the Cholesky root exists)
    G = fs.order_gram(36, 32, 8.0)
    ev = np.linalg.eigvalsh(G[1:, 1:].reshape(-1, 8, 8))
    assert ev.min() > 0


@pytest.mark.parametrize("J,N", [(6, 16), (36, 32)])
def test_root_reproduces_cross_spectrum(J, N):
    A0 = zernike.noll_matrix(J, 1.0)
    Rt = fs.full_root(J, N, 8.0, A0)
    S = spectrum.cross_spectrum_torus(J, N, 8.0, A0)
    RR = np.einsum("yxjr,yxkr->yxjk", Rt, np.conj(Rt))
    _, _, kx, ky = spectrum.torus_frequencies(N, 8.0)
    corner = ((2 * kx) % N == 0) & ((2 * ky) % N == 0)
    assert np.abs(RR[~corner] - S[~corner]).max() <= 1e-12 * np.abs(S).max()
    # on the corners S was made real (a real field): the real root [Re R, Im R] reproduces it
    Rc = Rt[corner]
    RRc = np.einsum("bjr,bkr->bjk", Rc.real, Rc.real) + np.einsum("bjr,bkr->bjk", Rc.imag, Rc.imag)
    assert np.abs(RRc - S[corner]).max() <= 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("J,N", [(3, 8), (6, 8), (9, 16)])
def test_sampler_covariance_is_the_full_tensor(J, N):
    A0 = zernike.noll_matrix(J, 1.0)
    M = fs.operator_matrix_full(J, N, 8.0, A0)
    A = spectrum.full_tensor_torus(J, N, 8.0, A0)
    assert np.linalg.norm(M @ M.T - A) <= 1e-13 * np.linalg.norm(A)
    # the paper's approximation differs from it (Sec. III-D), so the check can fail
    from oracle import sampler
    Aa = spectrum.approx_tensor_torus(spectrum.lambdas(J, N, 8.0), zernike.noll_cholesky(J, 1.0))
    assert np.linalg.norm(Aa - A) > 1e-3 * np.linalg.norm(A)
    assert sampler.grid_size(N, N) >= N


def _gaussians_in_operator_order(seed, frame, J, N):
    R = len(fs.radial_orders(J)[0])
    half = N // 2 + 1
    g = [np.asarray(noise.gaussian_block(seed, fs.TAG_FULL_FIELDS, frame, s, half, 2 * N), np.float64)
         .reshape(half, N, 2) for s in range(2 * R)]
    out = []
    for kx in range(half):
        for ky in range(N):
            if (kx == 0 and ky == 0) or ((kx in (0, N // 2)) and ky > N // 2):
                continue
            corner = (kx in (0, N // 2)) and (ky in (0, N // 2))
            line = (kx == N // 2 or ky == N // 2) and not corner
            for r in range(R):
                for c in (0, 1):
                    out.append(g[r][kx, ky, c])
                    if line:
                        out.append(g[R + r][kx, ky, c])
    return np.array(out)


@pytest.mark.parametrize("J,N", [(6, 8), (9, 16)])
def test_philox_draw_is_the_linear_map_of_its_gaussians(J, N):
    A0 = zernike.noll_matrix(J, 1.0)
    M = fs.operator_matrix_full(J, N, 8.0, A0)
    z = _gaussians_in_operator_order(11, 3, J, N)
    E = fs.full_spectrum(11, 3, J, N, 8.0, A0)
    assert np.abs(np.fft.ifft2(E, axes=(1, 2)).imag).max() < 1e-12 * np.abs(E).max()  # Hermitian
    a = np.real(np.fft.ifft2(E, axes=(1, 2))).ravel()
    assert np.allclose(a, M @ z, rtol=0, atol=1e-12 * np.abs(a).max())
    # the cropped, scaled fields
    f = fs.sample_fields_full(11, 3, J, N - 3, N - 1, 2.5, 8.0, N)
    assert np.allclose(f, 2.5 ** (5 / 6) * a.reshape(J, N, N)[:, : N - 3, : N - 1], rtol=0, atol=1e-12)


def test_zero_lag_variances_are_noll():
    # every field keeps Noll's variance A0_jj (the spectra are normalised per mode)
    J, N = 10, 32
    A0 = zernike.noll_matrix(J, 1.0)
    S = spectrum.cross_spectrum_torus(J, N, 8.0, A0)
    Rt = fs.full_root(J, N, 8.0, A0)
    var = np.einsum("yxjr,yxjr->j", Rt, np.conj(Rt)).real / N ** 2
    assert np.allclose(var, np.diag(A0), rtol=1e-9)
    assert np.allclose(var, np.einsum("yxjj->j", S).real / N ** 2, rtol=1e-12)


@pytest.mark.parametrize("j", [2, 3, 4, 5, 6, 7, 8, 9, 11, 16, 17])
def test_theta_is_nolls_aperture_transform(j):
    # Q_j(f) = (1/pi) int_{|rho| <= 1} Z_j(rho) exp(+2 pi i f . rho) d rho
    #        = sqrt(n+1) J_{n+1}(2 pi |f|) / (pi |f|) Theta_j(phi_f)
    n, _ = zernike.noll_nm(j)
    xr, wr = np.polynomial.legendre.leggauss(60)
    rho, wrho = (xr + 1) / 2, wr / 2
    nt = 128
    th = np.arange(nt) * 2 * np.pi / nt
    R, T = np.meshgrid(rho, th, indexing="ij")
    wt = np.outer(wrho * rho, np.full(nt, 2 * np.pi / nt))
    Z = zernike.zernike(j, R, T)
    X, Y = R * np.cos(T), R * np.sin(T)
    for f, phi in ((0.3, 0.4), (0.7, 2.1), (1.3, -1.0)):
        q = np.sum(wt * Z * np.exp(2j * np.pi * f * (np.cos(phi) * X + np.sin(phi) * Y))) / np.pi
        ref = math.sqrt(n + 1) * jv(n + 1, 2 * np.pi * f) / (np.pi * f) * spectrum.theta_complex(j, np.array(phi))
        assert abs(q - ref) <= 1e-9 * abs(ref), (j, f)
