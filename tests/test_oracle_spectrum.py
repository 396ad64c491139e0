"""Pins for the oracle's field spectra (Sec. III-B/III-C; readings R1, R2, R5)."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import jv

from oracle import spectrum, zernike


@pytest.mark.parametrize("n,n2,f", [(1, 1, 0.003), (1, 1, 0.4), (2, 2, 0.05), (3, 5, 1.3), (7, 7, 0.02),
                                    (8, 8, 2.5), (1, 3, 0.3)])
def test_v_form_matches_t_integral(n, n2, f):
    # the oracle's substituted integral against adaptive quadrature of the t-form of R1
    a = spectrum.radial_spectrum(n, n2, f)[0]
    b = spectrum.radial_spectrum_tform(n, n2, f)
    assert a == pytest.approx(b, rel=1e-7)


def _plane_integral_of_radial(n):
    # int G_nn(f) 2 pi f df over (0, inf); below f0 the small-f power law of G
    # (f^{-5/3} for tilt, f^{-1} otherwise) is integrated in closed form
    f0 = 1e-5
    fs = np.exp(np.linspace(math.log(f0), math.log(400.0), 9001))
    G = spectrum.radial_spectrum(n, n, fs)
    y = G * 2 * math.pi * fs * fs  # d f = f d ln f
    alpha = 5.0 / 3.0 if n == 1 else 1.0
    tail = 2 * math.pi * G[0] * f0 * f0 / (2.0 - alpha)
    return np.trapezoid(y, np.log(fs)) + tail


def _noll_integral(n):
    # int u^{-11/3} [J_{n+1}(2 pi u)/(pi u)]^2 d^2u
    g = lambda u: 2 * math.pi * u ** (-8.0 / 3.0) * jv(n + 1, 2 * math.pi * u) ** 2 / (math.pi * u) ** 2
    edges = [0.0, 1e-3, 0.1, 0.5] + list(np.arange(1.0, 60.0, 1.0))
    return sum(quad(g, a, b, limit=400, epsabs=0, epsrel=1e-12)[0] for a, b in zip(edges[:-1], edges[1:]))


@pytest.mark.parametrize("n", [1, 2, 4, 8])
def test_spectrum_integrates_to_path_weight_times_noll(n):
    # int d^2f P(f) = int_0^1 (1-t)^{5/3} dt * int d^2u u^{-11/3}|Q|^2 = (3/8) * Noll's integral
    # (the Jacobian ((1-t)/(2t))^2 of R1 makes the f-integral independent of t)
    assert _plane_integral_of_radial(n) == pytest.approx(0.375 * _noll_integral(n), rel=5e-4)


def test_lambda_normalisation_and_symmetry():
    N, ppd = 32, 4.0
    for j in (2, 3, 4, 5, 8, 11, 37):
        lam = spectrum.lambda_mode(j, N, ppd)
        assert lam[0, 0] == 0.0
        assert np.all(lam >= 0)
        assert lam.mean() == pytest.approx(1.0, rel=1e-13)       # unit-variance field (R2, R5)
        neg = lam[(-np.arange(N)) % N][:, (-np.arange(N)) % N]
        assert np.allclose(lam, neg, rtol=1e-12, atol=1e-14 * lam.max())         # even -> real field
        flipx = lam[:, (-np.arange(N)) % N]
        assert np.allclose(lam, flipx, rtol=1e-12, atol=1e-14 * lam.max())       # P(fx, fy) = P(-fx, fy)
    # x-tilt (cos phi) carries no power along ky, y-tilt none along kx
    l2 = spectrum.lambda_mode(2, N, ppd)
    l3 = spectrum.lambda_mode(3, N, ppd)
    assert np.all(l2[1:, 0] < 1e-25 * l2.max())
    assert np.all(l3[0, 1:] < 1e-25 * l3.max())


def test_cross_spectrum_is_hermitian_psd_and_matches_lambda():
    J, N, ppd = 6, 8, 2.0
    A0 = zernike.noll_matrix(J, 2.0)
    S = spectrum.cross_spectrum_torus(J, N, ppd, A0)
    assert np.allclose(S, np.conj(np.swapaxes(S, -1, -2)), atol=1e-14)
    ev = np.linalg.eigvalsh(S)
    assert ev.min() > -1e-12 * ev.max()
    for a in range(J):
        lam = spectrum.lambda_mode(a + 2, N, ppd)
        assert np.allclose(S[:, :, a, a].real, lam * A0[a, a], rtol=1e-12, atol=1e-300)


def _plane_integral_of_cross_radial(n, n2):
    # int G_nn'(f) f df over (0, inf) (the 2 pi of the plane goes with the angular integral); below f0 the
    # small-f power law of G (f^{-5/3} for the tilt pair, f^{-1} otherwise) is integrated in closed form
    f0 = 1e-5
    fs = np.exp(np.linspace(math.log(f0), math.log(400.0), 9001))
    G = spectrum.radial_spectrum(n, n2, fs)
    alpha = 5.0 / 3.0 if n == n2 == 1 else 1.0
    return np.trapezoid(G * fs * fs, np.log(fs)) + G[0] * f0 * f0 / (2.0 - alpha)


def _plane_integral_of_cross_spectrum(i, j):
    # int d^2f sqrt((n+1)(n'+1)) Theta_i(phi) conj(Theta_j(phi)) G_nn'(|f|): the zero-displacement value of
    # the (i, j) slice of the full correlation tensor (Sec. III-B), up to the constant shared by all pairs
    ni, _ = zernike.noll_nm(i)
    nj, _ = zernike.noll_nm(j)
    phi = np.arange(720) * (2 * math.pi / 720)  # exact for the trigonometric polynomials of Theta
    ang = 2 * math.pi * np.mean(spectrum.theta_complex(i, phi) * np.conj(spectrum.theta_complex(j, phi)))
    return math.sqrt((ni + 1) * (nj + 1)) * ang * _plane_integral_of_cross_radial(min(ni, nj), max(ni, nj))


@pytest.mark.parametrize("i,j", [(2, 8), (3, 7), (4, 11), (5, 13), (6, 12), (2, 16), (7, 17), (11, 22),
                                 (2, 3), (4, 6), (2, 4), (7, 8)])
def test_cross_spectrum_integrates_to_noll_correlation(i, j):
    # Sec. III-B: at s = 0 the tensor is Noll's matrix.  Integrated over the frequency plane, the cross
    # spectrum of the model (the angular phases of theta_complex and the off-diagonal radial spectra) must
    # give Noll's closed-form correlation A0_ij / sqrt(A0_ii A0_jj), sign included, for every pair; pairs
    # Noll makes zero (different m, or cos against sin) must integrate to zero
    Pij = _plane_integral_of_cross_spectrum(i, j)
    Pii = _plane_integral_of_cross_spectrum(i, i).real
    Pjj = _plane_integral_of_cross_spectrum(j, j).real
    rho = Pij / math.sqrt(Pii * Pjj)
    ref = zernike.noll_covariance_entry(i, j) / math.sqrt(zernike.noll_covariance_entry(i, i)
                                                           * zernike.noll_covariance_entry(j, j))
    assert abs(rho.imag) < 1e-12
    if ref == 0.0:
        assert abs(rho.real) < 1e-12
    else:
        assert rho.real == pytest.approx(ref, rel=2e-4)


def test_torus_cross_spectrum_at_zero_lag_has_noll_signs_and_converges():
    # The zero-lag block of the torus tensor, sum_k S_ij(k) / N^2 (cross_spectrum_torus), as correlations:
    #  - every pair Noll makes non-zero has Noll's sign;
    #  - pairs Noll makes zero by symmetry vanish on the torus too when the square lattice keeps that
    #    symmetry (cos against sin: the reflection ky -> -ky; m +- m' not a multiple of 4: the quarter turn);
    #    the others keep a cos(4 phi) lattice term, and so do all pairs a discretisation error, which must
    #    shrink as the frequency spacing pix_per_D / N is halved;
    #  - tilt pairs carry the torus's low-frequency deficit (Sec. IV-B: the FFT method misses the power
    #    inside the lowest bin), which also shrinks with the spacing (Noll 2 with Noll 8 is followed).
    J = 10
    A0 = zernike.noll_matrix(J, 1.0)
    ref = A0 / np.sqrt(np.outer(np.diag(A0), np.diag(A0)))
    m = np.array([zernike.noll_nm(j + 2)[1] for j in range(J)])
    par = np.array([(j + 2) % 2 if zernike.noll_nm(j + 2)[1] > 0 else -1 for j in range(J)])
    cos_sin = (par[:, None] >= 0) & (par[None, :] >= 0) & (par[:, None] != par[None, :])
    quarter = (((m[:, None] + m[None, :]) % 4) != 0) & ((np.abs(m[:, None] - m[None, :]) % 4) != 0)
    kept = (ref == 0.0) & (cos_sin | quarter)
    errs, errs28 = [], []
    for N, ppd in ((32, 8.0), (64, 8.0), (128, 8.0)):
        S = spectrum.cross_spectrum_torus(J, N, ppd, A0)
        C0 = S.sum(axis=(0, 1)) / (N * N)
        assert np.abs(C0.imag).max() < 1e-4 * np.abs(C0.real).max()
        C0 = C0.real
        rho = C0 / np.sqrt(np.outer(np.diag(C0), np.diag(C0)))
        nz = ref != 0.0
        assert np.all(np.sign(rho[nz]) == np.sign(ref[nz]))
        assert np.abs(rho[kept]).max() < 1e-4
        errs.append(np.abs(rho - ref).max())
        errs28.append(abs(rho[0, 6] - ref[0, 6]))  # Noll 2 with Noll 8
    assert errs[0] > errs[1] > errs[2]
    assert errs28[0] > errs28[1] > errs28[2]
