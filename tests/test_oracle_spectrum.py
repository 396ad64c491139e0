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
