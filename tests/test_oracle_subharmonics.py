"""Pins of the subharmonic sampler of the oracle (Sec. IV-B; reading R31)."""
import math

import numpy as np
import pytest
from scipy.special import jv

from oracle import sampler, spectrum
from oracle import subharmonics as sh


def test_unit_variance_and_the_plain_limit():
    J, N = 10, 64
    lam, s = sh.lambdas_and_amplitudes(J, N, 8.0, 4)
    var = lam.sum(axis=(1, 2)) / N ** 2 + (s ** 2).sum(axis=(1, 2))
    assert np.allclose(var, 1.0, rtol=0, atol=1e-12)
    # zero levels is the paper's sampler, bit for bit
    lam0, s0 = sh.lambdas_and_amplitudes(J, N, 8.0, 0)
    assert s0.size == 0 and np.array_equal(lam0, spectrum.lambdas(J, N, 8.0))
    a = sh.sample_fields(3, 1, J, 40, 30, 2.0, 0, 8.0, N)
    b = sampler.sample_fields(3, 1, J, 40, 30, 2.0, 8.0, N)
    assert np.array_equal(a, b)


def test_subharmonic_part_covariance_closed_form():
    # the subharmonic part is linear in its Gaussians: evaluating it on unit coefficients gives its operator, whose
    # Gram matrix must be sum s^2 cos(2 pi (n dx + m dy) / (N 3^p))
    N, H, W, levels = 16, 5, 6, 2
    _, s = sh.lambdas_and_amplitudes(3, N, 8.0, levels)
    cols = []
    for p in range(levels):
        for d in range(8):
            for unit in (1.0, 1j):
                c = np.zeros((1, levels, 8), dtype=np.complex128)
                c[0, p, d] = unit * s[0, p, d]
                cols.append(sh.subharmonic_part(c, N, H, W)[0].ravel())
    M = np.stack(cols, axis=1)
    C = M @ M.T
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    ys, xs = ys.ravel(), xs.ravel()
    want = np.zeros_like(C)
    for p in range(1, levels + 1):
        for d, (n, m) in enumerate(sh.DIRECTIONS):
            want += s[0, p - 1, d] ** 2 * np.cos(2 * np.pi * (n * (xs[None] - xs[:, None]) + m * (ys[None] - ys[:, None]))
                                                 / (N * 3 ** p))
    assert np.abs(C - want).max() < 1e-14


def _continuous_tilt_autocorrelation(s_over_D):
    # Noll 2 (x tilt): P(f) = 2 * 2 cos^2(phi) G_1(|f|); along x, the angular integral of cos^2(phi) cos(a cos phi)
    # is pi (J_0(a) - J_2(a)) (Jacobi-Anger), so C(s) = 4 pi int G_1(f) f (J_0 - J_2)(2 pi f s) df
    lf = np.linspace(math.log(1e-8), math.log(60.0), 6000)
    f = np.exp(lf)
    G = spectrum.radial_spectra([(1, 1)], f)[0]
    w = G * f * f  # df = f dln f
    c0 = np.trapezoid(w, lf)
    return np.array([np.trapezoid(w * (jv(0, 2 * np.pi * f * s) - jv(2, 2 * np.pi * f * s)), lf) / c0
                     for s in s_over_D])


@pytest.mark.parametrize("N", [128, 512])
def test_subharmonics_bring_the_tilt_correlation_to_the_continuous_one(N):
    # the torus misses the DC cell, where the tilt spectrum (~ f^{-5/3}) holds much of its power: its x-tilt
    # autocorrelation at large lags falls below the continuous-domain one; the subharmonic levels restore it
    lags = [N // 16, N // 8, N // 4]
    rho_c = _continuous_tilt_autocorrelation(np.array(lags) / 8.0)
    lam0 = spectrum.lambdas(1, N, 8.0)[0]
    lam6, s6 = sh.lambdas_and_amplitudes(1, N, 8.0, 6)
    for d, rc in zip(lags, rho_c):
        r0 = sh.unit_autocorrelation(lam0, np.zeros((0, 8)), 0, d)
        r6 = sh.unit_autocorrelation(lam6[0], s6[0], 0, d)
        assert r0 < rc - 0.02                       # the deficit is real
        assert abs(r6 - rc) < 0.35 * abs(r0 - rc), (d, r0, r6, rc)  # six levels remove most of it
    # more levels, smaller error (each level recovers a factor of about 3^(1/3) of the missing tilt power)
    lam3, s3 = sh.lambdas_and_amplitudes(1, N, 8.0, 3)
    d = lags[-1]
    e3 = abs(sh.unit_autocorrelation(lam3[0], s3[0], 0, d) - rho_c[-1])
    e6 = abs(sh.unit_autocorrelation(lam6[0], s6[0], 0, d) - rho_c[-1])
    assert e6 < e3


def test_philox_layout_of_the_subharmonic_gaussians():
    from oracle import noise
    g = sh.subharmonic_gaussians(5, 2, 3, 2)
    sub = noise.subsequence(sh.TAG_SUBHARMONICS, 2, 1)
    w0, w1, w2, w3 = noise.philox_words(5, sub, np.array([5], dtype=np.uint64))  # level 2, k = 1
    a, b = noise.box_muller(w0, w1)
    c, d = noise.box_muller(w2, w3)
    assert g[1, 1, 2] == complex(float(a[0]), float(b[0])) and g[1, 1, 3] == complex(float(c[0]), float(d[0]))


def test_deep_rule_reaches_the_small_frequency_limits():
    # the subharmonics need G_n far below the torus bins.  For n >= 2, g_n is integrable at 0 and
    # f G_n(f) -> (1/2) int g_n dv as f -> 0; for n = 1 the deep rule agrees with the t-form of R1 where that
    # adaptive quadrature converges; at the torus bins it agrees with the standard rule
    from scipy.integrate import quad
    for n in (2, 3):
        edges = [0, 1e-6, 1e-3, 0.1, 1, 2, 4, 8, 16, 32, 64, 128, 400]
        half = 0.5 * sum(quad(lambda v: spectrum.g_radial(n, n, v), a, b, limit=500, epsrel=1e-12)[0]
                         for a, b in zip(edges[:-1], edges[1:]))
        f = 1e-9
        assert f * spectrum.radial_spectra([(n, n)], [f], deep=True)[0, 0] == pytest.approx(half, rel=1e-6)
    for f in (1e-3, 1e-5, 1e-7, 3.7e-9):  # (the t-form's adaptive quadrature does not converge at every f)
        assert spectrum.radial_spectra([(1, 1)], [f], deep=True)[0, 0] == pytest.approx(
            spectrum.radial_spectrum_tform(1, 1, f), rel=1e-9)
    fs = np.array([2e-3, 0.05, 1.0, 4.0])
    pairs = [(1, 1), (2, 2), (5, 5)]
    assert np.allclose(spectrum.radial_spectra(pairs, fs, deep=True), spectrum.radial_spectra(pairs, fs), rtol=1e-9)
