"""Pins for the oracle's field statistics (Sec. III-D, Eq. A tilde).

  * field_covariance against a brute-force loop over pixel pairs (tiny frames, every lag sign) and a constant
    field (v v^T at every lag),
  * approx_covariance equals the (mode, y, x) blocks of the dense A~ of spectrum.approx_tensor_torus and is A_0
    at d = 0,
  * many sampler draws: the averaged field_covariance reaches approx_covariance within its standard error.
"""
import numpy as np
import pytest

from oracle import sampler, spectrum, stats, zernike


def test_covariance_brute_force():
    rng = np.random.default_rng(0)
    J, H, W = 3, 5, 4
    a = rng.standard_normal((J, H, W))
    lags = [(0, 0), (1, 0), (0, 2), (-2, 1), (3, -3)]
    got = stats.field_covariance(a, lags)
    for l, (dy, dx) in enumerate(lags):
        ref = np.zeros((J, J))
        n = 0
        for y in range(H):
            for x in range(W):
                if 0 <= y + dy < H and 0 <= x + dx < W:
                    n += 1
                    for i in range(J):
                        for j in range(J):
                            ref[i, j] += a[i, y, x] * a[j, y + dy, x + dx]
        assert n == (H - abs(dy)) * (W - abs(dx))
        assert np.allclose(got[l], ref / n, rtol=1e-14, atol=1e-15)
    v = np.array([1.5, -2.0, 0.25])
    c = stats.field_covariance(np.broadcast_to(v[:, None, None], (3, 6, 7)), [(0, 0), (2, -5)])
    assert np.allclose(c, np.outer(v, v)[None], rtol=1e-15)


def test_approx_covariance_is_the_dense_tensor():
    J, N, ppd, d = 4, 8, 2.0, 2.0
    lags = [(0, 0), (1, 0), (0, 3), (-2, 1)]
    got = stats.approx_covariance(J, N, ppd, d, lags)
    lam = spectrum.lambdas(J, N, ppd)
    At = spectrum.approx_tensor_torus(lam, zernike.noll_cholesky(J, d))
    n = N * N
    for l, (dy, dx) in enumerate(lags):
        p, q = 0, (dy % N) * N + (dx % N)  # pixel (0, 0) and pixel (dy, dx)
        assert np.allclose(got[l], At[p::n, q::n], rtol=1e-12, atol=1e-14)
    assert np.allclose(got[0], zernike.noll_matrix(J, d), rtol=1e-12)


def test_sampler_covariance_reaches_a_tilde():
    J, H, W, N, ppd, d = 6, 16, 16, 32, 4.0, 1.0
    lags = [(0, 0), (0, 1), (2, 0), (3, -2)]
    per = np.stack([stats.field_covariance(sampler.sample_fields(7, f, J, H, W, d, ppd, N), lags)
                    for f in range(400)])
    mean, se = per.mean(0), per.std(0, ddof=1) / np.sqrt(per.shape[0])
    target = stats.approx_covariance(J, N, ppd, d, lags)
    assert np.all(np.abs(mean - target) <= 5 * se + 1e-12)
