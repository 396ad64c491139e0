"""Pins for the oracle's field sampler (Sec. III-A, III-C, Eq. A tilde, Fig. rand_gen).

  * operator identity: the sampler is a linear map M of the white noise, and
    M M^T must equal Eq. (A tilde) built independently from lambda and L,
  * at s = 0 every pixel has covariance A_0 exactly (Sec. III-D, observation 1),
  * statistics of many Philox-driven draws against A_0 and A tilde,
  * brute-force eigen-root sampling of the full (non-approximated) tensor on an
    8 x 8 grid with 6 modes (the worked example of Fig. rand_gen, with 6 fields).
"""
import math

import numpy as np
import pytest

from oracle import noise, sampler, spectrum, zernike

J6, N8, PPD = 6, 8, 2.0


@pytest.fixture(scope="module")
def small():
    lam = spectrum.lambdas(J6, N8, PPD)
    L = zernike.noll_cholesky(J6, 2.0)
    At = spectrum.approx_tensor_torus(lam, L)
    return lam, L, At


def test_operator_identity(small):
    lam, L, At = small
    M = sampler.operator_matrix(lam, L)
    assert np.allclose(M @ M.T, At, atol=1e-12 * np.abs(At).max())


def test_dense_root_operator_identity(small):
    lam, L, At = small
    Fr = sampler.dense_root(lam, L)
    # F F^T = L diag(lambda) L^T at every frequency
    S = np.einsum("ik,kyx,jk->yxij", L, lam, L)
    assert np.allclose(np.einsum("yxik,yxjk->yxij", Fr, Fr), S, atol=1e-12 * np.abs(S).max())
    n = J6 * N8 * N8
    M = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1
        E = np.fft.fft2(e.reshape(J6, N8, N8), axes=(1, 2))
        M[:, c] = np.real(np.fft.ifft2(np.einsum("yxij,jyx->iyx", Fr, E), axes=(1, 2))).ravel()
    assert np.allclose(M @ M.T, At, atol=1e-12 * np.abs(At).max())


@pytest.mark.parametrize("N", [8, 16])
def test_fourier_domain_noise_is_the_transform_of_white_noise(N):
    # reading R27: the Gaussian rows g -> E (Hermitian) -> e = F^-1(E) is a linear map whose output is real
    # and has identity covariance (M M^T = I), i.e. E has exactly the distribution of FFT2 of white noise
    nz = 2 * (N // 2 + 1) * N
    M = np.empty((N * N, nz))
    for c in range(nz):
        g = np.zeros(nz)
        g[c] = 1.0
        e = np.fft.ifft2(noise.hermitian_spectrum(g, N))
        assert np.abs(e.imag).max() < 1e-15
        M[:, c] = e.real.ravel()
    assert np.allclose(M @ M.T, np.eye(N * N), atol=1e-13)
    # the columns a conjugate or a self-conjugate bin ignores: (kx in {0, N/2}, ky > N/2) and the imaginary
    # parts at (kx, ky) in {0, N/2}^2
    unused = [2 * (kx * N + ky) + c for kx in (0, N // 2) for ky in range(N // 2 + 1, N) for c in (0, 1)]
    unused += [2 * (kx * N + ky) + 1 for kx in (0, N // 2) for ky in (0, N // 2)]
    assert np.all(M[:, unused] == 0.0)
    assert np.count_nonzero(np.abs(M).sum(axis=0)) == N * N


def test_zero_displacement_is_noll(small):
    lam, L, At = small
    n = N8 * N8
    A0 = zernike.noll_matrix(J6, 2.0)
    for p in (0, 9, 63):
        blk = At[p::n, p::n]
        assert np.allclose(blk, A0, rtol=1e-12, atol=1e-14)


def _wishart_ok(emp, target, nsamp, k=5.0):
    d = np.sqrt(np.diag(target))
    sd = np.sqrt((np.outer(d, d) ** 2 + target ** 2) / nsamp)
    return np.all(np.abs(emp - target) <= k * sd + 1e-15)


def test_statistics_of_philox_draws(small):
    lam, L, At = small
    nf = 3000
    seed = 11
    samples = np.empty((nf, J6 * N8 * N8))
    for f in range(nf):
        E = noise.field_spectral_noise(seed, f, J6, N8)
        samples[f] = sampler.mix(L, sampler.unit_fields_spectral(E, lam)).ravel()
    n = N8 * N8
    idx = np.array([j * n + p for j in range(J6) for p in (0, 1, 8, 27)])
    emp = samples[:, idx].T @ samples[:, idx] / nf
    assert _wishart_ok(emp, At[np.ix_(idx, idx)], nf)


def test_brute_force_full_tensor_8x8x6(small):
    lam, L, At = small
    A0 = zernike.noll_matrix(J6, 2.0)
    A = spectrum.full_tensor_torus(J6, N8, PPD, A0)
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > -1e-10 * ev.max()  # PSD (rank deficient is allowed)
    rng = np.random.default_rng(5)
    ns = 6000
    Y = sampler.eig_root_sample(A, rng.standard_normal((A.shape[0], ns)))
    n = N8 * N8
    idx = np.array([j * n + p for j in range(J6) for p in (0, 1, 9)])
    emp = Y[idx] @ Y[idx].T / ns
    assert _wishart_ok(emp, A[np.ix_(idx, idx)], ns)
    # both tensors keep the auto-variances A0_ii at s = 0 (Sec. III-D: no loss at s = 0)
    for p in (0, 33):
        assert np.allclose(np.diag(A[p::n, p::n]), np.diag(A0), rtol=1e-12)
        assert np.allclose(At[p::n, p::n], A0, rtol=1e-12, atol=1e-14)
    # the samples tell the full tensor from its approximation: on the sampled index pairs their covariance is
    # much closer to A than to A tilde, which differ in the cross-mode terms (Sec. III-D)
    dA = np.linalg.norm(emp - A[np.ix_(idx, idx)])
    dAt = np.linalg.norm(emp - At[np.ix_(idx, idx)])
    assert dA < 0.5 * dAt
    # the zero-lag block of A has Noll's sign pattern (its magnitudes carry the 8 x 8 torus's
    # low-frequency deficit; the convergence is pinned in test_oracle_spectrum)
    blk = A[0::n, 0::n]
    nz = A0 != 0.0
    assert np.all(np.sign(blk[nz]) == np.sign(A0[nz]))
    assert np.abs(blk[~nz]).max() < 3e-3 * np.abs(np.diag(A0)).max()


def test_ar1_fields_special_cases_and_field_recursion():
    # alpha = 0: independent frames; any alpha: because the sampler is linear and time-invariant the noise
    # recursion equals a_t = alpha a_{t-1} + sqrt(1 - alpha^2) s_t on the fields (the form the kernels use)
    J, H, W, N, d = 6, 8, 8, 16, 2.0
    frames0 = sampler.sample_fields_ar1(4, 3, 0.0, J, H, W, d, PPD, N)
    for t in range(3):
        assert np.array_equal(frames0[t], sampler.sample_fields(4, t, J, H, W, d, PPD, N))
    alpha = 0.7
    frames = sampler.sample_fields_ar1(4, 4, alpha, J, H, W, d, PPD, N)
    assert np.array_equal(frames[0], frames0[0])
    for t in range(1, 4):
        rec = alpha * frames[t - 1] + math.sqrt(1 - alpha ** 2) * sampler.sample_fields(4, t, J, H, W, d, PPD, N)
        assert np.allclose(frames[t], rec, atol=1e-12 * np.abs(rec).max())


def test_ar1_fields_are_stationary_with_lag_one_correlation_alpha(small):
    # many independent chains (one Philox key each): Cov(a_1, a_1) = A tilde and Cov(a_1, a_0) = alpha A tilde
    lam, L, At = small
    alpha, nc = 0.6, 1500
    n = N8 * N8
    idx = np.array([j * n + p for j in range(J6) for p in (0, 9)])
    a0 = np.empty((nc, idx.size))
    a1 = np.empty((nc, idx.size))
    for c in range(nc):
        f = sampler.sample_fields_ar1(1000 + c, 2, alpha, J6, N8, N8, 2.0, PPD, N8)
        a0[c] = f[0].ravel()[idx]
        a1[c] = f[1].ravel()[idx]
    T = At[np.ix_(idx, idx)]
    assert _wishart_ok(a1.T @ a1 / nc, T, nc)
    lag = a1.T @ a0 / nc
    d = np.sqrt(np.diag(T))
    sd = np.sqrt((np.outer(d, d) ** 2 + (alpha * T) ** 2) / nc)
    assert np.all(np.abs(lag - alpha * T) <= 5 * sd + 1e-15)
