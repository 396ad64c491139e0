"""Random Zernike fields: the FFT sampler of Sec. III-A/III-C and its checks.

Test infrastructure only (see the package docstring).

Sec. III-A: for a homogeneous (circulant) covariance, y = F^{-1}(S^{1/2} F(e)).
The sampler draws F(e) directly as Hermitian Fourier-domain white noise
(reading R27 in noise.py), which has the same distribution.
Sec. III-C: step 1 draws N unit-variance fields, each from its own
autocovariance A_{i,i} with that Fourier method; step 2 mixes them pixel by
pixel with the Noll matrix through L L^T = A_0 (Cholesky, Fig. rand_gen), so
the covariance of the result is Eq. (A tilde) = L blockdiag(A_ii) L^T.
"""
from __future__ import annotations

import numpy as np

from . import noise, spectrum, zernike


def grid_size(H: int, W: int, pix_per_D: float = 8.0) -> int:
    """N = next power of two >= max(H, W) + 4 pix_per_D (reading R4)."""
    need = max(H, W) + int(np.ceil(4 * pix_per_D))
    N = 1
    while N < need:
        N *= 2
    return N


def unit_fields(e: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Step 1 of Sec. III-C: a~_j = Re IFFT2(sqrt(lambda_j) FFT2(e_j)), FP64, full N x N torus."""
    e = np.asarray(e, dtype=np.float64)
    return np.real(np.fft.ifft2(np.sqrt(lam) * np.fft.fft2(e, axes=(-2, -1)), axes=(-2, -1)))


def unit_fields_spectral(E: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Step 1 of Sec. III-C from Fourier-domain noise: a~_j = Re IFFT2(sqrt(lambda_j) E_j), FP64, full torus."""
    return np.real(np.fft.ifft2(np.sqrt(lam) * E, axes=(-2, -1)))


def mix(L: np.ndarray, fields: np.ndarray) -> np.ndarray:
    """Step 2 of Sec. III-C: a(x) = L a~(x) at every pixel."""
    return np.einsum("ij,jyx->iyx", L, fields)


def sample_fields(seed: int, frame: int, J: int, H: int, W: int, D_over_r0: float,
                  pix_per_D: float = 8.0, N: int | None = None) -> np.ndarray:
    """The J x H x W Zernike fields of one frame (factored form, the paper's method)."""
    if N is None:
        N = grid_size(H, W, pix_per_D)
    E = noise.field_spectral_noise(seed, frame, J, N)
    lam = spectrum.lambdas(J, N, pix_per_D)
    a_unit = unit_fields_spectral(E, lam)[:, :H, :W]
    return mix(zernike.noll_cholesky(J, D_over_r0), a_unit)


def sample_fields_ar1(seed: int, frames: int, alpha: float, J: int, H: int, W: int, D_over_r0: float,
                      pix_per_D: float = 8.0, N: int | None = None) -> list[np.ndarray]:
    """Temporally correlated fields (Sec. III, spatio-temporally correlated fields; reading R26).

    The paper enforces temporal correlation by an auto-regressive process; here the white noise of every
    mode and torus position follows e_0 = n_0, e_t = alpha e_{t-1} + sqrt(1 - alpha^2) n_t, n_t the noise
    of frame t, and each frame's fields are the FFT sampler applied to e_t.  The recursion is taken on the
    Fourier-domain noise (R27), which is the same linear recursion on F(e).  Returns frames 0..frames-1.
    """
    if N is None:
        N = grid_size(H, W, pix_per_D)
    lam = spectrum.lambdas(J, N, pix_per_D)
    L = zernike.noll_cholesky(J, D_over_r0)
    beta = np.sqrt(1.0 - alpha * alpha)
    out, e = [], None
    for t in range(frames):
        n = noise.field_spectral_noise(seed, t, J, N)
        e = n if e is None else alpha * e + beta * n
        out.append(mix(L, unit_fields_spectral(e, lam)[:, :H, :W]))
    return out


def dense_root(lam: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Per-frequency symmetric square root F(f) of S~(f) = L diag(lambda(f)) L^T, shape (N, N, J, J).

    Eigen-decomposition per frequency; negative eigenvalues (rounding of a
    near-singular matrix) are clamped to zero before the square root.
    """
    J, N, _ = lam.shape
    lt = np.moveaxis(lam, 0, -1)  # (N, N, J)
    S = np.einsum("ik,yxk,jk->yxij", L, lt, L)
    ev, U = np.linalg.eigh(S)
    ev = np.sqrt(np.clip(ev, 0.0, None))
    return np.einsum("yxik,yxk,yxjk->yxij", U, ev, U)


def sample_fields_dense(seed: int, frame: int, J: int, H: int, W: int, D_over_r0: float,
                        pix_per_D: float = 8.0, N: int | None = None) -> np.ndarray:
    """Fields from the per-frequency J x J symmetric root: a = Re IFFT2(F(f) E), E the Fourier-domain noise, cropped.

    Same covariance as sample_fields, different samples (reading R6).
    """
    if N is None:
        N = grid_size(H, W, pix_per_D)
    E = noise.field_spectral_noise(seed, frame, J, N)
    lam = spectrum.lambdas(J, N, pix_per_D)
    Fr = dense_root(lam, zernike.noll_cholesky(J, D_over_r0))
    Y = np.einsum("yxij,jyx->iyx", Fr, E)
    return np.real(np.fft.ifft2(Y, axes=(1, 2)))[:, :H, :W]


def operator_matrix(lam: np.ndarray, L: np.ndarray) -> np.ndarray:
    """The sampler as a dense linear map M (white noise -> mixed fields) on the full torus.

    Columns are the sampler applied to unit vectors; order (mode, y, x).
    """
    J, N, _ = lam.shape
    n = J * N * N
    M = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        M[:, c] = mix(L, unit_fields(e.reshape(J, N, N), lam)).ravel()
    return M


def eig_root_sample(A: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Sec. III-A brute force: y = U S^{1/2} U^T z with A = U S U^T (S clamped at 0).

    A may be rank deficient, so the eigen-root is used instead of Cholesky.
    z has shape (dim, n_samples).
    """
    ev, U = np.linalg.eigh(A)
    root = (U * np.sqrt(np.clip(ev, 0.0, None))) @ U.T
    return root @ z
