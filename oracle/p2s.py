"""Exact phase-to-space: Zernike vector -> PSF -> weights on the PSF basis.

Test infrastructure only (see the package docstring).

Eq. (2) (PSF formation): h_x(u) = |Fourier{P(xi) exp(-j phi_x(xi))}|^2, with
the optical constants withheld by the paper; reading R11 fixes them: a 64 x 64
pupil grid with sample coordinates (i - 32)/16 (so the aperture of radius 1 is
32 samples across and the PSF is Nyquist sampled), P = 1 for rho <= 1, FFT,
centre shift, a 33 x 33 crop centred at index 32, normalised to unit sum.
Eq. (p2s PSF): h_x = sum_m beta_{x,m} varphi_m; the basis comes from a
principal component analysis of a PSF database (Sec. II-C); reading R15 takes
the uncentred SVD of the stacked PSFs.  Reading R28 takes the least-squares
projection that keeps the PSF's unit sum: among all w with sum_u (Phi^T w)(u)
= s^T w = 1 (s_k = sum_u phi_k(u)), the one nearest h,
w = Phi h + s (1 - s^T Phi h) / (s^T s).  A flat image region of brightness I
then blurs to exactly I (Eq. varying blur), as with the true PSF, whereas the
plain projection Phi h keeps only the PSF's part inside the basis span and so
changes the local brightness by 1 - s^T Phi h (R13, the plain projection, is
`weights_unconstrained`).
Tilts (Noll 2, 3) are applied by the warp (Eq. 2's linear phase shifts the
PSF), so the PSFs here use the modes Noll 4..J+1 (reading R9).
"""
from __future__ import annotations

import functools
import math
import numpy as np

from . import noise, zernike

GRID = 64
CENTER = 32
SAMPLES_PER_RADIUS = 16
KS = 33          # PSF / basis support is KS x KS
HALF = KS // 2   # 16


@functools.lru_cache(maxsize=None)
def pupil_grid():
    """rho, theta and the aperture P on the 64 x 64 pupil grid (row = y, column = x)."""
    c = (np.arange(GRID) - CENTER) / SAMPLES_PER_RADIUS
    yy, xx = np.meshgrid(c, c, indexing="ij")
    rho = np.hypot(xx, yy)
    theta = np.arctan2(yy, xx)
    P = (rho <= 1.0).astype(np.float64)
    return rho, theta, P


@functools.lru_cache(maxsize=None)
def zernike_stack(J: int) -> np.ndarray:
    """Z_j on the pupil grid for Noll j = 2..J+1, shape (J, 64, 64)."""
    rho, theta, _ = pupil_grid()
    return np.stack([zernike.zernike(j + 2, rho, theta) for j in range(J)])


def phase(a: np.ndarray, J: int, with_tilt: bool = False) -> np.ndarray:
    """phi(xi) = sum_j a_j Z_j(rho) (Eq. Zernike decompose); a has shape (..., J), field 0 = Noll 2."""
    a = np.asarray(a, dtype=np.float64)
    if not with_tilt:
        a = a.copy()
        a[..., :2] = 0.0
    return np.einsum("...j,jyx->...yx", a, zernike_stack(J))


def psf_full(a: np.ndarray, J: int, with_tilt: bool = False) -> np.ndarray:
    """|FFT2(P exp(-j phi))|^2 on the full 64 x 64 grid, centre-shifted, not normalised."""
    _, _, P = pupil_grid()
    U = P * np.exp(-1j * phase(a, J, with_tilt))
    X = np.fft.fft2(U, axes=(-2, -1))
    return np.fft.fftshift(np.abs(X) ** 2, axes=(-2, -1))


def psf(a: np.ndarray, J: int) -> np.ndarray:
    """The 33 x 33 PSF of Eq. (2) under R11: crop around the centre, unit sum."""
    h = psf_full(a, J)[..., CENTER - HALF:CENTER + HALF + 1, CENTER - HALF:CENTER + HALF + 1]
    return h / h.sum(axis=(-2, -1), keepdims=True)


def basis_draws(seed: int, J: int, n_psf: int, D_over_r0_list) -> np.ndarray:
    """Zernike vectors a ~ N(0, A_0) for the basis database (Philox tag 1, R15).

    Row i uses the Gaussians of row i of the tag-1 block (4-aligned width); the
    D/r0 values are pooled evenly: draw i uses D_over_r0_list[i % len].
    """
    cols = (J + 3) // 4 * 4
    z = noise.gaussian_block(seed, noise.TAG_BASIS, 0, 0, n_psf, cols)[:, :J].astype(np.float64)
    a = np.empty((n_psf, J))
    for t, d in enumerate(D_over_r0_list):
        L = zernike.noll_cholesky(J, d)
        idx = np.arange(t, n_psf, len(D_over_r0_list))
        a[idx] = z[idx] @ L.T
    a[:, :2] = 0.0
    return a


def svd_basis(H: np.ndarray, K: int) -> tuple[np.ndarray, np.ndarray]:
    """Top-K right singular vectors of the stacked PSFs H (n_psf x 1089), uncentred (R15).

    Sign: the entry of largest magnitude is made positive (first such index on ties).
    Returns (Phi of shape (K, 1089), all singular values).
    """
    _, s, Vt = np.linalg.svd(H, full_matrices=False)
    Phi = Vt[:K].copy()
    for k in range(K):
        i = int(np.argmax(np.abs(Phi[k])))
        if Phi[k, i] < 0:
            Phi[k] = -Phi[k]
    return Phi, s


def build_basis(seed: int, J: int, K: int, n_psf: int, D_over_r0_list) -> np.ndarray:
    """Basis Phi (K x 33 x 33) from n_psf exact PSFs (Sec. II-C)."""
    a = basis_draws(seed, J, n_psf, D_over_r0_list)
    Hm = psf(a, J).reshape(n_psf, KS * KS)
    Phi, _ = svd_basis(Hm, K)
    return Phi.reshape(K, KS, KS)


def flux_vector(basis: np.ndarray) -> np.ndarray:
    """s_k = sum_u phi_k(u): the PSF sum (flux) that weight k contributes, shape (K,)."""
    b = np.asarray(basis, dtype=np.float64)
    return b.reshape(b.shape[0], -1).sum(axis=1)


def flux_projection(w: np.ndarray, s: np.ndarray) -> np.ndarray:
    """The nearest weights (Euclidean) with s^T w = 1: w + s (1 - s^T w) / (s^T s) (reading R28)."""
    w = np.asarray(w, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    return w + (1.0 - w @ s)[..., None] * s / (s @ s)


def weights_unconstrained(a: np.ndarray, J: int, basis: np.ndarray) -> np.ndarray:
    """The plain orthogonal projection Phi^T h of the PSFs of Zernike vectors a (..., J) (R13)."""
    K = basis.shape[0]
    h = psf(a, J).reshape(*np.shape(a)[:-1], KS * KS)
    return h @ basis.reshape(K, KS * KS).T


def weights(a: np.ndarray, J: int, basis: np.ndarray) -> np.ndarray:
    """The exact P2S weights (reading R28), shape (..., K): the least-squares projection of the unit-sum PSF
    on the basis under the constraint that the projected PSF keeps the unit sum."""
    return flux_projection(weights_unconstrained(a, J, basis), flux_vector(basis))


def weights_field(fields: np.ndarray, basis: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """Exact P2S weights for a J x H x W field stack, shape (H, W, K)."""
    J, H, W = fields.shape
    a = np.moveaxis(fields, 0, -1).reshape(H * W, J)
    out = np.empty((H * W, basis.shape[0]))
    for s in range(0, H * W, chunk):
        out[s:s + chunk] = weights(a[s:s + chunk], J, basis)
    return out.reshape(H, W, -1)
