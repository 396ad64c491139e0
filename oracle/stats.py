"""Lagged covariances of Zernike coefficient fields and their expectation.

Test infrastructure only (see the package docstring).

Sec. III-D judges the sampler by the covariance of the sampled fields: at
separation s it is A~(s) of Eq. (A tilde) (L blockdiag(rho_j) L^T with the
unit-variance autocorrelations rho_j of Sec. III-C step 1), and at s = 0 the
Noll matrix A_0 (observation 1 of Sec. III-D).
"""
from __future__ import annotations

import numpy as np

from . import spectrum, zernike


def field_covariance(a: np.ndarray, lags) -> np.ndarray:
    """out[l][i][j] = mean over pixels x with x + d_l inside the frame of a_i(x) a_j(x + d_l),
    d_l = (dy, dx), for J x H x W fields a; FP64."""
    a = np.asarray(a, dtype=np.float64)
    J, H, W = a.shape
    out = np.empty((len(lags), J, J))
    for l, (dy, dx) in enumerate(lags):
        y0, y1 = max(0, -dy), min(H, H - dy)
        x0, x1 = max(0, -dx), min(W, W - dx)
        u = a[:, y0:y1, x0:x1].reshape(J, -1)
        v = a[:, y0 + dy:y1 + dy, x0 + dx:x1 + dx].reshape(J, -1)
        out[l] = u @ v.T / u.shape[1]
    return out


def approx_covariance(J: int, N: int, pix_per_D: float, D_over_r0: float, lags) -> np.ndarray:
    """A~(d) of Eq. (A tilde) at the lags d = (dy, dx): L diag(rho_1(d) .. rho_J(d)) L^T, rho_j the inverse
    transform of lambda_j on the N x N torus (unit at d = 0, R2/R5) and L the Cholesky factor of A_0(D/r0):
    the expectation of field_covariance for the sampler's fields."""
    lam = spectrum.lambdas(J, N, pix_per_D)
    rho = np.real(np.fft.ifft2(lam, axes=(1, 2)))
    L = zernike.noll_cholesky(J, D_over_r0)
    return np.stack([(L * rho[:, dy % N, dx % N][None, :]) @ L.T for dy, dx in lags])
