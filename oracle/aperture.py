"""Aperture and spatial statistics of sampled Zernike fields (Sec. IV-B).

Test infrastructure only (see the package docstring).

Every pixel x of a frame carries a Zernike vector a(x) (all J fields, Noll
2..J+1); its phase over the pupil is phi = sum_j a_j Z_j (Eq. Zernike
decompose) on the 64 x 64 pupil grid of reading R11 (coordinates (i - 32)/16,
aperture P = 1 for rho <= 1).  Reading R30 takes the pixels of a sub-grid
(rows and columns 0, step, 2 step, ...) as the realisations the paper's
statistics average over.

Aperture statistics (Sec. IV-B):
  structure function  D(delta) = mean over realisations and over the pairs of
                      aperture samples (i, k), (i, k + delta) (along x; along
                      y likewise) of (phi(i, k) - phi(i, k + delta))^2, to be
                      compared with 6.88 (r / r0)^{5/3} (Eq. fried_struct) at
                      r = delta / 32 aperture diameters;
  LE OTF              Eq. (H_LE): the mean over realisations of the
                      autocorrelation of P e^{-j phi}; by linearity the inverse
                      transform of the mean PSF |F(P e^{-j phi})|^2, normalised
                      to 1 at zero frequency, real part; nu on the 64 x 64 grid
                      in FFT order (nu / 32 aperture diameters);
  SE OTF              Eq. (H_SE): the same with phi - (c0 + c1 x + c2 y), the
                      least-squares plane over the aperture samples removed
                      (the constant does not change |F|^2).
Spatial statistics (Sec. IV-B): the tilt correlation E[alpha(0) alpha(d)] and
the differential tilt variance E[(alpha(0) - alpha(d))^2] of the two tilt
fields at pixel lags d along x and y, each a mean over the pixel pairs inside
the frame; the identity DTV = 2 (E[alpha^2] - E[alpha(0) alpha(d)]) of the
paper holds for the window means as DTV = var(x) + var(x + d) - 2 corr.
"""
from __future__ import annotations

import functools

import numpy as np

from . import p2s

GRID = p2s.GRID
SF_LAGS = 33  # delta = 0 .. 32: the aperture is 33 samples across


@functools.lru_cache(maxsize=None)
def _aperture():
    rho, theta, P = p2s.pupil_grid()
    c = (np.arange(GRID) - p2s.CENTER) / p2s.SAMPLES_PER_RADIUS
    yy, xx = np.meshgrid(c, c, indexing="ij")
    return P, xx, yy


def realisations(fields: np.ndarray, step: int) -> np.ndarray:
    """The Zernike vectors of the sub-grid pixels, shape (n, J) (reading R30)."""
    f = np.asarray(fields, dtype=np.float64)[:, ::step, ::step]
    return f.reshape(f.shape[0], -1).T


def phases(avec: np.ndarray) -> np.ndarray:
    """phi on the 64 x 64 pupil grid for each vector (n, 64, 64); tilts included."""
    J = avec.shape[1]
    return p2s.phase(avec, J, with_tilt=True)


def remove_plane(phi: np.ndarray) -> np.ndarray:
    """phi minus its least-squares plane c0 + c1 x + c2 y over the aperture samples (zero outside)."""
    P, xx, yy = _aperture()
    m = P > 0
    X = np.stack([np.ones(m.sum()), xx[m], yy[m]], axis=1)
    vals = phi[:, m]                                  # (n, NA)
    coef, *_ = np.linalg.lstsq(X, vals.T, rcond=None)  # (3, n)
    out = np.zeros_like(phi)
    out[:, m] = vals - (X @ coef).T
    return out


def structure_function(phi: np.ndarray):
    """(D_x, D_y), each of length SF_LAGS (D(0) = 0): mean squared phase differences over aperture pairs."""
    P, _, _ = _aperture()
    Dx, Dy = np.zeros(SF_LAGS), np.zeros(SF_LAGS)
    for d in range(1, SF_LAGS):
        mx = (P[:, :-d] > 0) & (P[:, d:] > 0)
        my = (P[:-d, :] > 0) & (P[d:, :] > 0)
        Dx[d] = np.mean((phi[:, :, :-d] - phi[:, :, d:])[:, mx] ** 2)
        Dy[d] = np.mean((phi[:, :-d, :] - phi[:, d:, :])[:, my] ** 2)
    return Dx, Dy


def otf(phi: np.ndarray) -> np.ndarray:
    """Re of the inverse transform of the mean |F(P e^{-j phi})|^2, normalised to 1 at nu = 0 (64 x 64, FFT order)."""
    P, _, _ = _aperture()
    U = P * np.exp(-1j * phi)
    psf = np.mean(np.abs(np.fft.fft2(U, axes=(-2, -1))) ** 2, axis=0)
    H = np.fft.ifft2(psf)
    return np.real(H) / np.real(H[0, 0])


def aperture_statistics(fields: np.ndarray, step: int):
    """(D_x, D_y, H_LE, H_SE) of the sub-grid realisations of J x H x W fields."""
    phi = phases(realisations(fields, step))
    Dx, Dy = structure_function(phi)
    return Dx, Dy, otf(phi), otf(remove_plane(phi))


# ----------------------------------------------------------------- expectations for Gaussian vectors a ~ N(0, A)
def _zernike_grid(J: int) -> np.ndarray:
    return p2s.zernike_stack(J)  # (J, 64, 64), zero outside the aperture


def expected_structure_function(A: np.ndarray):
    """E[D_x], E[D_y] for a ~ N(0, A): the mean over aperture pairs of dZ^T A dZ."""
    J = A.shape[0]
    Z = _zernike_grid(J)
    P, _, _ = _aperture()
    Dx, Dy = np.zeros(SF_LAGS), np.zeros(SF_LAGS)
    for d in range(1, SF_LAGS):
        mx = (P[:, :-d] > 0) & (P[:, d:] > 0)
        my = (P[:-d, :] > 0) & (P[d:, :] > 0)
        dzx = (Z[:, :, :-d] - Z[:, :, d:])[:, mx]
        dzy = (Z[:, :-d, :] - Z[:, d:, :])[:, my]
        Dx[d] = np.mean(np.einsum("ip,ij,jp->p", dzx, A, dzx))
        Dy[d] = np.mean(np.einsum("ip,ij,jp->p", dzy, A, dzy))
    return Dx, Dy


def expected_otf(A: np.ndarray, tilt_removed: bool = False, nus=None) -> np.ndarray:
    """E[H](nu) for a ~ N(0, A): sum_rho P(rho) P(rho + nu) exp(-dZ^T A dZ / 2) / sum P, the shift circular on the
    64 grid (the DFT's autocorrelation); with tilt_removed, Z_j minus its least-squares plane over the aperture.
    nus: optional list of (nu_y, nu_x) to evaluate (the rest stay 0)."""
    J = A.shape[0]
    Z = _zernike_grid(J)
    if tilt_removed:
        Z = remove_plane(Z)
    P, _, _ = _aperture()
    H = np.zeros((GRID, GRID))
    todo = nus if nus is not None else [(vy, vx) for vy in range(GRID) for vx in range(GRID)]
    for vy, vx in todo:
        Ps = np.roll(P, (-vy, -vx), axis=(0, 1))  # P(rho + nu)
        m = (P > 0) & (Ps > 0)
        if not m.any():
            continue
        dz = (np.roll(Z, (-vy, -vx), axis=(1, 2)) - Z)[:, m]
        H[vy, vx] = np.sum(np.exp(-0.5 * np.einsum("ip,ij,jp->p", dz, A, dz)))
    return H / P.sum()


def diffraction_otf_analytic(nu_over_D: np.ndarray) -> np.ndarray:
    """The circular aperture's OTF (2/pi)(acos v - v sqrt(1 - v^2)), v = |nu| / D <= 1."""
    v = np.clip(np.asarray(nu_over_D, dtype=np.float64), 0.0, 1.0)
    return (2 / np.pi) * (np.arccos(v) - v * np.sqrt(1 - v * v))


# ----------------------------------------------------------------- spatial statistics
def tilt_statistics(fields: np.ndarray, max_lag: int) -> np.ndarray:
    """out[dir][lag] = (corr_x, corr_y, dtv_x, dtv_y, var0_x, var1_x, var0_y, var1_y) for dir 0 (lag along x) and
    1 (along y), lag = 0 .. max_lag; x = field 0 (Noll 2), y = field 1 (Noll 3); means over the pixel pairs
    (p, p + d) inside the frame: corr = mean a(p) a(p+d), dtv = mean (a(p) - a(p+d))^2, var0 = mean a(p)^2,
    var1 = mean a(p+d)^2."""
    a = np.asarray(fields, dtype=np.float64)[:2]
    _, H, W = a.shape
    out = np.zeros((2, max_lag + 1, 8))
    for direction in (0, 1):
        for d in range(max_lag + 1):
            if direction == 0:
                u, v = a[:, :, : W - d], a[:, :, d:]
            else:
                u, v = a[:, : H - d, :], a[:, d:, :]
            u = u.reshape(2, -1)
            v = v.reshape(2, -1)
            corr = (u * v).mean(axis=1)
            dtv = ((u - v) ** 2).mean(axis=1)
            v0 = (u * u).mean(axis=1)
            v1 = (v * v).mean(axis=1)
            out[direction, d] = [corr[0], corr[1], dtv[0], dtv[1], v0[0], v1[0], v0[1], v1[1]]
    return out
