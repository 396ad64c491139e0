"""Subharmonic low-frequency compensation of the FFT field sampler (Sec. IV-B; reading R31).

Test infrastructure only (see the package docstring).

Sec. IV-B notes that the remaining deviations of the simulated statistics may
be improved by subharmonic methods (the paper points to Schmidt's text).  The
FFT sampler on the N x N torus represents the spectrum by point samples at
f_k = k df, df = pix_per_D / N, and sets the DC bin to zero (R5); the cell
|fx|, |fy| < df/2 around DC is missing.  For the tilt modes the path-integrated
spectrum (R1) grows like f^{-5/3} towards DC, so that cell holds a large share
of their power (about 30 % at N = 1024), and the unit-variance normalisation
(R2) hands it to higher frequencies: the tilt correlation decays too fast.

Reading R31 (the subharmonic sampler).  The DC cell is divided into 3 x 3
sub-cells of side df/3; the eight outer ones are represented by their centres
f = (n, m) df / 3 (n, m in {-1, 0, 1}, not both 0), each with weight (df/3)^2;
the centre sub-cell is divided again, for levels p = 1 .. P, side df / 3^p.
In units of the torus bins (weight df^2) a level-p frequency carries
P_j(f) / 9^p.  The unit-variance normalisation covers both parts:
  Z_j = sum_{k != 0} P_j(f_k) + sum_{p, d} P_j(f_{p,d}) / 9^p,
  lambda_j(k) = N^2 P_j(f_k) / Z_j,   s_{j,p,d}^2 = P_j(f_{p,d}) / 9^p / Z_j,
(G at the subharmonic frequencies, down to df / 3^12, from the v-rule that reaches
v = 1e-14), and the unit field is the FFT part plus
  sum_{p, d} Re[(g_re + i g_im) s_{j,p,d} e^{2 pi i (n_d x + m_d y) / (N 3^p)}]
at pixel (y, x), (g_re, g_im) unit Gaussians: each term adds s^2 to the
variance, so the field keeps variance 1 exactly.  The eight directions d are
taken in the order (n, m) = (-1,-1), (0,-1), (1,-1), (-1,0), (1,0), (-1,1),
(0,1), (1,1); their Gaussians come from Philox tag 6, subsequence mode j,
counter 4 (p - 1) + k for directions 2k and 2k + 1 (four Gaussians: Re, Im of
each).  The mixing by L follows as in Sec. III-C.  The sub-cells at f and -f
carry independent amplitudes, as in the FFT part's two half planes.
"""
from __future__ import annotations

import numpy as np

from . import noise, spectrum, zernike

TAG_SUBHARMONICS = 6
DIRECTIONS = ((-1, -1), (0, -1), (1, -1), (-1, 0), (1, 0), (-1, 1), (0, 1), (1, 1))


def subharmonic_frequencies(N: int, pix_per_D: float, levels: int):
    """(|f|, phi) of the level-p direction-d frequencies, shape (levels, 8); f in cycles per unit s."""
    df = pix_per_D / N
    fmag = np.empty((levels, 8))
    phi = np.empty((levels, 8))
    for p in range(1, levels + 1):
        for d, (n, m) in enumerate(DIRECTIONS):
            fx, fy = n * df / 3 ** p, m * df / 3 ** p
            fmag[p - 1, d] = np.hypot(fx, fy)
            phi[p - 1, d] = np.arctan2(fy, fx)
    return fmag, phi


def mode_subharmonic_power(j: int, N: int, pix_per_D: float, levels: int) -> np.ndarray:
    """P_j(f_{p,d}) / 9^p, shape (levels, 8), in the units of mode_spectrum_shape's bins."""
    n, _ = zernike.noll_nm(j)
    fmag, phi = subharmonic_frequencies(N, pix_per_D, levels)
    G = spectrum.radial_spectra([(n, n)], fmag.ravel(), deep=True)[0].reshape(fmag.shape)
    w = 9.0 ** -np.arange(1, levels + 1)
    return (n + 1) * spectrum.angular_factor(j, phi) * G * w[:, None]


def lambdas_and_amplitudes(J: int, N: int, pix_per_D: float, levels: int):
    """lambda (J, N, N) and the subharmonic amplitudes s (J, levels, 8), normalised together to unit variance."""
    lam = np.empty((J, N, N))
    s = np.empty((J, levels, 8))
    for j in range(J):
        P = spectrum.mode_spectrum_shape(j + 2, N, pix_per_D)
        Psh = mode_subharmonic_power(j + 2, N, pix_per_D, levels)
        Z = P.sum() + Psh.sum()
        lam[j] = N * N * P / Z
        s[j] = np.sqrt(Psh / Z)
    return lam, s


def subharmonic_gaussians(seed: int, frame: int, J: int, levels: int) -> np.ndarray:
    """(g_re + i g_im) per mode, level and direction, shape (J, levels, 8) complex (Philox tag 6)."""
    out = np.empty((J, levels, 8), dtype=np.complex128)
    q = np.arange(4 * levels, dtype=np.uint64)
    for j in range(J):
        w0, w1, w2, w3 = noise.philox_words(seed, noise.subsequence(TAG_SUBHARMONICS, frame, j), q)
        a, b = noise.box_muller(w0, w1)
        c, d = noise.box_muller(w2, w3)
        g = np.stack([a, b, c, d], axis=-1).astype(np.float64).reshape(levels, 4, 4)  # [p][k][Re0, Im0, Re1, Im1]
        out[j, :, 0::2] = g[:, :, 0] + 1j * g[:, :, 1]
        out[j, :, 1::2] = g[:, :, 2] + 1j * g[:, :, 3]
    return out


def subharmonic_part(c: np.ndarray, N: int, H: int, W: int) -> np.ndarray:
    """sum_{p,d} Re[c_{j,p,d} e^{2 pi i (n x + m y)/(N 3^p)}] on the H x W frame, shape (J, H, W)."""
    J, levels, _ = c.shape
    y = np.arange(H)[:, None]
    x = np.arange(W)[None, :]
    out = np.zeros((J, H, W))
    for p in range(1, levels + 1):
        for d, (n, m) in enumerate(DIRECTIONS):
            e = np.exp(2j * np.pi * (n * x + m * y) / (N * 3 ** p))
            out += np.real(c[:, p - 1, d][:, None, None] * e[None])
    return out


def sample_fields(seed: int, frame: int, J: int, H: int, W: int, D_over_r0: float, levels: int,
                  pix_per_D: float = 8.0, N: int | None = None) -> np.ndarray:
    """The factored sampler (Sec. III-C) with `levels` subharmonic levels (R31), J x H x W FP64."""
    from . import sampler
    if N is None:
        N = sampler.grid_size(H, W, pix_per_D)
    lam, s = lambdas_and_amplitudes(J, N, pix_per_D, levels)
    E = noise.field_spectral_noise(seed, frame, J, N)
    unit = sampler.unit_fields_spectral(E, lam)[:, :H, :W]
    unit = unit + subharmonic_part(s * subharmonic_gaussians(seed, frame, J, levels), N, H, W)
    return sampler.mix(zernike.noll_cholesky(J, D_over_r0), unit)


def unit_autocorrelation(lam_j: np.ndarray, s_j: np.ndarray, dy: int, dx: int) -> float:
    """E[u(y, x) u(y + dy, x + dx)] of one unit field: the FFT part's inverse transform plus
    sum s^2 cos(2 pi (n dx + m dy) / (N 3^p))."""
    N = lam_j.shape[0]
    r = float(np.real(np.fft.ifft2(lam_j))[dy % N, dx % N])
    for p in range(1, s_j.shape[0] + 1):
        for d, (n, m) in enumerate(DIRECTIONS):
            r += s_j[p - 1, d] ** 2 * np.cos(2 * np.pi * (n * dx + m * dy) / (N * 3 ** p))
    return r
