"""Image formation: tilt warp and the basis blur.

Test infrastructure only (see the package docstring).

Eq. (1): I(x) = h_x(u) (*) I_g(u), keeping only the centre pixel of each
convolution.  Eq. (varying blur): with h_x = sum_m beta_{x,m} varphi_m,
I(x) = sum_m beta_{x,m} (varphi_m (*) I_g)(x).  The tilt part of the phase
(Noll 2, 3) only shifts the PSF (Eq. 2 with a linear phase), so it is applied as
a warp before the blur (reading R10): a_2 moves the PSF peak to
u = -(4/pi) a_2 columns, i.e. the image is sampled at x + (4/pi) a_2.
"""
from __future__ import annotations

import math
import numpy as np
from scipy.signal import fftconvolve

TILT_PIX = 4.0 / math.pi
HALF = 16


def tilt_warp(img: np.ndarray, a2: np.ndarray, a3: np.ndarray) -> np.ndarray:
    """Bilinear resampling of img (C x H x W) at (x + (4/pi) a2, y + (4/pi) a3), clamp to edge."""
    img = np.asarray(img, dtype=np.float64)
    C, H, W = img.shape
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    sx = xx + TILT_PIX * np.asarray(a2, dtype=np.float64)
    sy = yy + TILT_PIX * np.asarray(a3, dtype=np.float64)
    x0 = np.floor(sx)
    y0 = np.floor(sy)
    tx = sx - x0
    ty = sy - y0
    x0 = x0.astype(np.int64)
    y0 = y0.astype(np.int64)
    xa = np.clip(x0, 0, W - 1)
    xb = np.clip(x0 + 1, 0, W - 1)
    ya = np.clip(y0, 0, H - 1)
    yb = np.clip(y0 + 1, 0, H - 1)
    out = np.empty_like(img)
    for c in range(C):
        I = img[c]
        out[c] = ((1 - ty) * ((1 - tx) * I[ya, xa] + tx * I[ya, xb])
                  + ty * ((1 - tx) * I[yb, xa] + tx * I[yb, xb]))
    return out


def basis_convolutions(img: np.ndarray, basis: np.ndarray) -> np.ndarray:
    """(varphi_k (*) I_c)(x), true convolution with clamp-to-edge borders (R16); shape (C, K, H, W)."""
    img = np.asarray(img, dtype=np.float64)
    C, H, W = img.shape
    K = basis.shape[0]
    out = np.empty((C, K, H, W))
    for c in range(C):
        padded = np.pad(img[c], HALF, mode="edge")
        for k in range(K):
            out[c, k] = fftconvolve(padded, np.asarray(basis[k], dtype=np.float64), mode="valid")
    return out


def basis_blur(img: np.ndarray, w: np.ndarray, basis: np.ndarray) -> np.ndarray:
    """out_c(x) = sum_k w_k(x) (varphi_k (*) I_c)(x)  (Eq. varying blur); w has shape (H, W, K)."""
    conv = basis_convolutions(img, basis)
    return np.einsum("ckyx,yxk->cyx", conv, np.asarray(w, dtype=np.float64))


def direct_blur(img: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Eq. (1) directly: out_c(x) = sum_u h_x(u) I_c(x - u), h of shape (H, W, 33, 33), clamp-to-edge."""
    img = np.asarray(img, dtype=np.float64)
    C, H, W = img.shape
    out = np.zeros((C, H, W))
    ys = np.arange(H)
    xs = np.arange(W)
    for iu in range(2 * HALF + 1):
        uy = iu - HALF
        yi = np.clip(ys - uy, 0, H - 1)
        for ju in range(2 * HALF + 1):
            ux = ju - HALF
            xi = np.clip(xs - ux, 0, W - 1)
            out += h[None, :, :, iu, ju] * img[:, yi][:, :, xi]
    return out
