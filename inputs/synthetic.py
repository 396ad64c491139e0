"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This module holds no arithmetic of the simulation method itself: it only makes
clean images (the "distortion-free image" I_g of Eq. 1) and random arrays.
The paper measures on a heat-chamber data set that is not available; these
images stand in for it, with the sizes of the workloads:

  smooth_noise   64 x 64 x 1: uniform [0, 1] noise smoothed by a normalised
                 Gaussian (sigma 2, radius 6, edge clamp)
  blobs          256 x 256 x 3: 50 Gaussian blobs (centres uniform, sigma in
                 [3, 30] px, per-channel amplitude in [0, 1]) + 0.05 U[0, 1]
  shapes         512 x 512 x 3: background 0.5, 30 axis-aligned rectangles of
                 random colour, 10 step edges at random angles and contrasts
  texture        3840 x 2160 x 3: white Gaussian noise shaped to a 1/f^2 power
                 spectrum (amplitude 1 / max(|f|, 1/4096)), min-max scaled
All images are float32, planar C x H x W, values in [0, 1].
"""
from __future__ import annotations

import numpy as np


def _gauss_kernel(sigma: float, radius: int) -> np.ndarray:
    x = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    return k / k.sum()


def _sep_filter_clamp(img: np.ndarray, k: np.ndarray) -> np.ndarray:
    r = (len(k) - 1) // 2
    H, W = img.shape
    p = np.pad(img, r, mode="edge")
    tmp = np.zeros((H + 2 * r, W))
    for i, c in enumerate(k):
        tmp += c * p[:, i:i + W]
    out = np.zeros((H, W))
    for i, c in enumerate(k):
        out += c * tmp[i:i + H, :]
    return out


def smooth_noise(H: int = 64, W: int = 64, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    img = rng.random((H, W))
    img = _sep_filter_clamp(img, _gauss_kernel(2.0, 6))
    return img[None].astype(np.float32)


def blobs(H: int = 256, W: int = 256, C: int = 3, n: int = 50, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    img = np.zeros((C, H, W))
    for _ in range(n):
        cy, cx = rng.random() * H, rng.random() * W
        s = 3.0 + 27.0 * rng.random()
        amp = rng.random(C)
        g = np.exp(-0.5 * ((yy - cy) ** 2 + (xx - cx) ** 2) / s ** 2)
        img += amp[:, None, None] * g[None]
    img += 0.05 * rng.random((C, H, W))
    img /= max(img.max(), 1e-12)
    return img.astype(np.float32)


def shapes(H: int = 512, W: int = 512, C: int = 3, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    img = np.full((C, H, W), 0.5)
    for _ in range(30):
        y0, x0 = rng.integers(0, H), rng.integers(0, W)
        h, w = rng.integers(4, max(5, H // 4)), rng.integers(4, max(5, W // 4))
        img[:, y0:y0 + h, x0:x0 + w] = rng.random(C)[:, None, None]
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    for _ in range(10):
        ang = rng.random() * 2 * np.pi
        cy, cx = rng.random() * H, rng.random() * W
        side = (np.cos(ang) * (xx - cx) + np.sin(ang) * (yy - cy)) > 0
        contrast = (rng.random(C) - 0.5) * 0.4
        img += side[None] * contrast[:, None, None]
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def texture(H: int = 2160, W: int = 3840, C: int = 3, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.rfftfreq(W)[None, :]
    amp = 1.0 / np.maximum(np.hypot(fx, fy), 1.0 / 4096.0)
    out = np.empty((C, H, W), dtype=np.float32)
    for c in range(C):
        n = rng.standard_normal((H, W))
        t = np.fft.irfft2(np.fft.rfft2(n) * amp, s=(H, W))
        t = (t - t.min()) / (t.max() - t.min())
        out[c] = t.astype(np.float32)
    return out


def image_for(kind: str, H: int, W: int, C: int, seed: int = 0) -> np.ndarray:
    if kind == "smooth_noise":
        return np.repeat(smooth_noise(H, W, seed), C, axis=0)
    if kind == "blobs":
        return blobs(H, W, C, seed=seed)
    if kind == "shapes":
        return shapes(H, W, C, seed=seed)
    if kind == "texture":
        return texture(H, W, C, seed=seed)
    raise ValueError(kind)


def random_fields(J: int, H: int, W: int, scale: float = 0.3, seed: int = 0) -> np.ndarray:
    """Plain Gaussian arrays shaped like Zernike fields (for stage-level tests)."""
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal((J, H, W))).astype(np.float32)


def random_orthonormal_rows(K: int, n: int, seed: int = 0) -> np.ndarray:
    """K orthonormal rows of length n (a stand-in PSF basis for stage-level tests)."""
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, K)))
    return q.T.astype(np.float64)
