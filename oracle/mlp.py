"""The P2S surrogate network in FP64: forward, backward, Adam.

Test infrastructure only (see the package docstring).

Sec. II-C: the paper (after Mao et al. 2021) maps each pixel's Zernike vector
a_x to the basis coefficients beta_x with a small neural network.  The
network's shape and training are not given (reading R18): J -> 256 -> 256 -> K
with the erf form of GELU, trained with Adam (Kingma & Ba 2015) on per-k
standardised weights, with the loss of reading R25: the expected squared error
that a weight error causes in the blurred image under a 1/(|f|^2 + 1) image
spectrum (`image_prior_gram`); the flat spectrum gives the squared error of
the PSF, and lw = 1 the plain mean squared error.  Input features are
x = a * in_scale (in_scale is 0 on the two tilt fields, reading R9); the output
is w = y * out_scale + out_shift.
"""
from __future__ import annotations

import math
import numpy as np
from scipy.special import erf

SQRT1_2 = 1.0 / math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z * SQRT1_2))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z * SQRT1_2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def forward(params: dict, x: np.ndarray):
    """Returns (y, cache); params W1 (256 x J), b1, W2 (256 x 256), b2, W3 (K x 256), b3."""
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ params["W1"].T + params["b1"]
    h1 = gelu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = gelu(z2)
    y = h2 @ params["W3"].T + params["b3"]
    return y, (x, z1, h1, z2, h2)


def image_prior_gram(basis: np.ndarray, sd: np.ndarray, M: int = 64, flat: bool = False) -> np.ndarray:
    """Quadratic form of the training loss, reading R25.

    A weight error dw at a pixel changes the blurred image (Eq. varying blur) by
    e = sum_k dw_k (phi_k (*) I).  For images with power spectrum S(f) its expected
    energy is dw^T G dw, G_kl = sum_f S(f) Re(Phi_k(f) conj Phi_l(f)), Phi_k the DFT
    of phi_k (33 x 33, placed at the origin of an M x M torus), S(f) =
    1 / (fx^2 + fy^2 + 1) with integer frequencies (or S = 1 if `flat`).  In the
    network's standardised outputs dw = diag(sd) r, so the loss matrix is
    G^ = diag(sd) G diag(sd), scaled to a unit mean diagonal.
    """
    b = np.asarray(basis, dtype=np.float64)
    K = b.shape[0]
    pad = np.zeros((K, M, M))
    pad[:, :b.shape[1], :b.shape[2]] = b
    F = np.fft.fft2(pad).reshape(K, -1)
    f = np.fft.fftfreq(M) * M
    S = np.ones((M, M)) if flat else 1.0 / (f[:, None] ** 2 + f[None, :] ** 2 + 1.0)
    G = np.real((F * S.reshape(1, -1)) @ F.conj().T)
    D = np.asarray(sd, dtype=np.float64)
    Gh = D[:, None] * G * D[None, :]
    return Gh / np.mean(np.diag(Gh))


def loss_and_grads(params: dict, x: np.ndarray, t: np.ndarray, lw: np.ndarray | None = None,
                   G: np.ndarray | None = None):
    """Training loss over the B x K outputs and its gradient.

    With G (K x K, symmetric): sum_b r_b^T G r_b / (B K), r = y - t (reading R25).
    Otherwise the weighted squared error sum_k lw_k r_k^2 / (B K): lw = None is the
    plain mean squared error, lw_k = var(w_k) / mean var the squared error of the
    PSF (the basis is orthonormal; G^ of a flat spectrum), reading R18.
    """
    y, (x, z1, h1, z2, h2) = forward(params, x)
    B, K = y.shape
    r = y - np.asarray(t, dtype=np.float64)
    if G is not None:
        rg = r @ np.asarray(G, dtype=np.float64)
        loss = float(np.sum(rg * r) / (B * K))
        dy = 2.0 * rg / (B * K)
    else:
        wk = np.ones(K) if lw is None else np.asarray(lw, dtype=np.float64)
        loss = float(np.sum(wk * r * r) / (B * K))
        dy = 2.0 * wk * r / (B * K)
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dz2 = (dy @ params["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ params["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def adam_step(params: dict, grads: dict, state: dict, lr: float, step: int,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (bias-corrected moments) in place; step counts from 1."""
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** step)
        vh = v / (1 - beta2 ** step)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params


def predict_weights(params: dict, a: np.ndarray, in_scale: np.ndarray, out_scale: np.ndarray,
                    out_shift: np.ndarray, flux: np.ndarray | None = None) -> np.ndarray:
    """w = MLP(a * in_scale) * out_scale + out_shift for Zernike vectors a (..., J).

    flux (the basis sums s_k): the surrogate's P2S weights, the network's output moved to the nearest point
    with s^T w = 1 (reading R28: the exact weights the network learns keep the PSF's unit sum, and so do
    its outputs); None: the network's output itself.
    """
    a = np.asarray(a, dtype=np.float64)
    shp = a.shape[:-1]
    y, _ = forward(params, a.reshape(-1, a.shape[-1]) * in_scale)
    w = y * out_scale + out_shift
    if flux is not None:
        s = np.asarray(flux, dtype=np.float64)
        w = w + (1.0 - w @ s)[:, None] * s / (s @ s)
    return w.reshape(*shp, -1)
