"""Pins for the oracle's PSF (Eq. 2), basis (Sec. II-C), warp, blur (Eq. 1, Eq. varying blur)
and the surrogate network's gradients."""
import math

import numpy as np
import pytest

from inputs import synthetic
from oracle import image, mlp, p2s, zernike


# ------------------------------------------------------------------- PSF
def test_zero_phase_psf_symmetry_and_parseval():
    J = 10
    h = p2s.psf_full(np.zeros(J), J)
    assert np.allclose(h, h[::-1, ::-1][np.r_[-1, 0:63]][:, np.r_[-1, 0:63]], rtol=1e-10)  # u -> -u about index 32
    assert np.allclose(h, h.T, rtol=1e-10)
    _, _, P = p2s.pupil_grid()
    assert h.sum() == pytest.approx(64 * 64 * (P ** 2).sum(), rel=1e-12)  # Parseval
    assert h[32, 32] == pytest.approx(P.sum() ** 2, rel=1e-12)


@pytest.mark.parametrize("k", [1, 2, -3])
def test_tilt_is_an_exact_shift(k):
    # a_2 = (pi/4) k puts the PSF peak k pixels towards -x (reading R10): exact circular shift
    J = 6
    h0 = p2s.psf_full(np.zeros(J), J, with_tilt=True)
    a = np.zeros(J)
    a[0] = math.pi / 4 * k
    hx = p2s.psf_full(a, J, with_tilt=True)
    assert np.allclose(hx, np.roll(h0, -k, axis=1), atol=1e-9 * h0.max())
    a = np.zeros(J)
    a[1] = math.pi / 4 * k
    hy = p2s.psf_full(a, J, with_tilt=True)
    assert np.allclose(hy, np.roll(h0, -k, axis=0), atol=1e-9 * h0.max())


def test_psf_unit_sum_and_tilt_free():
    J = 36
    rng = np.random.default_rng(0)
    a = rng.standard_normal((5, J)) * 0.3
    h = p2s.psf(a, J)
    assert h.shape == (5, 33, 33)
    assert np.allclose(h.sum(axis=(1, 2)), 1.0)
    a2 = a.copy()
    a2[:, :2] += 5.0
    assert np.allclose(p2s.psf(a2, J), h)  # tilts never enter the P2S PSF (R9)


def test_svd_basis_eckart_young_and_orthonormal():
    J, n, K = 36, 120, 16
    a = p2s.basis_draws(3, J, n, [2.0])
    Hm = p2s.psf(a, J).reshape(n, -1)
    Phi, s = p2s.svd_basis(Hm, K)
    assert np.allclose(Phi @ Phi.T, np.eye(K), atol=1e-12)
    resid = Hm - Hm @ Phi.T @ Phi
    assert np.sum(resid ** 2) == pytest.approx(np.sum(s[K:] ** 2), rel=1e-9)
    for k in range(K):
        i = np.argmax(np.abs(Phi[k]))
        assert Phi[k, i] > 0


def test_basis_draws_have_noll_covariance():
    J = 8
    a = p2s.basis_draws(9, J, 20000, [3.0])
    A0 = zernike.noll_matrix(J, 3.0)
    emp = a.T @ a / a.shape[0]
    sub = A0[2:, 2:]
    sd = np.sqrt((np.outer(np.diag(sub), np.diag(sub)) + sub ** 2) / a.shape[0])
    assert np.all(np.abs(emp[2:, 2:] - sub) < 5 * sd)
    assert np.all(a[:, :2] == 0)


def test_weights_recover_in_span_coefficients():
    # a basis whose span holds the PSFs themselves (orthonormalised PSFs): the weights are their exact
    # coefficients, and since each PSF has unit sum the flux constraint of R28 changes nothing
    J, K = 12, 8
    a = np.random.default_rng(2).standard_normal((K, J)) * 0.2
    h = p2s.psf(a, J).reshape(K, -1)
    Q, _ = np.linalg.qr(h.T)  # 1089 x K, orthonormal columns spanning the PSFs
    Phi = Q.T.reshape(K, 33, 33)
    w = p2s.weights(a[:3], J, Phi)
    assert np.allclose(w, h[:3] @ Q, rtol=1e-12, atol=1e-14)
    assert np.allclose((w @ Q.T), h[:3], atol=1e-13)


def test_flux_preserving_projection_is_the_constrained_least_squares_solution():
    # reading R28: w = argmin ||h - Phi^T w||^2 subject to s^T w = 1, s_k = sum_u phi_k(u).  Checked against
    # the KKT system of that problem solved directly (no closed form, no orthonormality used), the constraint,
    # and the cost identity ||h - Phi^T w||^2 = ||h - Phi^T w_ls||^2 + (1 - s^T w_ls)^2 / s^T s
    J, K = 20, 24
    basis = p2s.build_basis(3, J, K, 300, [4.0])
    B = basis.reshape(K, -1)
    a = p2s.basis_draws(9, J, 6, [4.0])
    h = p2s.psf(a, J).reshape(6, -1)
    w = p2s.weights(a, J, basis)
    w_ls = p2s.weights_unconstrained(a, J, basis)
    s = B.sum(axis=1)
    kkt = np.zeros((K + 1, K + 1))
    kkt[:K, :K] = B @ B.T
    kkt[:K, K] = s
    kkt[K, :K] = s
    for i in range(6):
        sol = np.linalg.solve(kkt, np.concatenate([B @ h[i], [1.0]]))
        assert np.allclose(w[i], sol[:K], rtol=1e-10, atol=1e-13)
        assert w[i] @ s == pytest.approx(1.0, abs=1e-13)
        c = np.sum((h[i] - w[i] @ B) ** 2)
        c_ls = np.sum((h[i] - w_ls[i] @ B) ** 2)
        assert c == pytest.approx(c_ls + (1.0 - w_ls[i] @ s) ** 2 / (s @ s), rel=1e-9)
    # the plain projection loses flux at this strength (the reason for R28)
    assert np.abs(w_ls @ s - 1.0).max() > 1e-3


def test_surrogate_output_keeps_unit_flux():
    J, K = 10, 12
    rng = np.random.default_rng(4)
    params = {"W1": rng.standard_normal((256, J)) / 4, "b1": rng.standard_normal(256) * 0.1,
              "W2": rng.standard_normal((256, 256)) / 16, "b2": rng.standard_normal(256) * 0.1,
              "W3": rng.standard_normal((K, 256)) / 16, "b3": rng.standard_normal(K) * 0.1}
    s = rng.standard_normal(K)
    a = rng.standard_normal((5, 7, J))
    isc, osc, osh = np.ones(J), rng.uniform(0.5, 2, K), rng.standard_normal(K)
    raw = mlp.predict_weights(params, a, isc, osc, osh)
    w = mlp.predict_weights(params, a, isc, osc, osh, flux=s)
    assert np.allclose(w @ s, 1.0, atol=1e-12)
    # the smallest change that meets the constraint: along s only
    d = (w - raw).reshape(-1, K)
    assert np.allclose(d - np.outer(d @ s / (s @ s), s), 0.0, atol=1e-12)


# ------------------------------------------------------------------ image
def test_warp_identity_shift_and_ramp():
    img = synthetic.blobs(24, 20, 2, n=5, seed=1).astype(np.float64)
    z = np.zeros((24, 20))
    assert np.allclose(image.tilt_warp(img, z, z), img)
    k = 3
    out = image.tilt_warp(img, z + math.pi / 4 * k, z)  # sample at x + 3
    assert np.allclose(out[:, :, :20 - k], img[:, :, k:])
    assert np.allclose(out[:, :, 20 - k:], img[:, :, -1:])
    out = image.tilt_warp(img, z, z - math.pi / 4 * 2)  # sample at y - 2
    assert np.allclose(out[:, 2:], img[:, :-2])
    yy, xx = np.meshgrid(np.arange(24.0), np.arange(20.0), indexing="ij")
    ramp = (0.3 * xx + 0.7 * yy)[None]
    rng = np.random.default_rng(0)
    a2 = rng.uniform(-1, 1, (24, 20))
    a3 = rng.uniform(-1, 1, (24, 20))
    out = image.tilt_warp(ramp, a2, a3)
    sx = xx + 4 / math.pi * a2
    sy = yy + 4 / math.pi * a3
    inside = (sx >= 0) & (sx <= 19) & (sy >= 0) & (sy <= 23)
    assert np.allclose(out[0][inside], (0.3 * sx + 0.7 * sy)[inside], atol=1e-12)


def test_blur_equals_direct_per_pixel_convolution():
    C, H, W, K = 2, 20, 23, 5
    img = synthetic.blobs(H, W, C, n=6, seed=3).astype(np.float64)
    Phi = np.random.default_rng(4).standard_normal((K, 33, 33))
    w = np.random.default_rng(5).standard_normal((H, W, K))
    out = image.basis_blur(img, w, Phi)
    h = np.einsum("yxk,kab->yxab", w, Phi)
    assert np.allclose(out, image.direct_blur(img, h), atol=1e-10)


def test_blur_is_a_true_convolution():
    img = synthetic.blobs(16, 16, 1, n=4, seed=2).astype(np.float64)
    delta = np.zeros((1, 33, 33))
    delta[0, 16, 17] = 1.0  # u = (0, +1)
    out = image.basis_blur(img, np.ones((16, 16, 1)), delta)
    assert np.allclose(out[:, :, 1:], img[:, :, :-1])  # out(x) = I(x - (0, 1))
    const = np.full((1, 16, 16), 0.25)
    Phi = np.random.default_rng(1).standard_normal((3, 33, 33))
    w = np.random.default_rng(2).standard_normal((16, 16, 3))
    out = image.basis_blur(const, w, Phi)
    assert np.allclose(out[0], 0.25 * w @ Phi.sum(axis=(1, 2)))


# -------------------------------------------------------------------- MLP
def _params(J, Hd, K, seed=0):
    rng = np.random.default_rng(seed)
    return {"W1": rng.standard_normal((Hd, J)) / math.sqrt(J), "b1": rng.standard_normal(Hd) * 0.1,
            "W2": rng.standard_normal((Hd, Hd)) / math.sqrt(Hd), "b2": rng.standard_normal(Hd) * 0.1,
            "W3": rng.standard_normal((K, Hd)) / math.sqrt(Hd), "b3": rng.standard_normal(K) * 0.1}


@pytest.mark.parametrize("kind", ["plain", "weighted", "gram"])
def test_mlp_gradients_by_finite_differences(kind):
    J, Hd, K, B = 5, 7, 4, 6
    P = _params(J, Hd, K)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((B, J))
    t = rng.standard_normal((B, K))
    lw = rng.uniform(0.1, 3.0, K) if kind == "weighted" else None
    G = None
    if kind == "gram":
        Q = rng.standard_normal((K, K))
        G = Q @ Q.T + 0.1 * np.eye(K)
    _, g = mlp.loss_and_grads(P, x, t, lw, G)
    eps = 1e-6
    for name, val in P.items():
        flat = val.ravel()
        for i in range(0, flat.size, max(1, flat.size // 9)):
            old = flat[i]
            flat[i] = old + eps
            lp, _ = mlp.loss_and_grads(P, x, t, lw, G)
            flat[i] = old - eps
            lm, _ = mlp.loss_and_grads(P, x, t, lw, G)
            flat[i] = old
            assert g[name].ravel()[i] == pytest.approx((lp - lm) / (2 * eps), rel=1e-6, abs=1e-9)


def test_image_prior_gram_is_the_blurred_error_energy():
    # r^T G r = sum_f S |Phi_r|^2 = M^2 sum_x |(phi_r (*) g)(x)|^2 with DFT(g) = sqrt(S): the circular
    # convolution is done directly, shift by shift, so the DFT convention and the embedding are pinned
    M, K = 64, 3
    rng = np.random.default_rng(5)
    basis = rng.standard_normal((K, 33, 33))
    sd = np.ones(K)
    f = np.fft.fftfreq(M) * M
    S = 1.0 / (f[:, None] ** 2 + f[None, :] ** 2 + 1.0)
    g = np.real(np.fft.ifft2(np.sqrt(S)))
    G = mlp.image_prior_gram(basis, sd, M)
    scale = None
    for trial in range(3):
        r = rng.standard_normal(K)
        phi = np.tensordot(r, basis, axes=1)
        conv = np.zeros((M, M))
        for u in range(33):
            for v in range(33):
                conv += phi[u, v] * np.roll(np.roll(g, u, axis=0), v, axis=1)
        energy = M * M * np.sum(conv ** 2)
        # G^ carries the unit-mean-diagonal scale; recover it from the unscaled form
        Fb = np.fft.fft2(np.pad(basis, ((0, 0), (0, M - 33), (0, M - 33)))).reshape(K, -1)
        G_raw = np.real((Fb * S.reshape(1, -1)) @ Fb.conj().T)
        scale = np.mean(np.diag(G_raw))
        assert r @ G @ r * scale == pytest.approx(energy, rel=1e-10)


def test_image_prior_gram_flat_spectrum_is_the_psf_weighted_loss():
    # an orthonormal basis and a flat spectrum: G = M^2 I (Parseval), so G^ = diag(sd^2) / mean(sd^2) = lw
    K = 6
    basis = synthetic.random_orthonormal_rows(K, 33 * 33, seed=2).reshape(K, 33, 33)
    sd = np.random.default_rng(3).uniform(0.2, 2.0, K)
    G = mlp.image_prior_gram(basis, sd, flat=True)
    assert np.allclose(G, np.diag(sd ** 2 / np.mean(sd ** 2)), atol=1e-12)
    # with the image spectrum the form stays symmetric positive definite
    G2 = mlp.image_prior_gram(basis, sd)
    assert np.allclose(G2, G2.T, atol=1e-14)
    assert np.linalg.eigvalsh(G2).min() > 0


def test_gelu_and_adam_closed_forms():
    from scipy.stats import norm
    z = np.linspace(-5, 5, 101)
    assert np.allclose(mlp.gelu(z), z * norm.cdf(z), atol=1e-15)
    d = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    assert np.allclose(mlp.gelu_grad(z), d, atol=1e-8)
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    mlp.adam_step(p, g, {}, lr=0.01, step=1)
    # first Adam step moves each parameter by lr * g / (|g| + eps)
    assert np.allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01 * 1e-3 / (1e-3 + 1e-8)], rtol=1e-12)
