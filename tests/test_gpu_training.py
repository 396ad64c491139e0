"""The surrogate network's device training kernels against the FP64 oracle,
and what the trained network gains over the method without it."""
import numpy as np
import pytest
import torch

from inputs import synthetic
from oracle import image, mlp, p2s, sampler

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_06713_gb300 as d
    d.load()
    return d


def _flat_to_dict(flat, J, K):
    H = 256
    sizes = [("W1", (H, J)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (K, H)), ("b3", (K,))]
    out, o = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        out[name] = flat[o:o + n].reshape(shp).astype(np.float64)
        o += n
    assert o == flat.size
    return out


@pytest.mark.parametrize("J,K,B,gram", [(36, 16, 64, False), (15, 100, 33, False), (36, 100, 70, True),
                                        (36, 16, 5, True)])
def test_loss_and_gradients_match_oracle(lib, J, K, B, gram):
    n = lib.mlp_param_count(J, K)
    rng = np.random.default_rng(J + K)
    flat = (rng.standard_normal(n) * 0.1).astype(np.float32)
    X = rng.standard_normal((B, J)).astype(np.float32)
    T = rng.standard_normal((B, K)).astype(np.float32)
    lw = rng.uniform(0.2, 2.0, K).astype(np.float32)
    G = None
    if gram:  # a symmetric positive definite form (the image-prior form has this shape)
        Q = rng.standard_normal((K, K))
        G = ((Q @ Q.T) / K + 0.1 * np.eye(K)).astype(np.float32)
    loss, g = lib.mlp_loss_grad(torch.tensor(flat, device="cuda"), torch.tensor(X, device="cuda"),
                                torch.tensor(T, device="cuda"), None if gram else torch.tensor(lw, device="cuda"),
                                torch.tensor(G, device="cuda") if gram else None)
    P = _flat_to_dict(flat, J, K)
    lo, go = mlp.loss_and_grads(P, X, T, None if gram else lw, G)
    assert loss == pytest.approx(lo, rel=1e-5)
    gd = _flat_to_dict(g.cpu().numpy(), J, K)
    for name in P:
        ref = go[name]
        err = np.linalg.norm(gd[name] - ref) / np.linalg.norm(ref)
        assert err < 1e-4, (name, err)


@pytest.mark.parametrize("K", [16, 100])
def test_image_prior_gram_matches_oracle(lib, K):
    basis = p2s.build_basis(0, 36, K, 300, [2.0]) if K == 16 else \
        synthetic.random_orthonormal_rows(K, 33 * 33, seed=4).reshape(K, 33, 33)
    sd = np.random.default_rng(K).uniform(0.1, 2.0, K)
    P = lib.P2S(36, torch.as_tensor(basis, dtype=torch.float32, device="cuda"))
    G = lib.mlp_image_prior_gram(P, torch.as_tensor(sd, dtype=torch.float32, device="cuda")).cpu().numpy()
    # the oracle on the same float32-rounded basis and scales
    Go = mlp.image_prior_gram(basis.astype(np.float32), sd.astype(np.float32))
    assert np.linalg.norm(G - Go) / np.linalg.norm(Go) < 1e-5


def test_training_learns_and_beats_mean_weights(lib):
    # a short training run: the network must explain most of the weight variation and
    # its frame must be much closer to the exact-P2S frame than the spatially invariant
    # blur with the mean weights (the method without a per-pixel P2S)
    J, K, H, W, N, d = 36, 16, 64, 64, 128, 2.0
    basis = p2s.build_basis(0, J, K, 600, [d])
    f = lib.SpectralFactor(J, N, 8.0)
    P = lib.P2S(J, torch.as_tensor(basis, dtype=torch.float32, device="cuda"))
    rep = lib.mlp_train(P, f, n_pairs=1 << 16, D_over_r0=(d,), seed=3, batch=1024, steps=3000, lr=2e-3)
    assert rep["steps"] == 3000
    assert rep["val_weight_rel_l2"] < 0.05
    img = torch.as_tensor(synthetic.shapes(H, W, 3, seed=1), device="cuda")
    sim = lib.Simulator(f, P, 3, H, W)
    ex = sim.simulate_frame(img, d, 9, 0, lib.P2S_EXACT).double()
    le = sim.simulate_frame(img, d, 9, 0, lib.P2S_LEARNED).double()
    P.check()
    fields = lib.sample_zernike_fields(f, d, 9, 0, H, W)
    w_ex = lib.p2s_weights(P, lib.P2S_EXACT, fields)
    w_mean = w_ex.reshape(-1, K).mean(0).expand(H * W, K).reshape(H, W, K).contiguous()
    warped = lib.tilt_warp(img, fields[0].contiguous(), fields[1].contiguous())
    mean_frame = lib.basis_blur(P, warped, w_mean).double()
    e_learned = float((le - ex).norm() / ex.norm())
    e_mean = float((mean_frame - ex).norm() / ex.norm())
    assert e_learned < 0.5 * e_mean, (e_learned, e_mean)


@pytest.mark.parametrize("K,n_psf,drs", [(16, 300, (2.0,)), (100, 2000, (1.0, 2.0, 4.0))])
def test_basis_svd_matches_oracle(lib, K, n_psf, drs):
    J = 36
    f = lib.SpectralFactor(J, 64, 8.0)
    basis, sig, sweeps = lib.build_basis(f, K, n_psf, drs, seed=5)
    assert 1 <= sweeps < 40
    g = basis.double().cpu().numpy().reshape(K, -1)
    a = p2s.basis_draws(5, J, n_psf, list(drs))
    Hm = p2s.psf(a, J).reshape(n_psf, -1)
    Phi, s = p2s.svd_basis(Hm, K)
    assert np.allclose(sig[:K], s[:K], rtol=1e-5)
    # orthonormal rows, same subspace (projector distance), same vectors where the spectrum is not degenerate
    assert np.allclose(g @ g.T, np.eye(K), atol=1e-6)
    proj = np.linalg.norm(g.T @ g - Phi.T @ Phi) / np.sqrt(K)
    gap = (s[K - 1] - s[K]) / s[0]
    if gap > 1e-4:
        assert proj < 1e-3
    for k in range(K):
        sep = min(abs(s[k] - s[k - 1]) if k > 0 else 1.0, abs(s[k] - s[k + 1])) / s[0]
        if sep > 1e-3:
            assert np.dot(g[k], Phi[k]) > 1 - 1e-4, k
