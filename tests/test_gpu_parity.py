"""GPU parity: every stage of the CUDA path through the C ABI against the FP64 oracle.

Tolerances: integer work (Philox words) and the FP32 Gaussians bit-exact; FP32
stages rel-L2 <= 1e-5 (rel-L2 = ||x - y||_2 / ||y||_2 over the whole tensor, in
FP64).
"""
import math

import numpy as np
import pytest
import torch

from inputs import synthetic
from oracle import image, mlp, noise, p2s, sampler, spectrum, zernike

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_06713_gb300 as d
    d.load()
    return d


def cu(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


# ------------------------------------------------------------------ noise
@pytest.mark.parametrize("seed,sub,q0", [(0, 0, 0), (0x123456789ABCDEF, (3 << 40) | (77 << 8) | 5, 12345),
                                         (2 ** 64 - 1, 2 ** 64 - 1, 2 ** 40)])
def test_philox_words_bit_exact(lib, seed, sub, q0):
    n = 4 * 4096
    g = lib.philox_words(seed, sub, q0, n).cpu().numpy().view(np.uint32)
    q = np.arange(q0, q0 + n // 4, dtype=np.uint64)
    w = noise.philox_words(seed, sub, q)
    assert np.array_equal(g, np.stack(w, axis=-1).ravel())


@pytest.mark.parametrize("seed,tag,frame,mode", [(0, 0, 0, 0), (7, 0, 123456, 35), (2 ** 63 + 5, 3, 2 ** 32 - 1, 255)])
def test_gaussians_bit_exact(lib, seed, tag, frame, mode):
    g = lib.gaussian_noise(seed, tag, frame, mode, 256, 512).cpu().numpy()
    o = noise.gaussian_block(seed, tag, frame, mode, 256, 512)
    assert np.array_equal(g.view(np.uint32), o.view(np.uint32))


# ----------------------------------------------------------------- factor
@pytest.mark.parametrize("J,N,ppd", [(36, 128, 8.0), (15, 64, 2.0), (6, 16, 2.0), (36, 512, 8.0)])
def test_spectral_factor_matches_oracle(lib, J, N, ppd):
    f = lib.SpectralFactor(J, N, ppd)
    m = f.multiplier().cpu().numpy().astype(np.float64)  # [j][kx][ky]
    lam = spectrum.lambdas(J, N, ppd)  # [j][ky][kx]
    ref = np.sqrt(lam[:, :, : N // 2 + 1]).transpose(0, 2, 1) / N ** 2
    assert rel_l2(m, ref) < 1e-6
    assert np.max(np.abs(m - ref)) <= 2e-6 * ref.max()
    L = f.cholesky()
    assert np.allclose(L, zernike.noll_cholesky(J, 1.0), rtol=1e-11, atol=1e-14)


# ----------------------------------------------------------------- fields
@pytest.mark.parametrize("J,H,W,N,ppd,d,seed,frame", [
    (36, 64, 64, 128, 8.0, 2.0, 0, 0),      # small plain-method workload
    (36, 50, 37, 128, 8.0, 3.0, 5, 9),      # ragged crop, odd height
    (15, 16, 16, 64, 2.0, 1.0, 1, 1),       # J = 15
    (36, 256, 256, 512, 8.0, 3.0, 0, 3),    # 256 x 256 workload
    (6, 16, 9, 16, 2.0, 1.0, 4, 0),         # smallest grid: one thread per FFT
    (10, 30, 17, 32, 2.0, 2.0, 8, 6),       # N = 32: one radix-32 pass
    (4, 700, 1500, 2048, 8.0, 2.0, 2, 1),   # three passes (32 x 32 x 2), block-wide exchanges
    (36, 33, 21, 128, 8.0, 2.0, 3, 2),      # odd pixel count: one pixel per mixing thread
    (45, 31, 29, 128, 8.0, 2.0, 1, 0),      # J > 40: the 64-wide mixing bucket
])
def test_fields_match_oracle(lib, J, H, W, N, ppd, d, seed, frame):
    f = lib.SpectralFactor(J, N, ppd)
    g = lib.sample_zernike_fields(f, d, seed, frame, H, W).cpu().numpy()
    o = sampler.sample_fields(seed, frame, J, H, W, d, ppd, N)
    assert rel_l2(g, o) < TOL
    for j in (0, 1, J - 1):
        assert rel_l2(g[j], o[j]) < 3 * TOL


def test_fields_full_size_512(lib):
    # the 512 x 512 benchmark workload (N = 1024), every sample against the oracle
    J, H, W, N = 36, 512, 512, 1024
    f = lib.SpectralFactor(J, N, 8.0)
    g = lib.sample_zernike_fields(f, 4.0, 11, 2, H, W).cpu().numpy()
    o = sampler.sample_fields(11, 2, J, H, W, 4.0, 8.0, N)
    assert rel_l2(g, o) < TOL


@pytest.mark.slow
def test_fields_grid_4096(lib):
    # the 3840 x 2160 workload's grid (32 x 32 x 4 passes), few modes to bound the oracle's cost
    J, H, W, N = 3, 2160, 3840, 4096
    f = lib.SpectralFactor(J, N, 8.0)
    g = lib.sample_zernike_fields(f, 4.0, 1, 0, H, W).cpu().numpy()
    o = sampler.sample_fields(1, 0, J, H, W, 4.0, 8.0, N)
    assert rel_l2(g, o) < TOL


@pytest.mark.parametrize("J,H,W,N,alpha", [(36, 40, 33, 128, 0.8), (15, 64, 64, 128, 0.3)])
def test_ar1_fields_match_oracle(lib, J, H, W, N, alpha):
    f = lib.SpectralFactor(J, N, 8.0)
    o = sampler.sample_fields_ar1(5, 3, alpha, J, H, W, 2.0, 8.0, N)
    prev = None
    for t in range(3):
        g = lib.sample_zernike_fields_ar1(f, 2.0, 5, t, alpha, H, W, prev)
        assert rel_l2(g.cpu().numpy(), o[t]) < TOL
        prev = g
    with pytest.raises(lib.DFP2SError):
        lib.sample_zernike_fields_ar1(f, 2.0, 5, 3, alpha, H, W, prev, out=prev)  # aliasing


def test_fields_are_deterministic_and_frame_dependent(lib):
    f = lib.SpectralFactor(36, 128, 8.0)
    a = lib.sample_zernike_fields(f, 2.0, 3, 4, 64, 64).cpu()
    b = lib.sample_zernike_fields(f, 2.0, 3, 4, 64, 64).cpu()
    c = lib.sample_zernike_fields(f, 2.0, 3, 5, 64, 64).cpu()
    assert torch.equal(a, b)
    assert not torch.equal(a, c)
    # D/r0 only scales the fields by (D/r0)^{5/6}
    e = lib.sample_zernike_fields(f, 4.0, 3, 4, 64, 64).cpu()
    assert torch.allclose(e, a * 2 ** (5 / 6), rtol=1e-5, atol=1e-6)


# -------------------------------------------------------------------- warp
@pytest.mark.parametrize("C,H,W", [(1, 64, 64), (3, 37, 53), (2, 5, 3), (3, 256, 256)])
def test_tilt_warp_matches_oracle(lib, C, H, W):
    img = synthetic.blobs(H, W, C, n=8, seed=C)
    fld = synthetic.random_fields(2, H, W, scale=2.0, seed=H)
    g = lib.tilt_warp(cu(img), cu(fld[0]), cu(fld[1])).cpu().numpy()
    o = image.tilt_warp(img, fld[0], fld[1])
    assert rel_l2(g, o) < TOL


# --------------------------------------------------------------------- P2S
@pytest.mark.parametrize("J,K,H,W,d", [(36, 16, 24, 20, 2.0), (36, 100, 9, 13, 4.0), (15, 32, 8, 8, 1.0)])
def test_exact_weights_match_oracle(lib, J, K, H, W, d):
    basis = synthetic.random_orthonormal_rows(K, 33 * 33, seed=K).reshape(K, 33, 33)
    a = sampler.sample_fields(3, 1, J, H, W, d, 8.0, sampler.grid_size(H, W))
    P = lib.P2S(J, cu(basis))
    g = lib.p2s_weights(P, lib.P2S_EXACT, cu(a)).cpu().numpy()
    o = p2s.weights_field(a, basis)
    assert rel_l2(g, o) < TOL
    gb = lib.p2s_weights(P, lib.P2S_EXACT, cu(a), w_dtype=lib.W_BF16).float().cpu().numpy()
    assert rel_l2(gb, o) < 4e-3  # bfloat16 storage


def test_exact_weights_with_svd_basis(lib):
    J, K = 36, 16
    basis = p2s.build_basis(0, J, K, 400, [2.0])
    a = sampler.sample_fields(0, 0, J, 16, 16, 2.0, 8.0, 128)
    P = lib.P2S(J, cu(basis))
    g = lib.p2s_weights(P, lib.P2S_EXACT, cu(a)).cpu().numpy()
    assert rel_l2(g, p2s.weights_field(a, basis)) < TOL


# -------------------------------------------------------------------- blur
@pytest.mark.parametrize("C,H,W,K", [(1, 64, 64, 16), (3, 37, 45, 100), (5, 20, 33, 7)])
def test_blur_fp32_matches_oracle(lib, C, H, W, K):
    img = synthetic.blobs(H, W, C, n=6, seed=K)
    basis = synthetic.random_orthonormal_rows(K, 33 * 33, seed=C).reshape(K, 33, 33)
    w = np.random.default_rng(H).standard_normal((H, W, K)).astype(np.float32)
    P = lib.P2S(36, cu(basis))
    g = lib.basis_blur(P, cu(img), cu(w)).cpu().numpy()
    o = image.basis_blur(img, w, basis)
    assert rel_l2(g, o) < TOL


def _bf16(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


@pytest.mark.parametrize("C,H,W,K", [(3, 64, 130, 100), (1, 33, 200, 16), (5, 20, 128, 112), (2, 17, 19, 128),
                                     (3, 40, 256, 100), (3, 256, 512, 100), (3, 512, 512, 100)])
def test_blur_bf16_tensor_cores_match_oracle_on_bf16_operands(lib, C, H, W, K):
    # the tcgen05 blur rounds image and basis to bfloat16 and accumulates in FP32; against the oracle
    # evaluated on the same bfloat16 operands it must agree to FP32 accumulation error.  The last two shapes
    # give every CTA of the persistent grid several tiles (1024 and 2048 tiles over at most 152 CTAs; the
    # second is the 512 x 512 x 3 frame of the benchmark), so the operand rings and the accumulator slots
    # wrap around many times
    img = synthetic.blobs(H, W, C, n=6, seed=K)
    basis = synthetic.random_orthonormal_rows(K, 33 * 33, seed=C).reshape(K, 33, 33)
    w = torch.as_tensor(np.random.default_rng(H).standard_normal((H, W, K)), dtype=torch.bfloat16, device="cuda")
    P = lib.P2S(36, cu(basis))
    g = lib.basis_blur(P, cu(img), w).cpu().numpy()
    P.check()
    # the kernel's operands: bf16(I - 0.5) (the 0.5 added back exactly), bf16 basis, weights as stored
    img_q = _bf16(img - 0.5) + 0.5
    o = image.basis_blur(img_q, w.float().cpu().numpy(), _bf16(basis))
    assert rel_l2(g, o) < TOL
    # and stays within bfloat16 rounding of the FP32-operand result
    assert rel_l2(g, image.basis_blur(img, w.float().cpu().numpy(), basis)) < 1e-2
    # FP32 weights through the same tensor-core path
    wf = torch.as_tensor(np.random.default_rng(H + 1).standard_normal((H, W, K)), dtype=torch.float32, device="cuda")
    g32 = lib.basis_blur_tc(P, cu(img), wf).cpu().numpy()
    P.check()
    assert rel_l2(g32, image.basis_blur(img_q, wf.cpu().numpy(), _bf16(basis))) < TOL
    # the two public steps give the same result bit for bit
    lib.basis_blur_tc_prepare(P, cu(img))
    g2 = lib.basis_blur_tc_run(P, (C, H, W), wf).cpu().numpy()
    assert np.array_equal(g2, g32)


@pytest.mark.parametrize("C,H,W,K", [(3, 70, 200, 100), (2, 33, 17, 16)])
def test_fused_warp_prepare_is_bit_exact(lib, C, H, W, K):
    # the fused warp + operand preparation gives the same blur, bit for bit, as the warp followed by preparation
    img = synthetic.blobs(H, W, C, n=6, seed=K)
    fld = synthetic.random_fields(2, H, W, scale=2.0, seed=W)
    basis = synthetic.random_orthonormal_rows(K, 33 * 33, seed=C).reshape(K, 33, 33)
    P = lib.P2S(36, cu(basis))
    w = torch.as_tensor(np.random.default_rng(H).standard_normal((H, W, K)), dtype=torch.float32, device="cuda")
    warped = lib.tilt_warp(cu(img), cu(fld[0]), cu(fld[1]))
    lib.basis_blur_tc_prepare(P, warped)
    ref = lib.basis_blur_tc_run(P, (C, H, W), w).cpu().numpy()
    lib.tilt_warp_blur_tc_prepare(P, cu(img), cu(fld[0]), cu(fld[1]))
    got = lib.basis_blur_tc_run(P, (C, H, W), w).cpu().numpy()
    P.check()
    assert np.array_equal(got, ref)
    # and the frame against the oracle's warp + blur on the kernel's bfloat16 operands
    o = image.basis_blur(_bf16(image.tilt_warp(img, fld[0], fld[1]) - 0.5) + 0.5, w.cpu().numpy(), _bf16(basis))
    assert rel_l2(got, o) < 1e-4


def test_blur_tc_run_needs_a_prepared_image(lib):
    basis = synthetic.random_orthonormal_rows(16, 33 * 33, seed=3).reshape(16, 33, 33)
    P = lib.P2S(36, cu(basis))
    w = torch.zeros(20, 30, 16, device="cuda")
    with pytest.raises(lib.DFP2SError) as e:
        lib.basis_blur_tc_run(P, (1, 20, 30), w)  # nothing prepared yet
    assert e.value.code == -1
    lib.basis_blur_tc_prepare(P, torch.zeros(1, 20, 30, device="cuda"))
    with pytest.raises(lib.DFP2SError):
        lib.basis_blur_tc_run(P, (1, 20, 31), torch.zeros(20, 31, 16, device="cuda"))  # another shape
    lib.basis_blur_tc_run(P, (1, 20, 30), w)


# ---------------------------------------------------------------- network
def _bf(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


@pytest.mark.parametrize("K,H,W", [(100, 16, 24), (16, 9, 31), (128, 130, 3), (100, 256, 160)])
def test_mlp_forward_matches_oracle(lib, K, H, W):
    J = 36
    rng = np.random.default_rng(K)
    params = {"W1": rng.standard_normal((256, J)) / 6, "b1": rng.standard_normal(256) * 0.1,
              "W2": rng.standard_normal((256, 256)) / 16, "b2": rng.standard_normal(256) * 0.1,
              "W3": rng.standard_normal((K, 256)) / 16, "b3": rng.standard_normal(K) * 0.1}
    params = {k: v.astype(np.float32).astype(np.float64) for k, v in params.items()}
    in_scale = rng.uniform(0.5, 2.0, J).astype(np.float32).astype(np.float64)
    in_scale[:2] = 0
    out_scale = rng.uniform(0.5, 2, K).astype(np.float32).astype(np.float64)
    out_shift = rng.standard_normal(K).astype(np.float32).astype(np.float64)
    basis = synthetic.random_orthonormal_rows(K, 33 * 33, seed=1).reshape(K, 33, 33)
    P = lib.P2S(J, cu(basis))
    P.set_mlp(*[cu(params[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")], cu(in_scale), cu(out_scale),
              cu(out_shift))
    a = synthetic.random_fields(J, H, W, scale=0.5, seed=3)
    av = np.moveaxis(a, 0, -1).reshape(-1, J).astype(np.float64)
    fl = p2s.flux_vector(basis)
    o = mlp.predict_weights(params, av, in_scale, out_scale, out_shift, flux=fl).reshape(H, W, K)
    # FP32 CUDA-core form against the FP64 oracle
    g32 = lib.p2s_weights(P, lib.P2S_LEARNED_FP32, cu(a)).cpu().numpy()
    assert rel_l2(g32, o) < TOL
    # tensor-core form against the oracle evaluated with the kernel's bfloat16 roundings
    g = lib.p2s_weights(P, lib.P2S_LEARNED, cu(a)).cpu().numpy()
    P.check()
    z1 = _bf(av) @ _bf(params["W1"] * in_scale[None, :]).T + params["b1"]
    h1 = _bf(mlp.gelu(z1))
    z2 = h1 @ _bf(params["W2"]).T + params["b2"]
    h2 = _bf(mlp.gelu(z2))
    y = h2 @ _bf(params["W3"]).T
    ob = p2s.flux_projection(y * out_scale + (params["b3"] * out_scale + out_shift), fl).reshape(H, W, K)
    assert rel_l2(g, ob) < 1e-3
    assert rel_l2(g, o) < 2e-2
    gb = lib.p2s_weights(P, lib.P2S_LEARNED, cu(a), w_dtype=lib.W_BF16).float().cpu().numpy()
    assert rel_l2(gb, ob) < 4e-3


# ------------------------------------------------------------------- frame
def _device_view(ptr, shape):
    class _A:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (ptr, False), "version": 3}
    return torch.as_tensor(_A(), device="cuda")


@pytest.mark.parametrize("d", [1.0, 3.0])
def test_learned_frame_folds_the_mixing_into_warp_and_first_layer(lib, d):
    # the LEARNED frame skips the mixing pass: the warp forms its tilts from the unit fields u0, u1 and the first
    # layer takes W1 diag(in_scale) L on s u (s = (D/r0)^(5/6)).  Its weights against the oracle network evaluated
    # with the kernel's BF16 roundings of that input; the frame against the step-by-step calls on the mixed
    # fields (which round the network's input differently); a new install re-packs the first layer
    J, K, H, W, N = 36, 100, 96, 80, 256
    rng = np.random.default_rng(7)
    params = {"W1": rng.standard_normal((256, J)) / 6, "b1": rng.standard_normal(256) * 0.1,
              "W2": rng.standard_normal((256, 256)) / 16, "b2": rng.standard_normal(256) * 0.1,
              "W3": rng.standard_normal((K, 256)) / 16, "b3": rng.standard_normal(K) * 0.1}
    params = {k: v.astype(np.float32).astype(np.float64) for k, v in params.items()}
    in_scale = rng.uniform(0.5, 2.0, J).astype(np.float32).astype(np.float64)
    in_scale[:2] = 0
    basis = synthetic.random_orthonormal_rows(K, 33 * 33, seed=1).reshape(K, 33, 33)
    f = lib.SpectralFactor(J, N, 8.0)
    P = lib.P2S(J, cu(basis))
    img = cu(synthetic.shapes(H, W, 3, seed=2))
    sim = lib.Simulator(f, P, 3, H, W)
    L = zernike.noll_cholesky(J, 1.0).astype(np.float32).astype(np.float64)
    s = float(np.float32(d ** (5.0 / 6.0)))
    for it in range(2):
        prm = {k: (v * (1 + it)).astype(np.float32).astype(np.float64) for k, v in params.items()}
        sc = rng.uniform(0.01, 0.05, K).astype(np.float32).astype(np.float64)
        P.set_mlp(*[cu(prm[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")], cu(in_scale), cu(sc), cu(np.zeros(K)))
        g = sim.simulate_frame(img, d, 5, it, lib.P2S_LEARNED)
        P.check()
        fp, _, wp = sim.buffers(J, 3, H, W, K)
        u = _device_view(fp, (J, H * W)).cpu().numpy().astype(np.float64)
        wg = _device_view(wp, (H * W, K)).cpu().numpy()
        x = _bf((u.T.astype(np.float32) * np.float32(s)))
        z1 = x @ _bf((prm["W1"] * in_scale[None, :]) @ L).T + prm["b1"]
        h1 = _bf(mlp.gelu(z1))
        h2 = _bf(mlp.gelu(h1 @ _bf(prm["W2"]).T + prm["b2"]))
        ob = p2s.flux_projection((h2 @ _bf(prm["W3"]).T) * sc + prm["b3"] * sc, p2s.flux_vector(basis))
        assert rel_l2(wg, ob) < 1e-3
        a = lib.sample_zernike_fields(f, d, 5, it, H, W)
        lib.tilt_warp_blur_tc_prepare(P, img, a[0].contiguous(), a[1].contiguous())
        w = lib.p2s_weights(P, lib.P2S_LEARNED, a)
        o = lib.basis_blur_tc_run(P, (3, H, W), w)
        e = rel_l2(g.cpu().numpy(), o.cpu().numpy())
        assert e < 3e-3, e


def test_network_file_round_trip(lib, tmp_path):
    J, K = 36, 100
    rng = np.random.default_rng(2)
    prm = [rng.standard_normal((256, J)) / 6, rng.standard_normal(256) * 0.1, rng.standard_normal((256, 256)) / 16,
           rng.standard_normal(256) * 0.1, rng.standard_normal((K, 256)) / 16, rng.standard_normal(K) * 0.1,
           rng.uniform(0.5, 2.0, J), rng.uniform(0.01, 0.05, K), rng.standard_normal(K) * 0.01]
    basis = synthetic.random_orthonormal_rows(K, 33 * 33, seed=1).reshape(K, 33, 33)
    P = lib.P2S(J, cu(basis))
    path = str(tmp_path / "net.bin")
    with pytest.raises(lib.DFP2SError):
        P.save_mlp(path)  # nothing installed
    P.set_mlp(*[cu(x) for x in prm])
    P.save_mlp(path)
    raw = open(path, "rb").read()
    assert raw[:8] == b"DFP2SMLP" and len(raw) == 20 + 4 * (256 * J + 256 + 256 * 256 + 256 + 256 * K + K + J + 2 * K)
    body = np.frombuffer(raw[20:], dtype="<f4")
    assert np.array_equal(body[:256 * J], prm[0].astype(np.float32).ravel())  # W1 as given
    Q = lib.P2S(J, cu(basis))
    Q.load_mlp(path)
    a = cu(synthetic.random_fields(J, 40, 24, scale=0.5, seed=3))
    for mode in (lib.P2S_LEARNED, lib.P2S_LEARNED_FP32):
        assert torch.equal(lib.p2s_weights(P, mode, a), lib.p2s_weights(Q, mode, a))
    with pytest.raises(lib.DFP2SError):
        lib.P2S(J - 1, cu(basis)).load_mlp(path)  # another J
    open(str(tmp_path / "short.bin"), "wb").write(raw[:-4])
    with pytest.raises(lib.DFP2SError):
        Q.load_mlp(str(tmp_path / "short.bin"))


def test_frame_stage_timing(lib):
    J, K, H, W, N = 36, 16, 64, 48, 128
    basis = synthetic.random_orthonormal_rows(K, 33 * 33, seed=1).reshape(K, 33, 33)
    f = lib.SpectralFactor(J, N, 8.0)
    P = lib.P2S(J, cu(basis))
    sim = lib.Simulator(f, P, 3, H, W)
    img = cu(synthetic.shapes(H, W, 3, seed=2))
    sim.stage_timing(3)
    with pytest.raises(lib.DFP2SError):
        sim.stage_times(1)  # nothing recorded yet
    for i in range(5):
        sim.simulate_frame(img, 2.0, 1, i, lib.P2S_EXACT)
    t = sim.stage_times(3)
    assert t.shape == (3, 4) and np.all(t > 0) and np.all(t < 1e3)
    with pytest.raises(lib.DFP2SError):
        sim.stage_times(4)  # beyond the ring
    sim.stage_timing(0)
    sim.simulate_frame(img, 2.0, 1, 9, lib.P2S_EXACT)
    with pytest.raises(lib.DFP2SError):
        sim.stage_times(1)


def test_simulate_frame_exact_small_workload(lib):
    J, K, H, W, N, d = 36, 16, 64, 64, 128, 2.0
    img = synthetic.smooth_noise(H, W, seed=0)
    basis = p2s.build_basis(0, J, K, 2000, [d])
    f = lib.SpectralFactor(J, N, 8.0)
    P = lib.P2S(J, cu(basis))
    sim = lib.Simulator(f, P, 1, H, W)
    g = sim.simulate_frame(cu(img), d, 0, 0, lib.P2S_EXACT).cpu().numpy()
    o = __import__("oracle.frame", fromlist=["x"]).simulate_frame(img, d, 0, 0, J, basis, 8.0, N)
    assert rel_l2(g, o["out"]) < TOL


def test_exact_frame_full_size_sampled(lib):
    # the 512 x 512 x 3 workload (J = 36, N = 1024, K = 100) in the frame call the bench times (exact P2S and the
    # FP32 blur), against the oracle at sampled pixels: corners, edges and interior, each from the oracle's fields,
    # warp, per-pixel pupil-FFT weights and the blur sum written out over the 33 x 33 window
    from oracle import image as oimage
    J, K, H, W, N, d, seed, frame = 36, 100, 512, 512, 1024, 2.0, 17, 3
    img = synthetic.shapes(H, W, 3, seed=5)
    basis = synthetic.random_orthonormal_rows(K, 33 * 33, seed=2).reshape(K, 33, 33)
    f = lib.SpectralFactor(J, N, 8.0)
    P = lib.P2S(J, cu(basis))
    sim = lib.Simulator(f, P, 3, H, W)
    g = sim.simulate_frame(cu(img), d, seed, frame, lib.P2S_EXACT).cpu().numpy()
    a = sampler.sample_fields(seed, frame, J, H, W, d, 8.0, N)
    warped = oimage.tilt_warp(img, a[0], a[1])
    rng = np.random.default_rng(0)
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (5, 300), (300, 7), (H - 3, 200), (128, W - 2)]
    pts += [tuple(p) for p in rng.integers(0, [H, W], size=(24, 2))]
    u = np.arange(-16, 17)
    got, ref = [], []
    for y, x in pts:
        w = p2s.weights(a[:, y, x], J, basis)  # K
        win = warped[:, np.clip(y - u, 0, H - 1)][:, :, np.clip(x - u, 0, W - 1)]  # C x 33 x 33: I(y - uy, x - ux)
        h = np.tensordot(w, basis, axes=1)  # the pixel's PSF, 33 x 33 over (uy, ux)
        ref.append((win * h[None]).sum(axis=(1, 2)))
        got.append(g[:, y, x])
    assert rel_l2(np.array(got), np.array(ref)) < TOL


def test_bad_arguments_return_einval(lib):
    f = lib.SpectralFactor(6, 16, 2.0)
    with pytest.raises(lib.DFP2SError) as e:
        lib.sample_zernike_fields(f, 1.0, 0, 0, 17, 8)  # larger than the grid
    assert e.value.code == -1
    with pytest.raises(lib.DFP2SError):
        lib.SpectralFactor(6, 100, 2.0)  # not a power of two
    basis = torch.zeros(4, 33, 33, device="cuda")
    P = lib.P2S(6, basis)
    with pytest.raises(lib.DFP2SError):
        lib.p2s_weights(P, lib.P2S_LEARNED, torch.zeros(6, 4, 4, device="cuda"))  # no network installed
