"""The learned frame against the exact frame at the full 512 x 512 x 3 workload.

The surrogate network (Sec. II-C; J -> 256 -> 256 -> K, trained on the device on
2^20 exact-P2S pairs pooled over D/r0 = 1, 2, 4 for 60000 Adam steps, as the
benchmark trains it)
with its BF16 tensor-core inference and the BF16 tensor-core blur must give a
frame within 2e-3 rel-L2 of the exact-P2S FP32 frame at every D/r0 of the
workload, on frames of the same seeded fields and image.
"""
import numpy as np
import pytest
import torch

from inputs import synthetic

pytestmark = pytest.mark.gpu

TOL = 2e-3  # learned BF16 frame against the exact FP32 frame


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_06713_gb300 as lib
    lib.load()
    J, K, H, W, C = 36, 100, 512, 512, 3
    drs = (1.0, 2.0, 4.0)
    f = lib.SpectralFactor(J, lib.grid_size(H, W, 8.0), 8.0)
    basis, _, _ = lib.build_basis(f, K, 2000, drs, seed=0)
    P = lib.P2S(J, basis)
    lib.mlp_train(P, f, n_pairs=1 << 20, D_over_r0=drs, seed=1, batch=2048, steps=60000, lr=2e-3)
    img = torch.as_tensor(synthetic.shapes(H, W, C, seed=0), device="cuda")
    sim = lib.Simulator(f, P, C, H, W)
    return lib, P, sim, img, basis


@pytest.mark.parametrize("d", [1.0, 2.0, 4.0])
def test_learned_frame_within_tolerance_of_exact_frame(trained, d):
    lib, P, sim, img, _ = trained
    errs = []
    for seed, frame in ((77, 0), (5, 3)):
        ex = sim.simulate_frame(img, d, seed, frame, lib.P2S_EXACT).double()
        le = sim.simulate_frame(img, d, seed, frame, lib.P2S_LEARNED).double()
        P.check()
        errs.append(float((le - ex).norm() / ex.norm()))
    assert max(errs) <= TOL, errs


def test_learned_and_exact_weights_keep_unit_flux(trained):
    # both P2S forms return weights whose PSF keeps unit sum: s^T w = 1, s_k = sum_u phi_k(u) (reading R28)
    lib, P, sim, img, basis = trained
    s = basis.double().sum(dim=(1, 2))
    f = lib.sample_zernike_fields(sim.factor, 4.0, 9, 0, 128, 96)
    for mode in (lib.P2S_EXACT, lib.P2S_LEARNED, lib.P2S_LEARNED_FP32):
        w = lib.p2s_weights(P, mode, f).reshape(-1, P.K).double()
        P.check()
        assert (w @ s - 1.0).abs().max().item() < 2e-5, mode
