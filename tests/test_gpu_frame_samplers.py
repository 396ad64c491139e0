"""Frames whose fields come from the dense per-frequency root or from the full cross-spectral density
(dfp2s_ctx_set_field_sampler): each frame equals the composition of the entry points it is made of, bit for bit."""
import numpy as np
import pytest
import torch

from inputs import synthetic
from oracle import p2s

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_06713_gb300 as d
    d.load()
    return d


def _p2s(lib, J, K=16):
    basis = p2s.build_basis(0, J, K, 200, [1.0, 3.0])
    P = lib.P2S(J, torch.as_tensor(basis, dtype=torch.float32, device="cuda"))
    rng = np.random.default_rng(3)
    cu = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float32), device="cuda")
    P.set_mlp(cu(rng.standard_normal((256, J)) / 6), cu(np.zeros(256)), cu(rng.standard_normal((256, 256)) / 16),
              cu(np.zeros(256)), cu(rng.standard_normal((K, 256)) / 16), cu(np.zeros(K)),
              cu(np.r_[0.0, 0.0, np.ones(J - 2)]), cu(np.full(K, 0.02)), cu(p2s.weights(np.zeros(J), J, basis)))
    return P


@pytest.mark.parametrize("kind,sampler", [("FACTOR_FULL", "FIELDS_FULL"), ("FACTOR_DENSE", "FIELDS_DENSE")])
def test_frames_equal_their_composition(lib, kind, sampler):
    J, C, H, W, dr = 36, 3, 96, 80, 2.5
    f = lib.SpectralFactor(J, 128, 8.0, kind=getattr(lib, kind))
    P = _p2s(lib, J)
    sim = lib.Simulator(f, P, C, H, W)
    sim.set_field_sampler(getattr(lib, sampler))
    img = torch.as_tensor(synthetic.shapes(H, W, C, seed=2), device="cuda")
    fields = (lib.sample_zernike_fields_full if sampler == "FIELDS_FULL" else lib.sample_zernike_fields_dense)(
        f, dr, 7, 1, H, W)
    warped = lib.tilt_warp(img, fields[0], fields[1])
    # exact: fields -> warp -> exact weights -> FP32 blur
    w = lib.p2s_weights(P, lib.P2S_EXACT, fields)
    want = lib.basis_blur(P, warped, w)
    assert torch.equal(sim.simulate_frame(img, dr, 7, 1, lib.P2S_EXACT), want)
    # learned: the network's own first layer on the mixed fields, the tensor-core blur of the warped image
    wl = lib.p2s_weights(P, lib.P2S_LEARNED, fields)
    want_l = lib.basis_blur_tc(P, warped, wl)
    got_l = sim.simulate_frame(img, dr, 7, 1, lib.P2S_LEARNED)
    P.check()
    assert torch.equal(got_l, want_l)
    # and the factored sampler is still the default of a new context
    sim2 = lib.Simulator(f, P, C, H, W)
    a = sim2.simulate_frame(img, dr, 7, 1, lib.P2S_EXACT)
    assert not torch.equal(a, want)


def test_sampler_needs_its_factor(lib):
    f = lib.SpectralFactor(12, 64, 8.0)
    sim = lib.Simulator(f, _p2s(lib, 12), 1, 16, 16)
    with pytest.raises(lib.DFP2SError):
        sim.set_field_sampler(lib.FIELDS_FULL)
    with pytest.raises(lib.DFP2SError):
        sim.set_field_sampler(lib.FIELDS_DENSE)
    with pytest.raises(lib.DFP2SError):
        sim.set_field_sampler(7)
    sim.set_field_sampler(lib.FIELDS_FACTORED)
