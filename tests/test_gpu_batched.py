"""Batched, uneven requests (the mixed-size workload): frames of different sizes, D/r0 and J served
by simulators that share one spectral factor per (J, N) and one basis per J, each frame against the
oracle's frame."""
import numpy as np
import pytest
import torch

from inputs import synthetic
from oracle import frame as oframe
from oracle import p2s, sampler

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_06713_gb300 as d
    d.load()
    return d


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_uneven_requests_match_oracle(lib):
    rng = np.random.default_rng(17)
    # (H, W, C, J): sizes and mode counts vary request to request, two frames each
    requests = [(24, 32, 3, 15), (40, 24, 1, 36), (33, 17, 3, 36), (16, 48, 2, 15), (20, 20, 3, 36)]
    K = 16
    bases = {J: p2s.build_basis(0, J, K, 300, [1.0, 3.0, 5.0]) for J in (15, 36)}
    factors, sims = {}, {}
    for r, (H, W, C, J) in enumerate(requests):
        N = sampler.grid_size(H, W)
        key = (J, N)
        if key not in factors:
            factors[key] = lib.SpectralFactor(J, N, 8.0)
            sims[key] = lib.Simulator(factors[key], lib.P2S(J, torch.as_tensor(bases[J], dtype=torch.float32,
                                                                                  device="cuda")), 3, 48, 48)
        img = synthetic.shapes(H, W, C, seed=r)
        for fr in range(2):
            dr = float(rng.uniform(1.0, 5.0))
            g = sims[key].simulate_frame(torch.as_tensor(img, device="cuda"), dr, 100 + r, fr,
                                         lib.P2S_EXACT).cpu().numpy()
            o = oframe.simulate_frame(img, dr, 100 + r, fr, J, bases[J], 8.0, N)["out"]
            assert _rel(g, o) < TOL, (r, fr, H, W, J)
