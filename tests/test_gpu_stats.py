"""Field statistics on the GPU (Sec. III-D, Eq. A tilde): the lagged-covariance kernel against the oracle on
the same fields, and the GPU sampler's averaged covariances against A~(s)."""
import numpy as np
import pytest
import torch

from inputs import synthetic
from oracle import stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2210_06713_gb300 as d
    return d


@pytest.mark.parametrize("J,H,W", [
    (36, 50, 37),
    (3, 300, 211),   # one register tile per pixel group, 28 groups per CTA; many runs per CTA
    (15, 130, 97),   # tiles cut by J
    (64, 40, 33),    # the largest J: 121 threads per group, two groups
])
def test_covariance_matches_oracle(lib, J, H, W):
    a = synthetic.random_fields(J, H, W, scale=0.7, seed=4)
    lags = [(0, 0), (1, 0), (0, 1), (-3, 2), (7, -5), (H - 1, W - 1)]
    g = lib.field_covariance(torch.as_tensor(a, dtype=torch.float32, device="cuda"), lags).cpu().numpy()
    o = stats.field_covariance(a.astype(np.float32), lags)
    assert np.linalg.norm(g - o) / np.linalg.norm(o) < 1e-6
    for l in range(len(lags)):
        assert np.allclose(g[l], o[l], rtol=1e-5, atol=1e-7 * np.abs(o[l]).max())
    with pytest.raises(lib.DFP2SError):
        lib.field_covariance(torch.zeros(J, H, W, device="cuda"), [(H, 0)])


def test_gpu_sampler_reaches_a_tilde(lib):
    J, H, W, N, ppd, d = 10, 32, 32, 64, 8.0, 2.0
    lags = [(0, 0), (0, 1), (3, 0), (-4, 5)]
    f = lib.SpectralFactor(J, N, ppd)
    per = []
    for fr in range(300):
        a = lib.sample_zernike_fields(f, d, 21, fr, H, W)
        per.append(lib.field_covariance(a, lags))
    per = torch.stack(per).cpu().numpy()
    mean, se = per.mean(0), per.std(0, ddof=1) / np.sqrt(per.shape[0])
    target = stats.approx_covariance(J, N, ppd, d, lags)
    assert np.all(np.abs(mean - target) <= 5 * se + 1e-9)
