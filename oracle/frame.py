"""One simulated frame, step by step (Fig. dfp2s and the two-step recipe of Sec. III).

Test infrastructure only (see the package docstring).

Step 1 (Sec. III-C): correlated Zernike fields from the FFT sampler.
Step 2 (Sec. II-C, Eq. varying blur): tilt warp from fields 0, 1 (Noll 2, 3),
then per-pixel P2S weights (exact pupil-FFT projection, or the surrogate MLP)
and the basis blur.
"""
from __future__ import annotations

import numpy as np

from . import image, mlp, p2s, sampler


def simulate_frame(img: np.ndarray, D_over_r0: float, seed: int, frame: int, J: int,
                   basis: np.ndarray, pix_per_D: float = 8.0, N: int | None = None,
                   net: dict | None = None) -> dict:
    """Returns dict(fields, warped, weights, out).  net = None -> exact P2S, else the MLP
    (net holds params, in_scale, out_scale, out_shift)."""
    C, H, W = img.shape
    a = sampler.sample_fields(seed, frame, J, H, W, D_over_r0, pix_per_D, N)
    warped = image.tilt_warp(img, a[0], a[1])
    if net is None:
        w = p2s.weights_field(a, basis)
    else:
        av = np.moveaxis(a, 0, -1)
        w = mlp.predict_weights(net["params"], av, net["in_scale"], net["out_scale"], net["out_shift"],
                                flux=p2s.flux_vector(basis))
    out = image.basis_blur(warped, w, basis)
    return {"fields": a, "warped": warped, "weights": w, "out": out}
