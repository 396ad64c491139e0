"""Python binding of libdfp2s, the GB300 (sm_103a) DF-P2S turbulence simulator.

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of ``csrc/`` behind the C ABI declared in ``include/dfp2s.h``.
PyTorch supplies device memory and the current stream.  There is no host
fallback: a missing library or a missing GPU raises.

The names follow the C ABI: build_spectral_factor, sample_zernike_fields,
p2s_weights, tilt_warp, basis_blur, simulate_frame (plus handles).
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

OK = 0
W_F32, W_BF16 = 0, 1
P2S_EXACT, P2S_LEARNED, P2S_LEARNED_FP32 = 0, 1, 2
FACTOR_FACTORED, FACTOR_DENSE, FACTOR_FULL = 0, 1, 2
FIELDS_FACTORED, FIELDS_DENSE, FIELDS_FULL = 0, 1, 2
KS = 33
MAX_J = 64
MAX_K = 128

# every entry point declared in include/dfp2s.h, with its ctypes signature
_c = ctypes
_vp, _i, _u32, _u64, _d, _sz = _c.c_void_p, _c.c_int, _c.c_uint32, _c.c_uint64, _c.c_double, _c.c_size_t


class FactorParams(ctypes.Structure):
    _fields_ = [("J", _i), ("N", _i), ("pix_per_D", _d), ("kind", _i), ("subharmonic_levels", _i)]


class TrainParams(ctypes.Structure):
    _fields_ = [("n_pairs", _i), ("n_dr", _i), ("D_over_r0", _d * 8), ("seed", _u64), ("batch", _i), ("steps", _i),
                ("lr", _c.c_float), ("psf_weighted_loss", _i), ("val_fraction", _c.c_float),
                ("image_prior_loss", _i)]


class Request(ctypes.Structure):
    _fields_ = [("img_dev", _vp), ("C", _i), ("H", _i), ("W", _i), ("J", _i), ("D_over_r0", _d), ("seed", _u64),
                ("first_frame", _u32), ("n_frames", _i), ("p2s_mode", _i), ("out_dev", _vp)]


ENGINE_GRAPHS, ENGINE_AUTOTUNE = 1, 2

SIGNATURES = {
    "dfp2s_last_error": (_i, [_c.c_char_p, _sz]),
    "dfp2s_version": (_c.c_char_p, []),
    "dfp2s_grid_size": (_i, [_i, _i, _d]),
    "dfp2s_build_spectral_factor": (_i, [_c.POINTER(FactorParams), _c.POINTER(_vp), _vp]),
    "dfp2s_factor_destroy": (_i, [_vp]),
    "dfp2s_factor_copy_multiplier": (_i, [_vp, _vp, _vp]),
    "dfp2s_factor_copy_cholesky": (_i, [_vp, _vp]),
    "dfp2s_factor_info": (_i, [_vp, _c.POINTER(_i), _c.POINTER(_i), _c.POINTER(_sz)]),
    "dfp2s_sample_zernike_fields": (_i, [_vp, _d, _u64, _u32, _i, _i, _vp, _vp]),
    "dfp2s_sample_zernike_fields_ar1": (_i, [_vp, _d, _u64, _u32, _d, _i, _i, _vp, _vp, _vp]),
    "dfp2s_sample_zernike_fields_full": (_i, [_vp, _d, _u64, _u32, _i, _i, _vp, _vp]),
    "dfp2s_ctx_set_field_sampler": (_i, [_vp, _i]),
    "dfp2s_ctx_set_field_variant": (_i, [_vp, _i]),
    "dfp2s_sample_zernike_fields_dense": (_i, [_vp, _d, _u64, _u32, _i, _i, _vp, _vp]),
    "dfp2s_factor_copy_dense_root": (_i, [_vp, _vp, _vp]),
    "dfp2s_aperture_statistics": (_i, [_vp, _i, _i, _i, _i, _vp, _vp]),
    "dfp2s_tilt_statistics": (_i, [_vp, _i, _i, _i, _vp, _vp]),
    "dfp2s_sample_zernike_fields_noalloc": (_i, [_vp, _d, _u64, _u32, _i, _i, _vp, _vp]),
    "dfp2s_gaussian_noise": (_i, [_u64, _u32, _u32, _u32, _i, _i, _vp, _vp]),
    "dfp2s_philox_words": (_i, [_u64, _u64, _u64, _i, _vp, _vp]),
    "dfp2s_check_bounded_wait": (_i, [_u64, _vp]),
    "dfp2s_debug_fail_allocation": (_i, [_i]),
    "dfp2s_build_basis": (_i, [_vp, _i, _i, _vp, _i, _u64, _vp, _vp, _vp, _vp]),
    "dfp2s_p2s_create": (_i, [_i, _i, _vp, _c.POINTER(_vp)]),
    "dfp2s_p2s_destroy": (_i, [_vp]),
    "dfp2s_p2s_check": (_i, [_vp]),
    "dfp2s_p2s_set_mlp": (_i, [_vp] + [_vp] * 9),
    "dfp2s_mlp_save": (_i, [_vp, _c.c_char_p]),
    "dfp2s_field_covariance": (_i, [_vp, _i, _i, _i, _vp, _i, _vp, _vp]),
    "dfp2s_mlp_load": (_i, [_vp, _c.c_char_p]),
    "dfp2s_mlp_train": (_i, [_vp, _vp, _c.POINTER(TrainParams), _vp, _vp, _vp]),
    "dfp2s_mlp_param_count": (_i, [_i, _i]),
    "dfp2s_mlp_loss_grad": (_i, [_i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "dfp2s_mlp_image_prior_gram": (_i, [_vp, _vp, _vp, _vp]),
    "dfp2s_p2s_weights": (_i, [_vp, _i, _vp, _i, _i, _vp, _i, _vp]),
    "dfp2s_tilt_warp": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "dfp2s_basis_blur": (_i, [_vp, _vp, _i, _i, _i, _vp, _i, _vp, _vp]),
    "dfp2s_basis_blur_tc": (_i, [_vp, _vp, _i, _i, _i, _vp, _i, _vp, _vp]),
    "dfp2s_basis_blur_tc_prepare": (_i, [_vp, _vp, _i, _i, _i, _vp]),
    "dfp2s_tilt_warp_blur_tc_prepare": (_i, [_vp, _vp, _i, _i, _i, _vp, _vp, _vp]),
    "dfp2s_basis_blur_tc_run": (_i, [_vp, _i, _i, _i, _vp, _i, _vp, _vp]),
    "dfp2s_ctx_create": (_i, [_vp, _vp, _i, _i, _i, _c.POINTER(_vp)]),
    "dfp2s_ctx_destroy": (_i, [_vp]),
    "dfp2s_simulate_frame": (_i, [_vp, _vp, _i, _i, _i, _d, _u64, _u32, _i, _vp, _vp]),
    "dfp2s_ctx_buffers": (_i, [_vp, _c.POINTER(_vp), _c.POINTER(_vp), _c.POINTER(_vp)]),
    "dfp2s_ctx_stage_timing": (_i, [_vp, _i]),
    "dfp2s_ctx_stage_times": (_i, [_vp, _i, _vp]),
    "dfp2s_engine_create": (_i, [_c.POINTER(_vp), _i, _d, _i, _c.POINTER(_vp)]),
    "dfp2s_engine_run": (_i, [_vp, _c.POINTER(Request), _i, _vp]),
    "dfp2s_engine_info": (_i, [_vp, _c.POINTER(_i), _vp]),
    "dfp2s_engine_class_info": (_i, [_vp, _i, _vp, _vp]),
    "dfp2s_engine_destroy": (_i, [_vp]),
}

_LIB = None


class DFP2SError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dfp2s error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libdfp2s.so (building it first if needed); raises if that is impossible."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_build.LIB) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"libdfp2s is not built ({_build.LIB}); run paper_2210_06713_gb300.build")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(rc: int):
    if rc != OK:
        buf = ctypes.create_string_buffer(512)
        load().dfp2s_last_error(buf, 512)
        raise DFP2SError(rc, buf.value.decode(errors="replace"))


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: torch.Tensor):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def grid_size(H: int, W: int, pix_per_D: float = 8.0) -> int:
    n = load().dfp2s_grid_size(H, W, pix_per_D)
    if n < 0:
        _check(n)
    return n


# ------------------------------------------------------------------ factor
class SpectralFactor:
    """Spectral factor of the homogeneous tensor approximation for (J, N, pix_per_D)."""

    def __init__(self, J: int, N: int, pix_per_D: float = 8.0, kind: int = FACTOR_FACTORED, stream=None,
                 subharmonics: int = 0):
        lib = load()
        self.J, self.N, self.pix_per_D, self.kind, self.subharmonics = J, N, pix_per_D, kind, subharmonics
        h = ctypes.c_void_p()
        p = FactorParams(J, N, pix_per_D, kind, subharmonics)
        _check(lib.dfp2s_build_spectral_factor(ctypes.byref(p), ctypes.byref(h), _stream(stream)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def multiplier(self) -> torch.Tensor:
        out = torch.empty(self.J, self.N // 2 + 1, self.N, dtype=torch.float32, device="cuda")
        _check(load().dfp2s_factor_copy_multiplier(self._h, _ptr(out), _stream()))
        torch.cuda.current_stream().synchronize()
        return out

    def cholesky(self):
        import numpy as np
        L = np.empty((self.J, self.J), dtype=np.float64)
        _check(load().dfp2s_factor_copy_cholesky(self._h, L.ctypes.data_as(ctypes.c_void_p)))
        return L

    def scratch_bytes(self) -> int:
        s = ctypes.c_size_t()
        _check(load().dfp2s_factor_info(self._h, None, None, ctypes.byref(s)))
        return s.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dfp2s_factor_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_spectral_factor(J: int, N: int, pix_per_D: float = 8.0, kind: int = FACTOR_FACTORED) -> SpectralFactor:
    return SpectralFactor(J, N, pix_per_D, kind)


def sample_zernike_fields(factor: SpectralFactor, D_over_r0: float, seed: int, frame: int, H: int, W: int,
                          out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(factor.J, H, W, dtype=torch.float32, device="cuda")
    _check(load().dfp2s_sample_zernike_fields(factor.handle, D_over_r0, seed, frame, H, W, _ptr(out),
                                              _stream(stream)))
    return out


def sample_zernike_fields_full(factor: SpectralFactor, D_over_r0: float, seed: int, frame: int, H: int, W: int,
                               out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Fields of the full cross-spectral density (no approximation); the factor needs kind=FACTOR_FULL."""
    if out is None:
        out = torch.empty(factor.J, H, W, dtype=torch.float32, device="cuda")
    _check(load().dfp2s_sample_zernike_fields_full(factor.handle, D_over_r0, seed, frame, H, W, _ptr(out),
                                                   _stream(stream)))
    return out


def sample_zernike_fields_dense(factor: SpectralFactor, D_over_r0: float, seed: int, frame: int, H: int, W: int,
                                out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Fields from the per-frequency symmetric root of L diag(lambda) L^T; the factor needs kind=FACTOR_DENSE."""
    if out is None:
        out = torch.empty(factor.J, H, W, dtype=torch.float32, device="cuda")
    _check(load().dfp2s_sample_zernike_fields_dense(factor.handle, D_over_r0, seed, frame, H, W, _ptr(out),
                                                    _stream(stream)))
    return out


def dense_root(factor: SpectralFactor, stream=None) -> torch.Tensor:
    """F of a FACTOR_DENSE factor: (J, J, N/2+1, N) float32, [j, i, kx, ky], D/r0 = 1."""
    J, N = factor.J, factor.N
    out = torch.empty(J, J, N // 2 + 1, N, dtype=torch.float32, device="cuda")
    _check(load().dfp2s_factor_copy_dense_root(factor.handle, _ptr(out), _stream(stream)))
    return out


def sample_zernike_fields_ar1(factor: SpectralFactor, D_over_r0: float, seed: int, frame: int, alpha: float,
                              H: int, W: int, prev: torch.Tensor | None, out: torch.Tensor | None = None,
                              stream=None) -> torch.Tensor:
    """Temporally correlated fields: alpha * prev + sqrt(1 - alpha^2) * (this frame's fields); prev None for
    the first frame."""
    if out is None:
        out = torch.empty(factor.J, H, W, dtype=torch.float32, device="cuda")
    _check(load().dfp2s_sample_zernike_fields_ar1(factor.handle, D_over_r0, seed, frame, alpha, H, W,
                                                  _ptr(prev) if prev is not None else None, _ptr(out),
                                                  _stream(stream)))
    return out


def sample_zernike_fields_noalloc(factor: SpectralFactor, D_over_r0: float, seed: int, frame: int, H: int, W: int,
                                  out: torch.Tensor, stream=None) -> torch.Tensor:
    """sample_zernike_fields without any device allocation (static library scratch; see include/dfp2s.h)."""
    _check(load().dfp2s_sample_zernike_fields_noalloc(factor.handle, D_over_r0, seed, frame, H, W, _ptr(out),
                                                      _stream(stream)))
    return out


def gaussian_noise(seed: int, tag: int, frame: int, mode: int, rows: int, cols: int) -> torch.Tensor:
    out = torch.empty(rows, cols, dtype=torch.float32, device="cuda")
    _check(load().dfp2s_gaussian_noise(seed, tag, frame, mode, rows, cols, _ptr(out), _stream()))
    return out


def philox_words(seed: int, sub: int, q0: int, n: int) -> torch.Tensor:
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(load().dfp2s_philox_words(seed, sub, q0, n, _ptr(out), _stream()))
    return out


def build_basis(factor: SpectralFactor, K: int, n_psf: int = 2000, D_over_r0=(2.0,), seed: int = 0):
    """Top-K SVD basis of n_psf exact PSFs (device FP64); returns (basis K x 33 x 33, singular values, sweeps)."""
    import numpy as np
    basis = torch.empty(K, KS, KS, dtype=torch.float32, device="cuda")
    dr = np.asarray(D_over_r0, dtype=np.float64)
    sig = np.zeros(KS * KS, dtype=np.float64)
    sweeps = ctypes.c_int(0)
    _check(load().dfp2s_build_basis(factor.handle, K, n_psf, dr.ctypes.data_as(ctypes.c_void_p), len(dr), seed,
                                    _ptr(basis), sig.ctypes.data_as(ctypes.c_void_p), ctypes.byref(sweeps), _stream()))
    return basis, sig, sweeps.value


# --------------------------------------------------------------------- P2S
class P2S:
    """PSF basis (K x 33 x 33) and optional surrogate network."""

    def __init__(self, J: int, basis: torch.Tensor):
        lib = load()
        basis = basis.to(device="cuda", dtype=torch.float32).contiguous()
        self.J, self.K = J, basis.shape[0]
        h = ctypes.c_void_p()
        _check(lib.dfp2s_p2s_create(J, self.K, _ptr(basis), ctypes.byref(h)))
        self._h = h
        self.has_mlp = False

    @property
    def handle(self):
        return self._h

    def set_mlp(self, W1, b1, W2, b2, W3, b3, in_scale, out_scale, out_shift):
        ts = [torch.as_tensor(t, dtype=torch.float32, device="cuda").contiguous()
              for t in (W1, b1, W2, b2, W3, b3, in_scale, out_scale, out_shift)]
        _check(load().dfp2s_p2s_set_mlp(self._h, *[_ptr(t) for t in ts]))
        self.has_mlp = True

    def save_mlp(self, path: str) -> None:
        """Write the installed network to a file (include/dfp2s.h: dfp2s_mlp_save)."""
        _check(load().dfp2s_mlp_save(self._h, os.fsencode(path)))

    def load_mlp(self, path: str) -> None:
        """Install the network stored in a file by save_mlp."""
        _check(load().dfp2s_mlp_load(self._h, os.fsencode(path)))
        self.has_mlp = True

    def check(self):
        """Raises DFP2SError(-4) if a tensor-core kernel of this handle gave up on a bounded wait."""
        _check(load().dfp2s_p2s_check(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dfp2s_p2s_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_param_count(J: int, K: int) -> int:
    n = load().dfp2s_mlp_param_count(J, K)
    if n < 0:
        _check(n)
    return n


def mlp_loss_grad(params: torch.Tensor, X: torch.Tensor, T: torch.Tensor, lw: torch.Tensor | None = None,
                  G: torch.Tensor | None = None):
    """Loss and flat gradient of the surrogate on one batch (device FP32 tensors); G (K x K) selects the
    quadratic-form loss, else the per-k weights lw."""
    B, J = X.shape
    K = T.shape[1]
    grads = torch.empty_like(params)
    loss = torch.zeros(1, device="cuda")
    _check(load().dfp2s_mlp_loss_grad(J, K, B, _ptr(params), _ptr(X), _ptr(T), _ptr(lw) if lw is not None else None,
                                      _ptr(G) if G is not None else None, _ptr(grads), _ptr(loss), _stream()))
    return float(loss.item()), grads


def mlp_image_prior_gram(p: P2S, sd: torch.Tensor) -> torch.Tensor:
    """The training loss's K x K form for the basis of `p` and weight standard deviations `sd` (device)."""
    G = torch.empty(p.K, p.K, dtype=torch.float32, device="cuda")
    _check(load().dfp2s_mlp_image_prior_gram(p.handle, _ptr(sd), _ptr(G), _stream()))
    return G


def mlp_train(p: P2S, factor: SpectralFactor, n_pairs: int = 1 << 20, D_over_r0=(1.0, 2.0, 4.0), seed: int = 0,
              batch: int = 2048, steps: int = 20000, lr: float = 2e-3, psf_weighted_loss: bool = True,
              val_fraction: float = 0.05, return_params: bool = False, image_prior_loss: bool = True):
    """Trains the surrogate on the device and installs it in `p`; returns a report dict."""
    import numpy as np
    tp = TrainParams()
    tp.n_pairs, tp.n_dr = n_pairs, len(D_over_r0)
    for i, dval in enumerate(D_over_r0):
        tp.D_over_r0[i] = dval
    tp.seed, tp.batch, tp.steps, tp.lr = seed, batch, steps, lr
    tp.psf_weighted_loss, tp.val_fraction = int(psf_weighted_loss), val_fraction
    tp.image_prior_loss = int(image_prior_loss)
    rep = np.zeros(3, dtype=np.float32)
    params = np.zeros(mlp_param_count(p.J, p.K), dtype=np.float32) if return_params else None
    _check(load().dfp2s_mlp_train(p.handle, factor.handle, ctypes.byref(tp), rep.ctypes.data_as(ctypes.c_void_p),
                                  params.ctypes.data_as(ctypes.c_void_p) if return_params else None, _stream()))
    p.has_mlp = True
    out = {"final_loss": float(rep[0]), "val_weight_rel_l2": float(rep[1]), "steps": int(rep[2])}
    if return_params:
        out["params"] = params
    return out


def p2s_weights(p: P2S, mode: int, fields: torch.Tensor, w_dtype: int = W_F32, out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    J, H, W = fields.shape
    if out is None:
        out = torch.empty(H, W, p.K, dtype=torch.float32 if w_dtype == W_F32 else torch.bfloat16, device="cuda")
    _check(load().dfp2s_p2s_weights(p.handle, mode, _ptr(fields), H, W, _ptr(out), w_dtype, _stream(stream)))
    return out


def field_covariance(fields: torch.Tensor, lags, stream=None) -> torch.Tensor:
    """Lagged covariances (n_lags x J x J, float64, device) of J x H x W fields; lags = [(dy, dx), ...]."""
    J, H, W = fields.shape
    flat = (ctypes.c_int * (2 * len(lags)))(*[int(v) for lag in lags for v in lag])
    out = torch.empty(len(lags), J, J, device=fields.device, dtype=torch.float64)
    _check(load().dfp2s_field_covariance(_ptr(fields), J, H, W, ctypes.cast(flat, ctypes.c_void_p), len(lags),
                                         _ptr(out), _stream(stream)))
    return out


def aperture_statistics(fields: torch.Tensor, step: int = 1, stream=None):
    """Structure function and LE / SE OTFs of the sub-grid pixels' Zernike vectors (include/dfp2s.h): a dict of
    float64 device tensors D_x, D_y (33), H_LE, H_SE (64 x 64, FFT order)."""
    J, H, W = fields.shape
    out = torch.empty(2 * 33 + 2 * 64 * 64, device=fields.device, dtype=torch.float64)
    _check(load().dfp2s_aperture_statistics(_ptr(fields), J, H, W, step, _ptr(out), _stream(stream)))
    return {"D_x": out[:33], "D_y": out[33:66], "H_LE": out[66:66 + 4096].view(64, 64),
            "H_SE": out[66 + 4096:].view(64, 64)}


def tilt_statistics(fields: torch.Tensor, max_lag: int, stream=None) -> torch.Tensor:
    """Tilt correlation and DTV window means (2 x (max_lag+1) x 8, float64, device) of the first two planes."""
    _, H, W = fields.shape
    out = torch.empty(2, max_lag + 1, 8, device=fields.device, dtype=torch.float64)
    _check(load().dfp2s_tilt_statistics(_ptr(fields), H, W, max_lag, _ptr(out), _stream(stream)))
    return out


def tilt_warp(img: torch.Tensor, a2: torch.Tensor, a3: torch.Tensor, out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
    C, H, W = img.shape
    if out is None:
        out = torch.empty_like(img)
    _check(load().dfp2s_tilt_warp(_ptr(img), C, H, W, _ptr(a2), _ptr(a3), _ptr(out), _stream(stream)))
    return out


def basis_blur(p: P2S, img: torch.Tensor, w: torch.Tensor, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    C, H, W = img.shape
    if out is None:
        out = torch.empty_like(img)
    wdt = W_BF16 if w.dtype == torch.bfloat16 else W_F32
    _check(load().dfp2s_basis_blur(p.handle, _ptr(img), C, H, W, _ptr(w), wdt, _ptr(out), _stream(stream)))
    return out


def basis_blur_tc(p: P2S, img: torch.Tensor, w: torch.Tensor, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """Tensor-core (BF16 operands, FP32 accumulation) blur with FP32 or BF16 weights."""
    C, H, W = img.shape
    if out is None:
        out = torch.empty_like(img)
    wdt = W_BF16 if w.dtype == torch.bfloat16 else W_F32
    _check(load().dfp2s_basis_blur_tc(p.handle, _ptr(img), C, H, W, _ptr(w), wdt, _ptr(out), _stream(stream)))
    return out


def basis_blur_tc_prepare(p: P2S, img: torch.Tensor, stream=None) -> None:
    """First step of basis_blur_tc: the image's shifted BF16 operand, kept in the handle."""
    C, H, W = img.shape
    _check(load().dfp2s_basis_blur_tc_prepare(p.handle, _ptr(img), C, H, W, _stream(stream)))


def tilt_warp_blur_tc_prepare(p: P2S, img: torch.Tensor, a2: torch.Tensor, a3: torch.Tensor, stream=None) -> None:
    """tilt_warp fused with basis_blur_tc_prepare (the warped image itself is not written)."""
    C, H, W = img.shape
    _check(load().dfp2s_tilt_warp_blur_tc_prepare(p.handle, _ptr(img), C, H, W, _ptr(a2), _ptr(a3),
                                                  _stream(stream)))


def basis_blur_tc_run(p: P2S, shape, w: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Second step of basis_blur_tc: the contraction on the image prepared for `shape` = (C, H, W)."""
    C, H, W = shape
    if out is None:
        out = torch.empty(C, H, W, device=w.device, dtype=torch.float32)
    wdt = W_BF16 if w.dtype == torch.bfloat16 else W_F32
    _check(load().dfp2s_basis_blur_tc_run(p.handle, C, H, W, _ptr(w), wdt, _ptr(out), _stream(stream)))
    return out


# ------------------------------------------------------------------ frames
class Simulator:
    """A frame context: factor + P2S handle + per-frame scratch (Fig. dfp2s)."""

    def __init__(self, factor: SpectralFactor, p2s: P2S, max_C: int, max_H: int, max_W: int):
        h = ctypes.c_void_p()
        _check(load().dfp2s_ctx_create(factor.handle, p2s.handle, max_C, max_H, max_W, ctypes.byref(h)))
        self._h = h
        self.factor, self.p2s = factor, p2s
        self.max_shape = (max_C, max_H, max_W)

    def simulate_frame(self, img: torch.Tensor, D_over_r0: float, seed: int, frame: int, mode: int = P2S_EXACT,
                       out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        C, H, W = img.shape
        if out is None:
            out = torch.empty_like(img)
        _check(load().dfp2s_simulate_frame(self._h, _ptr(img), C, H, W, D_over_r0, seed, frame, mode, _ptr(out),
                                           _stream(stream)))
        return out

    def set_field_variant(self, variant: int) -> None:
        """The factored sampler's column-pass kernel: 0, 1, or -1 for the default (same fields)."""
        _check(load().dfp2s_ctx_set_field_variant(self._h, variant))

    def set_field_sampler(self, sampler: int) -> None:
        """FIELDS_FACTORED (default), FIELDS_DENSE (a FACTOR_DENSE factor) or FIELDS_FULL (a FACTOR_FULL factor)."""
        _check(load().dfp2s_ctx_set_field_sampler(self._h, sampler))

    def buffers(self, J: int, C: int, H: int, W: int, K: int, w_dtype=torch.float32):
        f, wp, w = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(load().dfp2s_ctx_buffers(self._h, ctypes.byref(f), ctypes.byref(wp), ctypes.byref(w)))
        return f.value, wp.value, w.value

    def stage_timing(self, n: int) -> None:
        """Record per-stage CUDA events for the next frames, in a ring of n (0: off)."""
        _check(load().dfp2s_ctx_stage_timing(self._h, n))

    def stage_times(self, count: int):
        """(count, 4) ms of the last `count` frames: fields, warp, P2S weights, blur (waits for them)."""
        import numpy as np
        out = np.zeros((count, 4), dtype=np.float32)
        _check(load().dfp2s_ctx_stage_times(self._h, count, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dfp2s_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulate_frame(sim: Simulator, img: torch.Tensor, D_over_r0: float, seed: int, frame: int,
                   mode: int = P2S_EXACT, out: torch.Tensor | None = None) -> torch.Tensor:
    return sim.simulate_frame(img, D_over_r0, seed, frame, mode, out)


# ---------------------------------------------------------------- batches
class Engine:
    """Batched frames of uneven requests (include/dfp2s.h: dfp2s_engine_*): one P2S handle per J."""

    def __init__(self, p2s_list, pix_per_D: float = 8.0, graphs: bool = True, autotune: bool = True):
        self._p2s = list(p2s_list)  # kept alive: the engine does not own them
        arr = (ctypes.c_void_p * len(self._p2s))(*[p.handle.value for p in self._p2s])
        h = ctypes.c_void_p()
        flags = (ENGINE_GRAPHS if graphs else 0) | (ENGINE_AUTOTUNE if autotune else 0)
        _check(load().dfp2s_engine_create(arr, len(self._p2s), pix_per_D, flags, ctypes.byref(h)))
        self._h = h

    def run(self, requests, stream=None):
        """requests: dicts with img (C x H x W CUDA tensor), J, D_over_r0, seed, first_frame, n_frames, mode and
        out (n_frames x C x H x W CUDA tensor)."""
        arr = (Request * max(1, len(requests)))()
        for i, r in enumerate(requests):
            C, H, W = r["img"].shape
            out = r["out"]
            if tuple(out.shape) != (r["n_frames"], C, H, W):
                raise ValueError("out must be n_frames x C x H x W")
            arr[i] = Request(_ptr(r["img"]).value, C, H, W, r["J"], r["D_over_r0"], r["seed"],
                             r.get("first_frame", 0), r["n_frames"], r.get("mode", P2S_EXACT), _ptr(out).value)
        _check(load().dfp2s_engine_run(self._h, arr, len(requests), _stream(stream)))

    def info(self):
        import numpy as np
        n = ctypes.c_int()
        cnt = np.zeros(4, dtype=np.int64)
        _check(load().dfp2s_engine_info(self._h, ctypes.byref(n), cnt.ctypes.data_as(ctypes.c_void_p)))
        classes = []
        for i in range(n.value):
            shp = np.zeros(6, dtype=np.int32)
            ms = np.zeros(2, dtype=np.float32)
            _check(load().dfp2s_engine_class_info(self._h, i, shp.ctypes.data_as(ctypes.c_void_p),
                                                  ms.ctypes.data_as(ctypes.c_void_p)))
            classes.append({"J": int(shp[0]), "C": int(shp[1]), "H": int(shp[2]), "W": int(shp[3]), "N": int(shp[4]),
                            "column_pass": int(shp[5]), "tuned_ms": [float(ms[0]), float(ms[1])]})
        return {"frames": int(cnt[0]), "graph_launches": int(cnt[1]), "graph_instantiations": int(cnt[2]),
                "graph_updates": int(cnt[3]), "classes": classes}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dfp2s_engine_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
