"""The full (non-approximated) homogeneous sampler of the Zernike fields.

Test infrastructure only (see the package docstring).

Sec. III-B: every slice A_{i,j} of the correlation tensor depends on the
displacement s alone, so the J fields are jointly homogeneous and have a J x J
cross-spectral density S(f), Hermitian and positive semi-definite at every
frequency.  The paper's sampler (Sec. III-C, Eq. A tilde) keeps only the
autocovariances and mixes with A_0; Sec. III-D measures what that loses.  The
exact FFT sampler draws E(k) = rho(k) xi(k) per frequency with rho rho^H the
spectral density the covariance needs, and returns F^-1(E).

Reading R29 (the root).  Under R1 the cross spectrum of modes i, j on the
torus is (spectrum.cross_spectrum_torus)
  S_ij(k) = c_i c_j Theta_i(phi_k) conj(Theta_j(phi_k)) sqrt((n_i+1)(n_j+1)) G_{n_i n_j}(|f_k|),
  c_j = N sqrt(A0_jj / sum_k P_jj(k)),
because the vector u of the aperture transform Q_j(u) is parallel to f: the
angular part leaves the path integral and the radial part depends on the
radial orders only.  With D(k) = diag(c_j sqrt(n_j+1) Theta_j(phi_k)), P the
J x R indicator of each mode's radial order (R distinct orders, 8 for J = 36)
and Gamma(|f|) the R x R matrix G_{n_o n_o'}(|f|) (a Gram matrix of the
functions J_{n+1}(2 pi v) under a positive weight, so positive definite),
  S(k) = D(k) P Gamma(|f_k|) P^T D(k)^H = R(k) R(k)^H,  R(k) = D(k) P chol(Gamma(|f_k|)).
So S has rank at most R and R complex noises per frequency give the exact
cross-spectrum: fewer than the J of the approximation.

Which spectral density the sample needs.  full_tensor_torus defines
E[a_i(x) a_j(x + d)] = Re sum_k S_ij(k) e^{2 pi i k.d/N} / N^2, i.e. the
Hermitian part S_sym(k) = (S(k) + conj S(-k)) / 2 (the real part on the four
self-conjugate bins).  For E(-k) = conj E(k), E[a_i(x) a_j(x + d)] =
sum_k Sigma_ij(k) e^{-2 pi i k.d/N} / N^4 with Sigma = E[E E^H], so the draw
needs Sigma(k) = N^2 conj(S_sym(k)).  Off the lines kx = N/2 and ky = N/2 the
signed frequency of -k is minus that of k, Theta(phi + pi) = conj Theta(phi),
and S(-k) = conj S(k); on those lines index N/2 is the frequency -N/2 for k
and -k alike, so S(-k) is another rank-R matrix and the root takes both halves.
Per bin of the half plane kx = 0 .. N/2 (z_r = g_re + i g_im, unit-variance
parts from Philox stream r, z'_r from stream R + r):
  generic bins          E = (N / sqrt 2) conj(R(k)) z
  lines kx or ky = N/2  E = (N / 2) (conj(R(k)) z + R(-k) z')
  three Nyquist corners E = N Re(conj(R(k)) z)          (real)
  DC                    E = 0 (S(0) = 0, R5)
and columns kx = 0, N/2 are completed by E(kx, N - ky) = conj E(kx, ky), the
other half plane by E(-k) = conj E(k).  The fields are Re F^-1(E) times
(D/r0)^{5/6} (A_0 is the D/r0 = 1 matrix).  No mixing step follows: the
cross-correlations are in S.
"""
from __future__ import annotations

import math

import numpy as np

from . import noise, spectrum, zernike

TAG_FULL_FIELDS = 5  # Philox subsequence tag of the full sampler's noise (R7)


def radial_orders(J: int):
    """The distinct radial orders of Noll modes 2..J+1 (ascending) and each mode's index into them."""
    ns = [zernike.noll_nm(j + 2)[0] for j in range(J)]
    orders = sorted(set(ns))
    return orders, np.array([orders.index(n) for n in ns])


def order_gram(J: int, N: int, pix_per_D: float) -> np.ndarray:
    """Gamma(|f_k|) on the N x N torus, shape (N, N, R, R): G_{n_o n_o'} for every pair of radial orders."""
    inv, Gu = order_gram_unique(J, N, pix_per_D)
    return Gu[inv]


def order_gram_unique(J: int, N: int, pix_per_D: float):
    """Gamma per distinct |k|^2 of the torus: (inverse index (N, N), Gamma (U, R, R)); zero at DC."""
    orders, _ = radial_orders(J)
    R = len(orders)
    pairs = spectrum._all_pairs()
    inv, vals = spectrum._radial_table(N, pix_per_D, pairs)
    Gu = np.zeros((vals.shape[1], R, R))
    for a in range(R):
        for b in range(a, R):
            g = vals[pairs.index((orders[a], orders[b]))]
            Gu[:, a, b] = g
            Gu[:, b, a] = g
    return inv, Gu


def order_cholesky_unique(J: int, N: int, pix_per_D: float):
    """(inverse index, C (U, R, R)): the lower Cholesky factor of Gamma per distinct |k|^2, zero at DC."""
    inv, Gu = order_gram_unique(J, N, pix_per_D)
    C = np.zeros_like(Gu)
    nz = np.abs(Gu).sum(axis=(1, 2)) > 0
    C[nz] = np.linalg.cholesky(Gu[nz])
    return inv, C


def mode_scales(J: int, N: int, pix_per_D: float, A0: np.ndarray) -> np.ndarray:
    """c_j sqrt(n_j + 1) with c_j = N sqrt(A0_jj / sum_k P_jj(k)), the diagonal of D(k) without Theta."""
    out = np.empty(J)
    for j in range(J):
        n, _ = zernike.noll_nm(j + 2)
        total = spectrum.mode_spectrum_shape(j + 2, N, pix_per_D).sum()
        out[j] = N * math.sqrt(A0[j, j] / total) * math.sqrt(n + 1)
    return out


def full_root(J: int, N: int, pix_per_D: float, A0: np.ndarray) -> np.ndarray:
    """R(k) = D(k) P chol(Gamma(|f_k|)) on the N x N torus, shape (N, N, J, R) complex, [ky, kx] order; 0 at DC."""
    _, phi, _, _ = spectrum.torus_frequencies(N, pix_per_D)
    _, order_of = radial_orders(J)
    inv, Cu = order_cholesky_unique(J, N, pix_per_D)
    C = Cu[inv]
    scale = mode_scales(J, N, pix_per_D, A0)
    Rt = np.empty((N, N, J, C.shape[-1]), dtype=np.complex128)
    for j in range(J):
        th = spectrum.theta_complex(j + 2, phi)
        Rt[:, :, j, :] = (scale[j] * th)[:, :, None] * C[:, :, order_of[j], :]
    return Rt


def _line_gaussians(seed, frame, stream, N):
    """z' of one stream on the half plane, drawn only where it is used: column kx = N/2 and row ky = N/2."""
    half = N // 2 + 1
    out = np.zeros((half, N), dtype=np.complex128)
    sub = noise.subsequence(TAG_FULL_FIELDS, frame, stream)
    kx = np.concatenate([np.full(N // 2, N // 2), np.arange(N // 2)])
    i = np.concatenate([np.arange(N // 2), np.full(N // 2, N // 4)])  # bins (kx, 2i), (kx, 2i + 1)
    w0, w1, w2, w3 = noise.philox_words(seed, sub, (kx * (N // 2) + i).astype(np.uint64))
    g0, g1 = noise.box_muller(w0, w1)
    g2, g3 = noise.box_muller(w2, w3)
    out[kx, 2 * i] = g0.astype(np.float64) + 1j * g1.astype(np.float64)
    out[kx, 2 * i + 1] = g2.astype(np.float64) + 1j * g3.astype(np.float64)
    return out


def full_spectrum(seed: int, frame: int, J: int, N: int, pix_per_D: float, A0: np.ndarray) -> np.ndarray:
    """The Fourier-domain fields E (J, N, N) complex, [j, ky, kx], of one frame of the full sampler (R29).

    conj(R(k)) z = conj(c_j sqrt(n_j+1) Theta_j(phi_k)) eta_{o_j}(k) with eta_o = sum_r C_or z_r, C real: the
    per-bin rules of the module docstring, evaluated for all bins of a mode at once.
    """
    orders, order_of = radial_orders(J)
    R = len(orders)
    half = N // 2 + 1
    inv, Cu = order_cholesky_unique(J, N, pix_per_D)
    Ch = Cu[inv.T[:half]]                              # (half, N, R, R) at [kx, ky]
    z = np.stack([np.asarray(noise.gaussian_block(seed, TAG_FULL_FIELDS, frame, r, half, 2 * N), np.float64)
                  .reshape(half, N, 2) @ np.array([1.0, 1j]) for r in range(R)], axis=-1)   # (half, N, R)
    z2 = np.stack([_line_gaussians(seed, frame, R + r, N) for r in range(R)], axis=-1)
    eta = np.einsum("xyor,xyr->xyo", Ch, z)
    eta2 = np.einsum("xyor,xyr->xyo", Ch, z2)
    _, phi, _, _ = spectrum.torus_frequencies(N, pix_per_D)
    phi_h = phi.T[:half]                               # phi at [kx, ky]
    phi_m = phi[(N - np.arange(N)[None, :]) % N, (N - np.arange(half)[:, None]) % N]  # phi(-k) at [kx, ky]
    kx = np.arange(half)[:, None] * np.ones((1, N), dtype=int)
    ky = np.ones((half, 1), dtype=int) * np.arange(N)[None, :]
    corner = np.isin(kx, (0, N // 2)) & np.isin(ky, (0, N // 2))
    line = ((kx == N // 2) | (ky == N // 2)) & ~corner
    scale = mode_scales(J, N, pix_per_D, A0)
    Eh = np.zeros((J, half, N), dtype=np.complex128)
    for j in range(J):
        th = spectrum.theta_complex(j + 2, phi_h)
        tm = spectrum.theta_complex(j + 2, phi_m)
        a = scale[j] * np.conj(th) * eta[:, :, order_of[j]]
        b = scale[j] * tm * eta2[:, :, order_of[j]]
        e = (N / math.sqrt(2.0)) * a
        e[line] = (N / 2) * (a[line] + b[line])
        e[corner] = N * a[corner].real
        e[0, 0] = 0.0
        Eh[j] = e
    for c in (0, N // 2):
        Eh[:, c, N // 2 + 1:] = np.conj(Eh[:, c, 1: N // 2][:, ::-1])
    E = np.empty((J, N, N), dtype=np.complex128)
    E[:, :, :half] = np.transpose(Eh, (0, 2, 1))
    kxs = np.arange(half, N)
    kys = np.arange(N)
    E[:, :, half:] = np.conj(Eh[:, (N - kxs)[None, :], ((N - kys) % N)[:, None]])
    return E


def sample_fields_full(seed: int, frame: int, J: int, H: int, W: int, D_over_r0: float,
                       pix_per_D: float = 8.0, N: int | None = None) -> np.ndarray:
    """The J x H x W fields of one frame from the full cross-spectral density (Sec. III-B, R29), FP64."""
    from .sampler import grid_size
    if N is None:
        N = grid_size(H, W, pix_per_D)
    A0 = zernike.noll_matrix(J, 1.0)
    E = full_spectrum(seed, frame, J, N, pix_per_D, A0)
    a = np.real(np.fft.ifft2(E, axes=(1, 2)))[:, :H, :W]
    return a * D_over_r0 ** (5.0 / 6.0)


def operator_matrix_full(J: int, N: int, pix_per_D: float, A0: np.ndarray):
    """The full sampler as a linear map from its Gaussians to the fields on the whole torus.

    Columns: every Gaussian of the 2R streams that reaches the output, order (mode, y, x) for rows.
    Built by replaying full_spectrum's per-bin rules on unit inputs (no Philox), so M M^T is the
    covariance the sampler realises.
    """
    Rt = full_root(J, N, pix_per_D, A0)
    R = Rt.shape[-1]
    half = N // 2 + 1
    cols = []

    def fields_of(Eh):
        Eh = Eh.copy()
        for kx in (0, N // 2):
            for ky in range(N // 2 + 1, N):
                Eh[:, kx, ky] = np.conj(Eh[:, kx, N - ky])
        E = np.empty((J, N, N), dtype=np.complex128)
        E[:, :, :half] = np.transpose(Eh, (0, 2, 1))
        kxs = np.arange(half, N)
        kys = np.arange(N)
        E[:, :, half:] = np.conj(Eh[:, (N - kxs)[None, :], ((N - kys) % N)[:, None]])
        return np.real(np.fft.ifft2(E, axes=(1, 2))).ravel()

    for kx in range(half):
        for ky in range(N):
            if kx == 0 and ky == 0:
                continue
            if (kx in (0, N // 2)) and ky > N // 2:
                continue  # overwritten by the completion: its Gaussians never reach the output
            Rk = Rt[ky, kx]
            corner = (kx in (0, N // 2)) and (ky in (0, N // 2))
            line = (kx == N // 2 or ky == N // 2) and not corner
            for r in range(R):
                for part in (1.0, 1j):
                    if corner:
                        e = N * np.real(np.conj(Rk[:, r]) * part)
                    elif line:
                        e = (N / 2) * np.conj(Rk[:, r]) * part
                    else:
                        e = (N / math.sqrt(2.0)) * np.conj(Rk[:, r]) * part
                    Eh = np.zeros((J, half, N), dtype=np.complex128)
                    Eh[:, kx, ky] = e
                    cols.append(fields_of(Eh))
                    if line:
                        Rm = Rt[(N - ky) % N, (N - kx) % N]
                        Eh = np.zeros((J, half, N), dtype=np.complex128)
                        Eh[:, kx, ky] = (N / 2) * Rm[:, r] * part
                        cols.append(fields_of(Eh))
    return np.stack(cols, axis=1)
