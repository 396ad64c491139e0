"""Spatial spectra of the Zernike coefficient fields.

Test infrastructure only (see the package docstring).

Paper: Sec. III-B describes the slices A_{i,j} of the correlation tensor as
functions of the displacement s = (x - x')/D (footnote to Sec. III-B) and
Sec. III-C draws each field from its autocovariance A_{i,i} through the
Fourier method of Sec. III-A.  The paper defers the form of A_{i,j}(s) to its
reference [Chimitt 2020] under a constant-C_n^2 path; this module takes reading
R1: the path-integrated point-source model.  A turbulent layer at fraction t of
the path (t = 0 at the aperture) is seen by the two cones of a pair of object
points through sub-apertures of diameter D(1 - t) whose centres are t s D
apart, so with Noll's aperture transform Q_j

  P_ij(f) = int_0^1 (1-t)^{5/3} ((1-t)/(2t))^2 u^{-11/3} Q_i(u) conj(Q_j(u)) dt,
            u = f (1-t)/(2t)                 (vector u parallel to f)

is the spectral density of A_{i,j}(s) up to one constant shared by all i, j;
f is in cycles per unit s.  |Q_j(u)|^2 = (n+1) [J_{n+1}(2 pi u)/(pi u)]^2
times 1 (m = 0), 2 cos^2(m phi) (even j) or 2 sin^2(m phi) (odd j).

The substitution v = |u| turns the t-integral into an integral over v with a
kernel that carries all the f-dependence:

  G_nn'(f) = int_0^inf (2v/(2v+f))^{5/3} 2 v^2 / (f (2v+f)^2) g_nn'(v) dv,
  g_nn'(v) = v^{-11/3} J_{n+1}(2 pi v) J_{n'+1}(2 pi v) / (pi v)^2.

Here it is evaluated with a composite Gauss-Legendre rule (log-spaced panels
below v = 1, uniform panels above); a test compares it with adaptive
quadrature of the t-form.
"""
from __future__ import annotations

import functools
import math
import numpy as np
from scipy.special import jv

from .zernike import noll_nm


# ---------------------------------------------------------------- quadrature
@functools.lru_cache(maxsize=None)
def _v_rule():
    """Nodes and weights on (0, V_MAX] for the v-integral."""
    xs8, ws8 = np.polynomial.legendre.leggauss(8)
    xs16, ws16 = np.polynomial.legendre.leggauss(16)
    nodes, weights = [], []
    # log-spaced panels in y = ln v from ln(1e-8) to 0, width ~0.2
    ys = np.linspace(math.log(1e-8), 0.0, 93)
    for a, b in zip(ys[:-1], ys[1:]):
        y = 0.5 * (b - a) * xs8 + 0.5 * (a + b)
        v = np.exp(y)
        nodes.append(v)
        weights.append(0.5 * (b - a) * ws8 * v)  # dv = v dy
    # uniform panels in v from 1 to 48, width 1/4
    vs = np.linspace(1.0, 48.0, 189)
    for a, b in zip(vs[:-1], vs[1:]):
        nodes.append(0.5 * (b - a) * xs16 + 0.5 * (a + b))
        weights.append(0.5 * (b - a) * ws16)
    return np.concatenate(nodes), np.concatenate(weights)


@functools.lru_cache(maxsize=None)
def _v_rule_deep():
    """The v-rule for frequencies far below the torus bins (the subharmonics, R31): 8-point panels of width 0.2
    in ln v from 1e-14 to 1 (the integrand's mass lies at v >~ f), then the uniform panels of _v_rule."""
    xs8, ws8 = np.polynomial.legendre.leggauss(8)
    nodes, weights = [], []
    y0 = math.log(1e-14)
    npan = int(math.ceil(-y0 / 0.2))
    for p in range(npan):
        a, b = y0 * (1 - p / npan), y0 * (1 - (p + 1) / npan)
        y = 0.5 * (b - a) * xs8 + 0.5 * (a + b)
        v = np.exp(y)
        nodes.append(v)
        weights.append(0.5 * (b - a) * ws8 * v)
    v1, w1 = _v_rule()
    up = v1 >= 1.0
    return np.concatenate(nodes + [v1[up]]), np.concatenate(weights + [w1[up]])


def g_radial(n: int, n2: int, v: np.ndarray) -> np.ndarray:
    """g_nn'(v) = v^{-11/3} J_{n+1}(2 pi v) J_{n'+1}(2 pi v) / (pi v)^2."""
    v = np.asarray(v, dtype=np.float64)
    return v ** (-11.0 / 3.0) * jv(n + 1, 2 * math.pi * v) * jv(n2 + 1, 2 * math.pi * v) / (math.pi * v) ** 2


def radial_spectra(pairs, f: np.ndarray, deep: bool = False) -> np.ndarray:
    """G_nn'(f) for f > 0 and every (n, n') in pairs (reading R1, v-form); shape (len(pairs), len(f)).
    deep: the rule that reaches v = 1e-14, for f far below the torus bins."""
    f = np.atleast_1d(np.asarray(f, dtype=np.float64))
    v, w = _v_rule_deep() if deep else _v_rule()
    Gw = np.stack([w * g_radial(n, n2, v) for n, n2 in pairs], axis=1)  # (Q, P)
    out = np.empty((len(pairs), f.size))
    chunk = 1024
    lv = np.log(2 * v)
    for s in range(0, f.size, chunk):
        fc = f[s:s + chunk, None]
        d = 2 * v + fc
        K = np.exp((5.0 / 3.0) * (lv - np.log(d))) * (2 * v * v) / (fc * d * d)
        out[:, s:s + chunk] = (K @ Gw).T
    return out


def radial_spectrum(n: int, n2: int, f: np.ndarray) -> np.ndarray:
    """G_nn'(f) for f > 0 (reading R1, v-form)."""
    return radial_spectra([(n, n2)], f)[0]


def radial_spectrum_tform(n: int, n2: int, f: float) -> float:
    """G_nn'(f) straight from the t-integral of reading R1, by adaptive quadrature (slow)."""
    from scipy.integrate import quad

    def integrand(t):
        if t <= 0.0 or t >= 1.0:
            return 0.0
        u = f * (1 - t) / (2 * t)
        return ((1 - t) ** (5.0 / 3.0) * ((1 - t) / (2 * t)) ** 2
                * u ** (-11.0 / 3.0) * jv(n + 1, 2 * math.pi * u) * jv(n2 + 1, 2 * math.pi * u)
                / (math.pi * u) ** 2)

    # split at t values where u = 50, 10, 2, 0.5, 0.1 so quad sees the structure
    cuts = sorted({f / (f + 2 * uu) for uu in (200.0, 50.0, 10.0, 2.0, 0.5, 0.1)})
    pts = [0.0] + cuts + [1.0]
    total = 0.0
    for a, b in zip(pts[:-1], pts[1:]):
        val, _ = quad(integrand, a, b, limit=2000, epsabs=0.0, epsrel=1e-12)
        total += val
    return total


# --------------------------------------------------------- angular factors
def angular_factor(j: int, phi: np.ndarray) -> np.ndarray:
    """|Theta_j(phi)|^2: 1 for m = 0, 2cos^2(m phi) for even j, 2 sin^2(m phi) for odd j."""
    n, m = noll_nm(j)
    phi = np.asarray(phi, dtype=np.float64)
    if m == 0:
        return np.ones_like(phi)
    if j % 2 == 0:
        return 2.0 * np.cos(m * phi) ** 2
    return 2.0 * np.sin(m * phi) ** 2


def theta_complex(j: int, phi: np.ndarray) -> np.ndarray:
    """Theta_j(phi), the complex angular part of Noll's Q_j (phase convention of Noll 1976)."""
    n, m = noll_nm(j)
    phi = np.asarray(phi, dtype=np.float64)
    if m == 0:
        return (-1.0) ** (n // 2) * np.ones_like(phi, dtype=np.complex128)
    pre = (-1.0) ** ((n - m) // 2) * (1j ** m) * math.sqrt(2.0)
    if j % 2 == 0:
        return pre * np.cos(m * phi)
    return pre * np.sin(m * phi)


# ------------------------------------------------------------ torus grids
def torus_frequencies(N: int, pix_per_D: float):
    """|f| and direction phi of every bin of the N x N FFT grid, FFT order.

    Bin k of an axis is the signed frequency k (k < N/2) or k - N, times
    pix_per_D / N cycles per unit s (reading R3/R5).  Row index = ky, column = kx.
    """
    k = np.fft.fftfreq(N, d=1.0 / N)  # signed integers
    ky, kx = np.meshgrid(k, k, indexing="ij")
    scale = pix_per_D / N
    fx, fy = kx * scale, ky * scale
    return np.hypot(fx, fy), np.arctan2(fy, fx), kx.astype(np.int64), ky.astype(np.int64)


@functools.lru_cache(maxsize=8)
def _radial_table(N: int, pix_per_D: float, pairs: tuple):
    """G for every distinct |k|^2 of the N x N torus and every pair; returns (inverse index, table)."""
    _, _, kx, ky = torus_frequencies(N, pix_per_D)
    r2 = kx * kx + ky * ky
    uniq, inv = np.unique(r2, return_inverse=True)
    vals = np.zeros((len(pairs), uniq.size))
    nz = uniq > 0
    vals[:, nz] = radial_spectra(list(pairs), np.sqrt(uniq[nz].astype(np.float64)) * pix_per_D / N)
    return inv.reshape(N, N), vals


def _all_pairs(nmax: int = 10):
    return tuple((a, b) for a in range(1, nmax + 1) for b in range(a, nmax + 1))


def _diag_pairs(nmax: int = 10):
    return tuple((a, a) for a in range(1, nmax + 1))


def _radial_on_torus(N: int, pix_per_D: float, n: int, n2: int) -> np.ndarray:
    if n == n2:
        pairs = _diag_pairs()
    else:
        pairs = _all_pairs()
    inv, vals = _radial_table(N, pix_per_D, pairs)
    return vals[pairs.index((min(n, n2), max(n, n2)))][inv]


def mode_spectrum_shape(j: int, N: int, pix_per_D: float) -> np.ndarray:
    """P_jj(f_k) on the N x N torus (unnormalised), with the DC bin set to 0 (R5)."""
    n, _ = noll_nm(j)
    fmag, phi, _, _ = torus_frequencies(N, pix_per_D)
    P = (n + 1) * angular_factor(j, phi) * _radial_on_torus(N, pix_per_D, n, n)
    P[0, 0] = 0.0
    return P


def lambda_mode(j: int, N: int, pix_per_D: float) -> np.ndarray:
    """lambda_j(k) = N^2 P_jj(f_k) / sum_{k' != 0} P_jj(f_k'), lambda_j(0) = 0 (R2, R5).

    The field  Re IFFT2(sqrt(lambda_j) FFT2(e)) / N^2  of white noise e then has
    variance exactly 1 at every pixel and autocovariance proportional to A_jj.
    """
    P = mode_spectrum_shape(j, N, pix_per_D)
    return N * N * P / P.sum()


def lambdas(J: int, N: int, pix_per_D: float) -> np.ndarray:
    """lambda for the J modes Noll 2..J+1, shape (J, N, N)."""
    return np.stack([lambda_mode(j + 2, N, pix_per_D) for j in range(J)])


def autocorrelation(lam: np.ndarray) -> np.ndarray:
    """rho_j(s) on the torus: IFFT2(lambda_j)/N^2 -> unit value at s = 0."""
    N = lam.shape[-1]
    return np.real(np.fft.ifft2(lam)) * 1.0  # ifft2 already divides by N^2


def cross_spectrum_torus(J: int, N: int, pix_per_D: float, A0: np.ndarray) -> np.ndarray:
    """Full J x J cross-spectral density on the N x N torus, shape (N, N, J, J), complex.

    S_ij(k) = N^2 Theta_i conj(Theta_j) sqrt((n_i+1)(n_j+1)) G_{n_i n_j}(|f_k|)
              * sqrt(A0_ii A0_jj / (sum_k' P_ii sum_k' P_jj)),    S(0) = 0.
    The diagonal reproduces the per-mode normalisation of lambda_mode scaled by
    A0_ii; self-conjugate bins (k = -k mod N) are made real so the tensor belongs
    to a real field.  Used for the brute-force full-tensor sampler (Fig. rand_gen,
    Sec. III-D) only.
    """
    fmag, phi, kx, ky = torus_frequencies(N, pix_per_D)
    sums = np.array([mode_spectrum_shape(j + 2, N, pix_per_D).sum() for j in range(J)])
    S = np.zeros((N, N, J, J), dtype=np.complex128)
    th = [theta_complex(j + 2, phi) for j in range(J)]
    for a in range(J):
        na, _ = noll_nm(a + 2)
        for b in range(J):
            nb, _ = noll_nm(b + 2)
            G = _radial_on_torus(N, pix_per_D, min(na, nb), max(na, nb))
            S[:, :, a, b] = (N * N * th[a] * np.conj(th[b]) * math.sqrt((na + 1) * (nb + 1)) * G
                             * math.sqrt(A0[a, a] * A0[b, b] / (sums[a] * sums[b])))
    S[0, 0] = 0.0
    selfconj = ((2 * kx) % N == 0) & ((2 * ky) % N == 0)
    S[selfconj] = S[selfconj].real
    return S


def full_tensor_torus(J: int, N: int, pix_per_D: float, A0: np.ndarray) -> np.ndarray:
    """The non-approximated homogeneous tensor A on the N x N torus as a dense matrix.

    Index order (mode, y, x) for rows and columns; entry
    E[a_i(x) a_j(x + s)] = sum_k S_ij(k) e^{2 pi i k.s/N} / N^2.
    """
    S = cross_spectrum_torus(J, N, pix_per_D, A0)
    C = np.fft.ifft2(S, axes=(0, 1))  # C[sy, sx, i, j]
    C = np.real(C)
    n = N * N
    A = np.empty((J * n, J * n))
    ys, xs = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ys, xs = ys.ravel(), xs.ravel()
    dy = (ys[None, :] - ys[:, None]) % N
    dx = (xs[None, :] - xs[:, None]) % N
    for a in range(J):
        for b in range(J):
            A[a * n:(a + 1) * n, b * n:(b + 1) * n] = C[dy, dx, a, b]
    return A


def approx_tensor_torus(lam: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Eq. (A tilde): (L x I) blockdiag(rho_1..rho_J) (L x I)^T as a dense matrix, order (mode, y, x)."""
    J, N, _ = lam.shape
    n = N * N
    rho = np.fft.ifft2(lam, axes=(1, 2)).real
    ys, xs = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    ys, xs = ys.ravel(), xs.ravel()
    dy = (ys[None, :] - ys[:, None]) % N
    dx = (xs[None, :] - xs[:, None]) % N
    B = np.zeros((J * n, J * n))
    for a in range(J):
        B[a * n:(a + 1) * n, a * n:(a + 1) * n] = rho[a][dy, dx]
    LI = np.kron(L, np.eye(n))
    return LI @ B @ LI.T
