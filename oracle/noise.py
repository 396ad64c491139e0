"""White Gaussian noise e ~ N(0, I) drawn from a counter-based generator.

Test infrastructure only (see the package docstring).

Paper: Sec. III-A starts each draw from white noise e ~ Gaussian(0, I); Sec.
III-C step 1 and Fig. rand_gen draw it for every field.  The paper does not
say how; these readings fix it so the CUDA path can reproduce every bit:

R7  Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
    easy as 1, 2, 3", SC 2011): key = (seed lo32, seed hi32), counter =
    (q lo32, q hi32, sub lo32, sub hi32) with q = (y N + x) / 4 and
    sub = (tag << 40) | (frame << 8) | mode.  The four words of counter q feed
    the positions x = 4q' .. 4q'+3 of row y.  This is the same (seed,
    subsequence, offset/4) mapping as cuRAND's Philox4_32_10.
R8  word w -> u = (2 (w >> 9) + 1) 2^-24, an odd multiple of 2^-24 in (0, 1)
    that is exact in FP32.  Box-Muller in FP32 on the pairs (u0, u1),
    (u2, u3): z0 = r cos(2 pi u1), z1 = r sin(2 pi u1), r = sqrt(-2 ln u0).
    ln is evaluated as  e ln2 + 2 atanh((m-1)/(m+1))  (exponent split, m in
    [sqrt(1/2), sqrt(2)), atanh series to s^11); cos/sin of 2 pi u as a
    quadrant taken exactly from the integer (w >> 9) plus Taylor series of
    sin and cos of (pi/2) r on r in [-1/2, 1/2].  Every step is one IEEE FP32
    operation in a fixed order, and the steps of the form x y + z (the Horner
    steps of the three polynomials, the atanh series' s^3 p + 2s, and the two
    e ln2 terms) are fused multiply-adds, x y + z with one rounding (fma_f32).
R27 The field sampler takes its white noise in the Fourier domain.  For real
    e ~ N(0, I) on the N x N torus, E = FFT2(e) is Hermitian (E(-k) = conj E(k))
    with independent components: Re and Im of each conjugate pair N(0, N^2 / 2),
    and the four self-conjugate bins (kx, ky in {0, N/2}) real N(0, N^2).  The
    sampler draws such an E directly, which has exactly the distribution of
    FFT2(e), so y = F^-1(S^1/2 E) is the method of Sec. III-A without the forward
    transform.  Mode j's Gaussians form rows kx = 0 .. N/2 of 2N values,
    (Re, Im) of E(kx, ky) at columns 2 ky, 2 ky + 1 (counter q = (kx N + ky) / 2
    for ky even; the R7 layout with y = kx and row length 2N).  In columns
    kx = 0 and N/2, E(kx, ky) for ky > N/2 is the conjugate of E(kx, N - ky), and
    at ky = 0, N/2 only the real Gaussian is used, scaled to variance N^2.
"""
from __future__ import annotations

import math
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

TAG_FIELDS = 0
TAG_BASIS = 1
TAG_MLP_DATA = 2
TAG_IMAGE = 3
TAG_MLP_INIT = 4


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox-4x32 with 10 rounds on arrays of uint32 counters; returns 4 uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint32).copy()
    c1 = np.asarray(c1, dtype=np.uint32).copy()
    c2 = np.asarray(c2, dtype=np.uint32).copy()
    c3 = np.asarray(c3, dtype=np.uint32).copy()
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            p0 = M0 * c0.astype(np.uint64)
            p1 = M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            if rnd < 9:
                k0 = np.uint32(k0 + W0)
                k1 = np.uint32(k1 + W1)
    return c0, c1, c2, c3


def subsequence(tag: int, frame: int, mode: int) -> int:
    """sub = (tag << 40) | (frame << 8) | mode (reading R7)."""
    if not (0 <= mode < 256 and 0 <= frame < 2 ** 32 and 0 <= tag < 2 ** 24):
        raise ValueError("tag/frame/mode out of range")
    return (tag << 40) | (frame << 8) | mode


def philox_words(seed: int, sub: int, q: np.ndarray):
    """The four Philox words for counters (q, sub) under key = seed."""
    q = np.asarray(q, dtype=np.uint64)
    return philox4x32_10((q & MASK32).astype(np.uint32), (q >> np.uint64(32)).astype(np.uint32),
                         np.uint32(sub & 0xFFFFFFFF), np.uint32(sub >> 32),
                         seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


# --------------------------------------------------------------- FP32 math
F = np.float32


def fma_f32(a, b, c) -> np.ndarray:
    """x y + z rounded once to FP32 (round to nearest, ties to even), for normal FP32 inputs.

    The product of two FP32 values is exact in FP64 (48 significant bits).  The FP64 sum is rounded to odd
    (TwoSum gives its exact error; an inexact sum with an even last bit moves one FP64 ulp towards the exact
    value), and a round-to-odd result with 53 >= 24 + 2 bits rounds to FP32 exactly as the exact sum would
    (Boldo and Melquiond, "Emulation of FMA and correctly rounded sums: proved algorithms using rounding to
    odd", IEEE Trans. Computers 57(4), 2008).
    """
    a = np.asarray(a, dtype=np.float32).astype(np.float64)
    b = np.asarray(b, dtype=np.float32).astype(np.float64)
    c = np.asarray(c, dtype=np.float32).astype(np.float64)
    p = a * b
    s = p + c
    bp = s - p
    err = (p - (s - bp)) + (c - bp)
    odd = (s.view(np.uint64) & np.uint64(1)) != 0
    fix = (err != 0) & ~odd
    s = np.where(fix, np.nextafter(s, np.where(err > 0, np.inf, -np.inf)), s)
    return s.astype(np.float32)

_SQRT2 = F(math.sqrt(2.0))
# ln 2 split: a 12-significant-bit head (so e * head is exact) and the FP32 rest
_LN2_HI = F(math.ldexp(math.floor(math.ldexp(math.log(2.0), 12)), -12))
_LN2_LO = F(math.log(2.0) - float(_LN2_HI))
# 2 atanh(s) = 2s + s s2 (2/3 + s2 (2/5 + s2 (2/7 + s2 (2/9 + s2 2/11))))
_LOG_C = [F(2.0 / 11.0), F(2.0 / 9.0), F(2.0 / 7.0), F(2.0 / 5.0), F(2.0 / 3.0)]
# sin((pi/2) r) = r (s1 + r2 (s3 + r2 (s5 + r2 (s7 + r2 s9))))
_H = math.pi / 2.0
_SIN_C = [F(_H ** 9 / math.factorial(9)), F(-_H ** 7 / math.factorial(7)), F(_H ** 5 / math.factorial(5)),
          F(-_H ** 3 / math.factorial(3)), F(_H)]
# cos((pi/2) r) = 1 + r2 (c2 + r2 (c4 + r2 (c6 + r2 (c8 + r2 c10))))
_COS_C = [F(-_H ** 10 / math.factorial(10)), F(_H ** 8 / math.factorial(8)), F(-_H ** 6 / math.factorial(6)),
          F(_H ** 4 / math.factorial(4)), F(-_H ** 2 / math.factorial(2))]


def word_to_uniform(w: np.ndarray) -> np.ndarray:
    """u = (2 (w >> 9) + 1) 2^-24, exact in FP32 (R8)."""
    k = (np.asarray(w, dtype=np.uint32) >> np.uint32(9)).astype(np.int64)
    return ((2 * k + 1).astype(np.float32) * F(2.0 ** -24)).astype(np.float32)


def log_f32(u: np.ndarray) -> np.ndarray:
    """Natural log of positive normal FP32 values (R8: exponent split + atanh series)."""
    u = np.asarray(u, dtype=np.float32)
    bits = u.view(np.uint32)
    e = ((bits >> np.uint32(23)).astype(np.int32) - 127)
    m = ((bits & np.uint32(0x7FFFFF)) | np.uint32(0x3F800000)).view(np.float32)
    big = m > _SQRT2
    m = np.where(big, m * F(0.5), m).astype(np.float32)
    e = np.where(big, e + 1, e)
    s = (m - F(1.0)) / (m + F(1.0))
    s2 = s * s
    p = _LOG_C[0]
    for c in _LOG_C[1:]:
        p = fma_f32(p, s2, c)
    logm = fma_f32(s * s2, p, s + s)
    ef = e.astype(np.float32)
    lo = fma_f32(ef, _LN2_LO, logm)
    return fma_f32(ef, _LN2_HI, lo)  # e * head is exact (12-bit head, |e| <= 149)


def sincos_2pi_f32(k: np.ndarray):
    """cos and sin of 2 pi u for u = (2k+1) 2^-24, k = w >> 9 (R8).

    Quarter turns v = 4u = (2k+1) 2^-22; the quadrant q = round(v) and the rest
    r = v - q in [-1/2, 1/2] are taken exactly in integers.
    """
    k = np.asarray(k, dtype=np.int64)
    num = 2 * k + 1                       # v = num * 2^-22
    q = (num + (1 << 21)) >> 22           # round half up
    rnum = num - (q << 22)                # in [-2^21, 2^21]
    r = (rnum.astype(np.float32) * F(2.0 ** -22)).astype(np.float32)
    r2 = r * r
    sp = _SIN_C[0]
    for c in _SIN_C[1:]:
        sp = fma_f32(sp, r2, c)
    s = r * sp
    cp = _COS_C[0]
    for c in _COS_C[1:]:
        cp = fma_f32(cp, r2, c)
    c = fma_f32(cp, r2, F(1.0))
    qm = q & 3
    cosv = np.select([qm == 0, qm == 1, qm == 2], [c, -s, -c], s).astype(np.float32)
    sinv = np.select([qm == 0, qm == 1, qm == 2], [s, c, -s], -c).astype(np.float32)
    return cosv, sinv


def box_muller(wa: np.ndarray, wb: np.ndarray):
    """Two Gaussians from two Philox words (R8)."""
    ua = word_to_uniform(wa)
    lg = log_f32(ua)
    t = lg * F(-2.0)
    r = np.sqrt(t).astype(np.float32)
    cv, sv = sincos_2pi_f32(np.asarray(wb, dtype=np.uint32) >> np.uint32(9))
    return (r * cv).astype(np.float32), (r * sv).astype(np.float32)


def gaussian_block(seed: int, tag: int, frame: int, mode: int, rows: int, cols: int) -> np.ndarray:
    """FP32 Gaussians e[y, x] for one mode: counter q = (y cols + x)/4 (cols % 4 == 0)."""
    if cols % 4:
        raise ValueError("row length must be a multiple of 4")
    sub = subsequence(tag, frame, mode)
    nq = rows * cols // 4
    w0, w1, w2, w3 = philox_words(seed, sub, np.arange(nq, dtype=np.uint64))
    z0, z1 = box_muller(w0, w1)
    z2, z3 = box_muller(w2, w3)
    return np.stack([z0, z1, z2, z3], axis=-1).reshape(rows, cols)


def hermitian_spectrum(g: np.ndarray, N: int) -> np.ndarray:
    """Full N x N Fourier-domain white noise E[ky, kx] (FP64 complex) from the Gaussian rows of one mode,
    g[kx, 2 ky + c], kx = 0..N/2, c = 0 (Re) / 1 (Im) (R27)."""
    g = np.asarray(g, dtype=np.float64).reshape(N // 2 + 1, N, 2)
    half = (g[..., 0] + 1j * g[..., 1]) * (N / math.sqrt(2.0))  # half[kx, ky]
    for kx in (0, N // 2):
        for ky in range(N // 2 + 1, N):
            half[kx, ky] = np.conj(half[kx, N - ky])
        for ky in (0, N // 2):
            half[kx, ky] = N * g[kx, ky, 0]
    E = np.empty((N, N), dtype=np.complex128)
    E[:, : N // 2 + 1] = half.T
    kx = np.arange(N // 2 + 1, N)
    ky = np.arange(N)
    E[:, N // 2 + 1:] = np.conj(half[(N - kx)[None, :], ((N - ky) % N)[:, None]])  # E(-k) = conj E(k)
    return E


def field_spectral_noise(seed: int, frame: int, J: int, N: int) -> np.ndarray:
    """Fourier-domain white noise of the J fields, shape (J, N, N) complex, indexed [j, ky, kx] (tag 0, R27)."""
    return np.stack([hermitian_spectrum(gaussian_block(seed, TAG_FIELDS, frame, j, N // 2 + 1, 2 * N), N)
                     for j in range(J)])
