"""Pins for the oracle's white noise (readings R7, R8).

Philox words are checked against cuRAND's own Philox4_32_10 host generator (a
separate implementation of the published algorithm, run on the CPU through
libcurand); the FP32 transforms against libm in FP64 over every reachable input.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

from oracle import noise


def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and os.path.exists(cand) if cand.startswith("/") else cand:
            try:
                return ctypes.CDLL(cand)
            except OSError:
                pass
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 2 ** 64 - 1])
def test_philox_matches_curand_host_generator(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 3 * 4 * 65536
        buf = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    # the host generator interleaves 65536 subsequences: group g = (offset q) * 65536 + subsequence
    g = np.arange(n // 4)
    q = (g // 65536).astype(np.uint32)
    sub = (g % 65536).astype(np.uint32)
    zero = np.zeros_like(q)
    w = noise.philox4x32_10(q, zero, sub, zero, seed & 0xFFFFFFFF, seed >> 32)
    mine = np.stack(w, axis=-1).ravel()
    assert np.array_equal(mine, buf)


def test_uniform_exact_and_open_interval():
    w = np.array([0, 1, 511, 512, 2 ** 31, 2 ** 32 - 1], dtype=np.uint32)
    u = noise.word_to_uniform(w)
    assert u.dtype == np.float32
    k = (w >> 9).astype(np.float64)
    assert np.array_equal(u.astype(np.float64), (2 * k + 1) * 2.0 ** -24)
    assert u.min() > 0 and u.max() < 1


def test_log_within_2ulp_of_libm_everywhere():
    k = np.arange(2 ** 23, dtype=np.int64)
    u = ((2 * k + 1) * 2.0 ** -24).astype(np.float32)
    mine = noise.log_f32(u).astype(np.float64)
    ref = np.log(u.astype(np.float64))
    ulp = np.spacing(np.abs(ref.astype(np.float32))).astype(np.float64)
    assert np.max(np.abs(mine - ref) / ulp) <= 2.0


def test_sincos_accuracy_everywhere():
    k = np.arange(2 ** 23, dtype=np.int64)
    c, s = noise.sincos_2pi_f32(k)
    ang = 2 * math.pi * (2 * k + 1) * 2.0 ** -24
    assert np.max(np.abs(c - np.cos(ang))) < 1.2e-7
    assert np.max(np.abs(s - np.sin(ang))) < 1.2e-7
    assert np.max(np.abs(c.astype(np.float64) ** 2 + s.astype(np.float64) ** 2 - 1)) < 3e-7


def test_gaussian_moments_and_distribution():
    from scipy import stats
    z = noise.gaussian_block(7, noise.TAG_FIELDS, 3, 5, 1024, 1024).astype(np.float64).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs(stats.kurtosis(z, fisher=False) - 3) < 5 * math.sqrt(24 / n)
    assert stats.kstest(z[::7], "norm").pvalue > 1e-4


def test_streams_are_distinct():
    a = noise.gaussian_block(0, noise.TAG_FIELDS, 0, 0, 8, 8)
    b = noise.gaussian_block(0, noise.TAG_FIELDS, 0, 1, 8, 8)
    c = noise.gaussian_block(0, noise.TAG_FIELDS, 1, 0, 8, 8)
    d = noise.gaussian_block(1, noise.TAG_FIELDS, 0, 0, 8, 8)
    e = noise.gaussian_block(0, noise.TAG_BASIS, 0, 0, 8, 8)
    for x in (b, c, d, e):
        assert not np.array_equal(a, x)

def _round_to_f32(x):
    """Exact rational x rounded to the nearest FP32 (ties to even), for |x| in the normal range or 0."""
    from fractions import Fraction
    if x == 0:
        return 0.0
    sign = -1 if x < 0 else 1
    x = abs(x)
    e = x.numerator.bit_length() - x.denominator.bit_length()
    while Fraction(2) ** e > x:
        e -= 1
    while Fraction(2) ** (e + 1) <= x:
        e += 1
    scaled = x / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    q = scaled.numerator // scaled.denominator
    rem = scaled - q
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and q % 2 == 1):
        q += 1
    return sign * float(Fraction(q) * Fraction(2) ** (e - 23))


def test_fma_f32_is_correctly_rounded():
    # against exact rational arithmetic: random triples over many exponents, near-cancellations and exact ties
    from fractions import Fraction
    rng = np.random.default_rng(0)
    n = 3000
    a = (rng.standard_normal(n) * 2.0 ** rng.integers(-20, 20, n)).astype(np.float32)
    b = (rng.standard_normal(n) * 2.0 ** rng.integers(-20, 20, n)).astype(np.float32)
    c = (rng.standard_normal(n) * 2.0 ** rng.integers(-40, 40, n)).astype(np.float32)
    c[: n // 4] = (-(a[: n // 4].astype(np.float64) * b[: n // 4]) * (1 + 1e-6)).astype(np.float32)  # cancellation
    # ties: a*b exact with 48 bits, c chosen so that the sum lies halfway between two FP32 values
    t = n // 4
    a[t:2 * t] = np.float32(1.0) + np.float32(2.0 ** -23) * rng.integers(1, 2 ** 10, t).astype(np.float32)
    b[t:2 * t] = np.float32(1.0) + np.float32(2.0 ** -23) * rng.integers(1, 2 ** 10, t).astype(np.float32)
    c[t:2 * t] = np.float32(2.0 ** -24) * rng.choice([1.0, -1.0, 3.0], t).astype(np.float32)
    # exact ties: (1 + 2^-12)^2 = 1 + 2^-11 + 2^-24 lies halfway between two FP32 values (ulp 2^-23 at 1)
    x = np.float32(1 + 2.0 ** -12)
    a[:4], b[:4] = x, x
    c[:4] = np.array([0.0, 2.0 ** -40, -2.0 ** -40, 2.0 ** -23], dtype=np.float32)
    got = noise.fma_f32(a, b, c).astype(np.float64)
    assert got[0] == 1 + 2.0 ** -11                  # the tie goes to the even neighbour
    assert got[1] == 1 + 2.0 ** -11 + 2.0 ** -23     # just above the tie: up
    assert got[2] == 1 + 2.0 ** -11                  # just below: down
    for i in range(n):
        want = _round_to_f32(Fraction(float(a[i])) * Fraction(float(b[i])) + Fraction(float(c[i])))
        assert got[i] == want, (i, a[i], b[i], c[i], got[i], want)
    # and it is not the two-rounding sum
    two = ((a * b).astype(np.float32) + c).astype(np.float64)
    assert np.any(two != got)
