"""Pins for the oracle's Zernike modes and Noll covariance (Sec. II-B, Eq. A matrix at s = 0).

Each pin uses mathematics other than the code under test:
  * orthonormality of Z_j on the unit disk (numerical polar quadrature),
  * the closed form A_0 against Noll's spectral integral (Bessel quadrature),
  * the aperture-averaged piston-removed variance from the structure function
    6.88 (r/r0)^{5/3} of Eq. (fried_struct),
  * the structure function itself rebuilt from many modes.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import jv

from oracle import zernike


def _disk_quadrature(nr=64, nt=128):
    x, w = np.polynomial.legendre.leggauss(nr)
    r = 0.5 * (x + 1.0)
    wr = 0.5 * w * r  # r dr
    t = 2 * np.pi * np.arange(nt) / nt
    R, T = np.meshgrid(r, t, indexing="ij")
    Wt = np.repeat(wr[:, None], nt, axis=1) * (2 * np.pi / nt)
    return R, T, Wt


def test_orthonormal_on_disk():
    R, T, Wt = _disk_quadrature()
    J = 36
    Z = np.stack([zernike.zernike(j, R, T) for j in range(1, J + 1)])
    G = np.einsum("iab,jab,ab->ij", Z, Z, Wt) / math.pi
    assert np.allclose(G, np.eye(J), atol=1e-10)


def test_noll_order_pairs_cos_even_sin_odd():
    # every (n, m) with m > 0 appears at one even (cos) and one odd (sin) index
    seen = {}
    for j in range(2, 67):
        n, m = zernike.noll_nm(j)
        assert (n - m) % 2 == 0 and 0 <= m <= n
        seen.setdefault((n, m), []).append(j)
    for (n, m), js in seen.items():
        if m == 0:
            assert len(js) == 1
        else:
            assert sorted(j % 2 for j in js) == [0, 1]
    # tilt x (cos) is Noll 2 and along x: Z_2 = 2 x on the disk
    assert zernike.zernike(2, np.array(0.5), np.array(0.0)) == pytest.approx(1.0)
    assert zernike.zernike(3, np.array(0.5), np.array(math.pi / 2)) == pytest.approx(1.0)


def test_noll_residuals_match_table():
    # Noll (1976) Table IV residuals Delta_J (tests/golden/noll_residuals.txt)
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "noll_residuals.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    table = {int(a): float(b) for a, b in rows}
    sigma2 = _piston_removed_variance_from_structure_function()
    cum = sigma2
    for J in range(1, 12):
        if J >= 2:
            cum -= zernike.noll_covariance_entry(J, J)
        # table printed to 3 significant digits
        assert cum == pytest.approx(table[J], rel=1.2e-2, abs=6e-4), J


def _radial_integral(n1, n2):
    # int_0^inf u^{-11/3} J_{n1+1}(2 pi u) J_{n2+1}(2 pi u) / (pi u)^2  u du
    f = lambda u: u ** (-14.0 / 3.0) * jv(n1 + 1, 2 * math.pi * u) * jv(n2 + 1, 2 * math.pi * u) / math.pi ** 2
    total = 0.0
    edges = [0.0, 1e-3, 0.1, 0.5] + list(np.arange(1.0, 60.0, 1.0))
    for a, b in zip(edges[:-1], edges[1:]):
        total += quad(f, a, b, limit=400, epsabs=0, epsrel=1e-12)[0]
    return total


def test_closed_form_matches_spectral_integral():
    # A0_ij is proportional to int Phi(k) Q_i Q_j^* d^2k with ONE constant for all pairs
    J = 20
    A = zernike.noll_matrix(J)
    ratios = []
    for a in range(J):
        for b in range(a, J):
            i, j = a + 2, b + 2
            ni, mi = zernike.noll_nm(i)
            nj, mj = zernike.noll_nm(j)
            same = mi == mj and (mi == 0 or i % 2 == j % 2)
            if not same:
                assert A[a, b] == 0.0
                continue
            sign = (-1) ** ((ni - mi) // 2 + (nj - mj) // 2)
            I = 2 * math.pi * math.sqrt((ni + 1) * (nj + 1)) * sign * _radial_integral(ni, nj)
            ratios.append(A[a, b] / I)
    ratios = np.array(ratios)
    assert np.all(ratios > 0)
    assert np.ptp(ratios) / ratios.mean() < 1e-6


def _piston_removed_variance_from_structure_function():
    # sigma^2 = (1/2) int int W W' 6.88 (|xi - xi'| / r0)^{5/3}, D = 1, r0 = 1, W = 1/area on the disk
    R = 0.5
    area = math.pi * R * R

    def overlap(r):
        return 2 * R * R * math.acos(r / (2 * R)) - 0.5 * r * math.sqrt(4 * R * R - r * r)

    val = quad(lambda r: 2 * math.pi * r * 6.88 * r ** (5.0 / 3.0) * overlap(r), 0.0, 2 * R,
               epsabs=0, epsrel=1e-12, limit=200)[0]
    return 0.5 * val / area ** 2


def test_sum_of_variances_is_piston_removed_variance():
    Jbig = 2000
    total = 0.0
    for j in range(2, Jbig + 2):
        total += zernike.noll_covariance_entry(j, j)
    # Noll's asymptotic residual after J modes, 0.2944 J^{-sqrt(3)/2}
    tail = 0.2944 * (Jbig + 1) ** (-math.sqrt(3) / 2)
    sigma2 = _piston_removed_variance_from_structure_function()
    assert sigma2 == pytest.approx(1.0299, rel=2e-3)  # Noll's Delta_1
    assert total + tail == pytest.approx(sigma2, rel=2e-3)


@pytest.mark.slow
def test_structure_function_from_modes():
    J = 300
    A = zernike.noll_matrix(J)
    pts = [((-0.5, 0.0), (0.5, 0.0)), ((0.0, -0.5), (0.0, 0.5)), ((-0.35, -0.35), (0.35, 0.35)),
           ((-0.2, 0.1), (0.3, 0.1))]
    for p, q in pts:
        r1, t1 = math.hypot(*p), math.atan2(p[1], p[0])
        r2, t2 = math.hypot(*q), math.atan2(q[1], q[0])
        dz = np.array([zernike.zernike(j + 2, np.array(r1), np.array(t1))
                       - zernike.zernike(j + 2, np.array(r2), np.array(t2)) for j in range(J)])
        D = float(dz @ A @ dz)
        sep = math.hypot(p[0] - q[0], p[1] - q[1]) / 2.0  # in units of D
        assert D == pytest.approx(6.88 * sep ** (5.0 / 3.0), rel=1e-2)
