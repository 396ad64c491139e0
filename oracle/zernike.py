"""Zernike modes in Noll's convention and Noll's covariance matrix A_0.

Test infrastructure only (see the package docstring).

Paper: Sec. II-B, Eq. (Zernike decompose): the phase over the aperture of the
pixel x is phi_x(R rho) = sum_j a_{x,j} Z_j(rho); Eq. (A matrix) and the text
after it: at zero displacement the correlation matrix A_0 is Noll's covariance
of the coefficients.  The modes simulated are Noll 2..J+1 (piston excluded,
reading R9); field index 0 is Noll mode 2.
"""
from __future__ import annotations

import math
import numpy as np
from scipy.special import gammaln, gamma


def noll_nm(j: int) -> tuple[int, int]:
    """Radial order n and azimuthal frequency m >= 0 of Noll index j >= 1.

    Within order n the indices run n(n+1)/2+1 .. (n+1)(n+2)/2 and m takes the
    values of the parity of n in increasing order, each m > 0 twice (the even
    index carries cos(m theta), the odd index sin(m theta)).
    """
    if j < 1:
        raise ValueError("Noll index starts at 1")
    n = 0
    while (n + 1) * (n + 2) // 2 < j:
        n += 1
    r = j - n * (n + 1) // 2 - 1  # 0-based position inside order n
    if n % 2 == 0:
        m = 2 * ((r + 1) // 2)
    else:
        m = 2 * (r // 2) + 1
    return n, m


def radial_poly(n: int, m: int, rho: np.ndarray) -> np.ndarray:
    """Zernike radial polynomial R_n^m(rho) (explicit factorial sum)."""
    rho = np.asarray(rho, dtype=np.float64)
    out = np.zeros_like(rho)
    for s in range((n - m) // 2 + 1):
        c = ((-1) ** s * math.factorial(n - s)
             / (math.factorial(s) * math.factorial((n + m) // 2 - s)
                * math.factorial((n - m) // 2 - s)))
        out = out + c * rho ** (n - 2 * s)
    return out


def zernike(j: int, rho: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Noll-normalised Z_j(rho, theta): unit mean square over the unit disk.

    Z_j = sqrt(n+1) R_n^0 for m = 0, sqrt(2(n+1)) R_n^m cos(m theta) for even j,
    sqrt(2(n+1)) R_n^m sin(m theta) for odd j.  theta is measured from +x
    (image column) towards +y (image row), reading R10.
    """
    n, m = noll_nm(j)
    R = radial_poly(n, m, rho)
    if m == 0:
        return math.sqrt(n + 1) * R
    ang = np.cos(m * theta) if j % 2 == 0 else np.sin(m * theta)
    return math.sqrt(2 * (n + 1)) * R * ang


def noll_constant() -> float:
    """Leading constant K of Noll's closed-form covariance, consistent with Eq. (fried_struct).

    Noll's covariance is the integral of the Kolmogorov phase spectrum
    c r0^{-5/3} f^{-11/3} (f in cycles per unit length) against the aperture
    transforms Q_i Q_j^*; the radial Bessel integral has the closed form of
    Weber and Schafheitlin, which gives K sqrt((n+1)(n'+1)) times the Gamma
    ratio of noll_covariance_entry with

        K = c Gamma(14/3) 2^{-5/3} pi^{8/3},
        c = [(24/5) Gamma(6/5)]^{5/6} Gamma(11/6)^2 / (2 pi^{11/3}),

    where c is the spectrum coefficient for which the structure function is
    2 [(24/5) Gamma(6/5)]^{5/6} (r/r0)^{5/3} = 6.88 (r/r0)^{5/3}.  K = 2.2461.
    (The constant is often printed as 2.2698, which is larger by 2^{5/3}/pi and
    disagrees with 6.88 and with Noll's own tabulated residual variances.)
    """
    c = ((24.0 / 5.0) * gamma(6.0 / 5.0)) ** (5.0 / 6.0) * gamma(11.0 / 6.0) ** 2 / (2.0 * math.pi ** (11.0 / 3.0))
    return c * gamma(14.0 / 3.0) * 2.0 ** (-5.0 / 3.0) * math.pi ** (8.0 / 3.0)


def noll_covariance_entry(i: int, j: int) -> float:
    """E[a_i a_j] / (D/r0)^(5/3) for Noll indices i, j >= 2 (Noll's closed form).

    Zero unless the two modes share m and, for m > 0, the same angular function
    (both even or both odd indices).  Otherwise

      K sqrt((n+1)(n'+1)) (-1)^((n+n'-2m)/2) Gamma((n+n'-5/3)/2)
        / [Gamma((n-n'+17/3)/2) Gamma((n'-n+17/3)/2) Gamma((n+n'+23/3)/2)]

    with K = noll_constant().
    """
    ni, mi = noll_nm(i)
    nj, mj = noll_nm(j)
    if mi != mj:
        return 0.0
    if mi != 0 and (i % 2) != (j % 2):
        return 0.0
    sign = (-1) ** ((ni + nj - 2 * mi) // 2)
    lg = (gammaln((ni + nj - 5.0 / 3.0) / 2.0)
          - gammaln((ni - nj + 17.0 / 3.0) / 2.0)
          - gammaln((nj - ni + 17.0 / 3.0) / 2.0)
          - gammaln((ni + nj + 23.0 / 3.0) / 2.0))
    return noll_constant() * math.sqrt((ni + 1) * (nj + 1)) * sign * math.exp(lg)


def noll_matrix(J: int, D_over_r0: float = 1.0) -> np.ndarray:
    """A_0 for the J modes Noll 2..J+1 at strength D/r0 (Eq. A matrix at s = 0)."""
    A = np.empty((J, J))
    for a in range(J):
        for b in range(J):
            A[a, b] = noll_covariance_entry(a + 2, b + 2)
    return A * D_over_r0 ** (5.0 / 3.0)


def noll_cholesky(J: int, D_over_r0: float = 1.0) -> np.ndarray:
    """Lower Cholesky factor L with L L^T = A_0 (Sec. III-C, the mixing matrix of Fig. rand_gen)."""
    return np.linalg.cholesky(noll_matrix(J, D_over_r0))
