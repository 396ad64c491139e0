// Noll-indexed Zernike polynomials on the unit disk (Noll 1976), evaluated in FP64 for the device-built tables.
#pragma once

#include <math.h>

#include "common.cuh"

// (n, m) of Noll index j >= 1.
DFP2S_DEV void dfp2s_noll_nm(int j, int* n, int* m) {
  int nn = 0;
  while ((nn + 1) * (nn + 2) / 2 < j) ++nn;
  const int r = j - nn * (nn + 1) / 2 - 1;
  *n = nn;
  *m = (nn % 2 == 0) ? 2 * ((r + 1) / 2) : 2 * (r / 2) + 1;
}

// k! as an integer (k <= 20).
DFP2S_DEV long long dfp2s_factorial(int k) {
  long long f = 1;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

// Z_j(rho, theta): sqrt(n+1) R_n^0 (m = 0), sqrt(2(n+1)) R_n^m cos(m theta) (even j), sin(m theta) (odd j),
// R_n^m(rho) = sum_s (-1)^s (n-s)! / (s! ((n+m)/2-s)! ((n-m)/2-s)!) rho^(n-2s).  Each coefficient is a
// multinomial coefficient, formed exactly in integers (n <= 20); the powers of rho by repeated multiplication.
DFP2S_DEV double dfp2s_zernike(int j, double rho, double th) {
  int n, m;
  dfp2s_noll_nm(j, &n, &m);
  double R = 0.0;
  for (int s = 0; s <= (n - m) / 2; ++s) {
    const long long c = dfp2s_factorial(n - s) /
                        (dfp2s_factorial(s) * dfp2s_factorial((n + m) / 2 - s) * dfp2s_factorial((n - m) / 2 - s));
    double pw = 1.0;
    for (int e = 0; e < n - 2 * s; ++e) pw *= rho;
    R += ((s & 1) ? -(double)c : (double)c) * pw;
  }
  if (m == 0) return sqrt((double)(n + 1)) * R;
  return sqrt(2.0 * (n + 1)) * R * ((j & 1) ? sin(m * th) : cos(m * th));
}
