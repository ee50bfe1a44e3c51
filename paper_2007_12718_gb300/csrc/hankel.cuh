// Device evaluation of the kernel G(r) = (i/4) H0^(1)(kappa r)  (Eq. 2) and of
// the corrected discrete kernel entries h^2 (G(h|m|) + tau_m)  (Eqs. 8, 10).
//
// H0^(1) = J0 + i Y0 is computed with our own routines, FP64:
//  * 0 < z <= 20: Miller's backward recurrence for J_k (k = N..0), normalised
//    with J0 + 2 sum J_2k = 1, and Neumann's series
//    Y0 = (2/pi) [(log(z/2) + gamma) J0 - 2 sum_{k>=1} (-1)^k J_2k / k]
//    (Abramowitz & Stegun 9.1.88, 9.12).  Absolute error ~ 1e-15.
//  * z > 20: Hankel's asymptotic expansion
//    H0^(1)(z) ~ sqrt(2/(pi z)) e^{i(z - pi/4)} sum_k i^k a_k z^-k,
//    a_k = prod_{j<=k} (-(2j-1)^2) / (k! 8^k)   (DLMF 10.17.5), 18 terms:
//    relative error ~ 3e-15 at z = 20, better beyond.
#pragma once
#include "common.cuh"

namespace ls {

struct KernelSpec {
  double kappa, h;
  int npts;            // number of corrected stencil offsets
  int m1[25], m2[25];  // stencil offsets
  double wr[25], wi[25];  // tau_m
};

__device__ __forceinline__ z64 hankel1_0(double z) {
  if (z <= 20.0) {
    int N = 2 * (int)((z + 25.0 + 4.0 * cbrt(z)) * 0.5);
    const double tz = 2.0 / z;
    double jp1 = 0.0, j = 1e-30, norm = 0.0, neu = 0.0;
    for (int k = N; k > 0; --k) {
      double jm1 = (k * tz) * j - jp1;
      if ((k & 1) == 0) {
        norm += 2.0 * j;
        int kk = k >> 1;
        neu += ((kk & 1) ? -j : j) / kk;
      }
      jp1 = j;
      j = jm1;
      if (fabs(j) > 1e250) {
        j *= 1e-250;
        jp1 *= 1e-250;
        norm *= 1e-250;
        neu *= 1e-250;
      }
    }
    norm += j;
    double J0 = j / norm;
    const double kEuler = 0.57721566490153286061;
    double Y0 = (2.0 / M_PI) * ((log(0.5 * z) + kEuler) * J0 - 2.0 * neu / norm);
    return mk<double>(J0, Y0);
  }
  // asymptotic: s = sum_k i^k a_k z^-k
  double sr = 0.0, si = 0.0, a = 1.0, zi = 1.0 / z, p = 1.0;
  for (int k = 0; k < 18; ++k) {
    double t = a * p;
    switch (k & 3) {
      case 0: sr += t; break;
      case 1: si += t; break;
      case 2: sr -= t; break;
      default: si -= t; break;
    }
    a *= -(double)((2 * k + 1) * (2 * k + 1)) / (8.0 * (k + 1));
    p *= zi;
  }
  double sn, cs;
  sincos(z, &sn, &cs);
  // e^{i(z - pi/4)} = e^{iz} (1 - i)/sqrt(2)
  const double r2 = 0.70710678118654752440;
  double er = (cs + sn) * r2, ei = (sn - cs) * r2;
  double amp = sqrt(2.0 / (M_PI * z));
  return mk<double>(amp * (er * sr - ei * si), amp * (er * si + ei * sr));
}

// G(r) = (i/4) H0^(1)(kappa r)
__device__ __forceinline__ z64 green(double z) {
  z64 hz = hankel1_0(z);
  return mk<double>(-0.25 * hz.im, 0.25 * hz.re);
}

// Corrected-stencil part tau_d (zero off the stencil), times h^2.
__device__ __forceinline__ z64 stencil_entry(const KernelSpec& ks, int d1, int d2) {
  z64 v = mk<double>(0.0, 0.0);
  if (abs(d1) + abs(d2) <= 3) {
    for (int p = 0; p < ks.npts; ++p)
      if (ks.m1[p] == d1 && ks.m2[p] == d2) {
        v.re += ks.wr[p];
        v.im += ks.wi[p];
      }
  }
  double h2 = ks.h * ks.h;
  return mk<double>(v.re * h2, v.im * h2);
}

// Discrete kernel entry for the lattice offset (d1, d2): h^2 (G(h|d|) + tau_d),
// with tau only on the stencil and h^2 tau_0 on the diagonal.
__device__ __forceinline__ z64 kernel_entry(const KernelSpec& ks, int d1, int d2) {
  z64 v = mk<double>(0.0, 0.0);
  if (d1 != 0 || d2 != 0) v = green(ks.kappa * ks.h * sqrt((double)d1 * d1 + (double)d2 * d2));
  if (abs(d1) + abs(d2) <= 3) {
    for (int p = 0; p < ks.npts; ++p)
      if (ks.m1[p] == d1 && ks.m2[p] == d2) {
        v.re += ks.wr[p];
        v.im += ks.wi[p];
      }
  }
  double h2 = ks.h * ks.h;
  return mk<double>(v.re * h2, v.im * h2);
}

// Lattice-offset table T[|d2| * tx + |d1|] = h^2 G(h |d|) (0 at d = 0): every
// kernel block of the build is a lookup in it plus the stencil correction.
struct KernelTable {
  const z64* t;
  int tx, ty;
};

__device__ __forceinline__ z64 table_entry(const KernelTable& kt, const KernelSpec& ks, int d1, int d2) {
  z64 v = kt.t[(long long)abs(d2) * kt.tx + abs(d1)];
  if (abs(d1) + abs(d2) <= 3) v = v + stencil_entry(ks, d1, d2);
  return v;
}

}  // namespace ls
