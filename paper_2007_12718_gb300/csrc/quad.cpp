// Corrected-trapezoidal quadrature weights for the 2D Helmholtz kernel
// (Sec. 2.2, Eq. 8, Fig. 1), computed on the host in long double.
//
// The paper fixes the stencils (the L1 diamonds of radius 0..3 for orders
// 4..10, Fig. 1) and states that the weights follow from the logarithmic
// singularity of H0 and the smoothness of sigma, depending on kappa*h only.
// Writing G(r) = -(1/2pi) J0(kappa r) log r + S(r), the punctured rule misses
// h^2 S(0) sigma_i plus the lattice finite parts of the log singularity:
// for every polynomial moment P the correction constants c_m must satisfy
//     sum_m c_m P(m) = (1/2) d/ds [ sum_{m != 0} P(m) |m|^{-2s} ] at s = 0,
// for the D4-invariant P of degree <= 2r.  Then
//     tau_0 = i/4 - (1/2pi) (log(kappa h / 2) + gamma + c_0)
//     tau_m = -(1/2pi) c_m J0(kappa h |m|)          (m != 0).
// The zeta derivatives are evaluated here from the Mellin transform of lattice
// theta series, split at t = 1 and folded with the theta inversion formula
// (Jacobi for P = |u|^2j, Hecke for the harmonic H4 = u1^4 - 6u1^2u2^2 + u2^4);
// the t-integrals are done by composite Gauss-Legendre quadrature.
#include <math.h>
#include <string.h>

#include "quad.h"

namespace ls {
namespace {

typedef long double ld;
const ld kPi = 3.141592653589793238462643383279502884L;
const ld kEuler = 0.577215664901532860606512090082402431L;

// theta_P(t) = sum_{m != 0} P(m) exp(-pi t |m|^2) for P = |m|^(2j) (harm = 0)
// or P = |m|^(2j) H4(m) (harm = 1); |m| <= 9 is exact to far below 1e-30 for t >= 1.
ld theta(ld t, int j, int harm) {
  ld s = 0;
  for (int a = -9; a <= 9; ++a)
    for (int b = -9; b <= 9; ++b) {
      if (!a && !b) continue;
      ld r2 = (ld)(a * a + b * b);
      ld p = powl(r2, (ld)j);
      if (harm) p *= (ld)a * a * a * a - 6.0L * a * a * b * b + (ld)b * b * b * b;
      s += p * expl(-kPi * t * r2);
    }
  return s;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, ld* x, ld* w) {
  for (int i = 0; i < n; ++i) {
    ld z = cosl(kPi * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) {
        ld p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      ld dp = n * (z * p1 - p0) / (z * z - 1);
      ld dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    ld p0 = 1, p1 = z;
    for (int k = 2; k <= n; ++k) {
      ld p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    ld dp = n * (z * p1 - p0) / (z * z - 1);
    x[i] = z;
    w[i] = 2 / ((1 - z * z) * dp * dp);
  }
}

// int_1^inf (t^a1 + t^a2) theta_P(t) dt; theta decays like exp(-pi t).
ld mellin_tail(ld a1, ld a2, int j, int harm) {
  const int n = 20;
  ld x[n], w[n];
  gauss_legendre(n, x, w);
  ld s = 0;
  const ld width = 0.5L;
  for (ld lo = 1; lo < 40; lo += width) {
    for (int i = 0; i < n; ++i) {
      ld t = lo + width * (x[i] + 1) / 2;
      s += width / 2 * w[i] * (powl(t, a1) + powl(t, a2)) * theta(t, j, harm);
    }
  }
  return s;
}

// Z'(-j) for Z(s) = sum' |m|^-2s, j = 0..3.
ld zeta_lattice_deriv(int j) {
  if (j == 0) {
    // pi^-s Gamma(s) Z(s) = F(s) - 1/s, F(s) = int_1^inf (t^(s-1) + t^-s) theta dt + 1/(s-1)
    ld F0 = mellin_tail(-1, 0, 0, 0) - 1;
    return F0 - kEuler - logl(kPi);
  }
  ld lam = mellin_tail(-j - 1, j, 0, 0) + 1.0L / (-j - 1) + 1.0L / j;
  ld fact = 1;
  for (int k = 2; k <= j; ++k) fact *= k;
  ld sign = (j % 2) ? -1 : 1;
  return powl(kPi, -(ld)j) * sign * fact * lam;
}

// Z_H4'(-j), j = 0, 1, for Z_H4(s) = sum' H4(m) |m|^-2s (theta_H4(t) = t^-5 theta_H4(1/t)).
ld zeta_h4_deriv(int j) {
  ld lam = mellin_tail(-j - 1, 4 + j, 0, 1);
  return j == 0 ? lam : -lam / kPi;
}

ld bessel_j0_series(ld z) {
  ld q = -z * z / 4, term = 1, s = 1;
  for (int k = 1; k < 80; ++k) {
    term *= q / ((ld)k * k);
    s += term;
    if (fabsl(term) < 1e-30L) break;
  }
  return s;
}

void solve_small(int n, ld* A, ld* b) {  // Gaussian elimination, partial pivoting
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (fabsl(A[i * n + k]) > fabsl(A[p * n + k])) p = i;
    if (p != k) {
      for (int c = 0; c < n; ++c) {
        ld t = A[k * n + c];
        A[k * n + c] = A[p * n + c];
        A[p * n + c] = t;
      }
      ld t = b[k];
      b[k] = b[p];
      b[p] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      ld f = A[i * n + k] / A[k * n + k];
      for (int c = k; c < n; ++c) A[i * n + c] -= f * A[k * n + c];
      b[i] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    ld s = b[k];
    for (int c = k + 1; c < n; ++c) s -= A[k * n + c] * b[c];
    b[k] = s / A[k * n + k];
  }
}

// Cached moment targets (1/2) Z_P'(0) for P = 1, |u|^2, |u|^4, H4, |u|^6, |u|^2 H4.
struct Targets {
  bool ready = false;
  ld v[6];
};
Targets g_targets;

const ld* targets() {
  if (!g_targets.ready) {
    g_targets.v[0] = 0.5L * zeta_lattice_deriv(0);
    g_targets.v[1] = 0.5L * zeta_lattice_deriv(1);
    g_targets.v[2] = 0.5L * zeta_lattice_deriv(2);
    g_targets.v[3] = 0.5L * zeta_h4_deriv(0);
    g_targets.v[4] = 0.5L * zeta_lattice_deriv(3);
    g_targets.v[5] = 0.5L * zeta_h4_deriv(1);
    g_targets.ready = true;
  }
  return g_targets.v;
}

int orbit_key(int a, int b) {
  a = a < 0 ? -a : a;
  b = b < 0 ? -b : b;
  int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo * 16 + hi;
}

}  // namespace

void lattice_zeta_targets(double out[6]) {
  const ld* t = targets();
  for (int i = 0; i < 6; ++i) out[i] = (double)t[i];
}

int quad_corrections(int order, double kh, QuadCorr* out) {
  memset(out, 0, sizeof(*out));
  if (order == 2) return 0;
  int r;
  switch (order) {
    case 4: r = 0; break;
    case 6: r = 1; break;
    case 8: r = 2; break;
    case 10: r = 3; break;
    default: return -1;
  }
  const int neq = (r == 0) ? 1 : (r == 1) ? 2 : (r == 2) ? 4 : 6;
  // stencil points and their orbits
  int keys[8], nkeys = 0;
  for (int b = -r; b <= r; ++b)
    for (int a = -r; a <= r; ++a) {
      if (abs(a) + abs(b) > r) continue;
      out->m1[out->npts] = a;
      out->m2[out->npts] = b;
      ++out->npts;
      int k = orbit_key(a, b), f = 0;
      for (int i = 0; i < nkeys; ++i) f |= keys[i] == k;
      if (!f) keys[nkeys++] = k;
    }
  if (nkeys != neq) return -1;
  ld A[36] = {0}, c[6];
  for (int e = 0; e < neq; ++e) c[e] = targets()[e];
  for (int p = 0; p < out->npts; ++p) {
    ld a = out->m1[p], b = out->m2[p];
    ld r2 = a * a + b * b, h4 = a * a * a * a - 6 * a * a * b * b + b * b * b * b;
    ld basis[6] = {1, r2, r2 * r2, h4, r2 * r2 * r2, r2 * h4};
    int col = 0;
    for (int i = 0; i < nkeys; ++i)
      if (keys[i] == orbit_key(out->m1[p], out->m2[p])) col = i;
    for (int e = 0; e < neq; ++e) A[e * neq + col] += basis[e];
  }
  solve_small(neq, A, c);
  for (int p = 0; p < out->npts; ++p) {
    int col = 0;
    for (int i = 0; i < nkeys; ++i)
      if (keys[i] == orbit_key(out->m1[p], out->m2[p])) col = i;
    ld cm = c[col];
    if (out->m1[p] == 0 && out->m2[p] == 0) {
      out->wr[p] = (double)(-(logl((ld)kh / 2) + kEuler + cm) / (2 * kPi));
      out->wi[p] = 0.25;
    } else {
      ld rr = sqrtl((ld)out->m1[p] * out->m1[p] + (ld)out->m2[p] * out->m2[p]);
      out->wr[p] = (double)(-cm * bessel_j0_series((ld)kh * rr) / (2 * kPi));
      out->wi[p] = 0.0;
    }
  }
  return 0;
}

}  // namespace ls
