// Host-side corrected-quadrature weights (Sec. 2.2, Eq. 8, Fig. 1).
#pragma once

namespace ls {

// tau_m for the order-p stencil at kappa*h: entry (m1[i], m2[i]) of the
// discrete kernel gets h^2 * (wr[i] + i wi[i]) added (on top of h^2 G(h|m|)
// for m != 0; the diagonal is h^2 tau_0 alone).
struct QuadCorr {
  int npts;
  int m1[25], m2[25];
  double wr[25], wi[25];
};

// Returns 0, or -1 for an unsupported order.  order 2 = punctured rule (no points).
int quad_corrections(int order, double kh, QuadCorr* out);

// (1/2) Z_P'(0) for P = 1, |u|^2, |u|^4, H4, |u|^6, |u|^2 H4 (for tests).
void lattice_zeta_targets(double out[6]);

}  // namespace ls
