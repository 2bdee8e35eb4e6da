// Confocal ellipses of the Chebyshev filter of the Arnoldi iteration (Section 1 methods paragraph and its
// ref. 21): the level of a point in a family of real-centred confocal ellipses, the rightmost real point
// of one ellipse, and the scan that picks the ellipse enclosing the unwanted Ritz values with the best
// damping of the wanted ones.  Host only (FP64).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "fv_internal.h"

namespace fv {

// |w| with w = xi + sqrt(xi^2 - 1), xi = (z - d)/c, the branch with |w| >= 1: the level of z in the
// family of ellipses with foci d +- c (c^2 real, possibly negative; c^2 = 0 gives circles about d).
double ellipse_level(double zr, double zi, double d, double c2) {
  const std::complex<double> z(zr, zi);
  if (std::fabs(c2) < 1e-300) return std::abs(z - d);
  const std::complex<double> c = std::sqrt(std::complex<double>(c2, 0.0));
  const std::complex<double> xi = (z - d) / c;
  const std::complex<double> s = std::sqrt(xi * xi - 1.0);
  return std::max(std::abs(xi + s), std::abs(xi - s));
}

// Rightmost real point of the confocal ellipse of the given level: z = d + c (w + 1/w) / 2, |w| = level
// (w = level for real foci, w = -i level for imaginary foci; a circle of radius `level` for c^2 = 0).
double ellipse_right_end(double d, double c2, double level) {
  if (std::fabs(c2) < 1e-300) return d + level;
  if (c2 > 0.0) return d + std::sqrt(c2) * (level + 1.0 / level) / 2.0;
  return d + std::sqrt(-c2) * (level - 1.0 / level) / 2.0;
}

// Scan of real-centred confocal ellipses maximising min_w level(w) / max_u level(u), among those whose
// rightmost real point stays left of every wanted real part (anything on the real axis further right
// would rank among the wanted and must not be damped; at high Gr the first Ritz values are far-off ones
// with large imaginary parts, and an ellipse around them can cover the leading eigenvalues near the
// origin); the best of all if no candidate qualifies.
void best_ellipse(const std::vector<Ritz>& wanted, const std::vector<Ritz>& unwanted, double& d_out,
                         double& c2_out, double& rate_out) {
  double amin = 1e300, amax = -1e300, bmax = 0.0, wleft = 1e300;
  for (auto& u : unwanted) {
    amin = std::min(amin, u.re);
    amax = std::max(amax, u.re);
    bmax = std::max(bmax, std::fabs(u.im));
  }
  for (auto& w : wanted) wleft = std::min(wleft, w.re);
  const double span = std::max(amax - amin, 1e-12 * std::max(1.0, std::fabs(amax)));
  double rate_any = -1.0, d_any = 0.0, c2_any = 0.0;
  rate_out = -1.0;
  for (int a = 0; a < 13; ++a) {
    const double d = amin + (0.2 + 0.05 * a) * span;
    const double a0 = std::max(amax - d, d - amin);
    for (int t = 0; t <= 40; ++t) {
      const double c2 = (-1.0 + 0.05 * t) * std::max(a0 * a0, bmax * bmax);
      double lu = 0.0, lw = 1e300;
      for (auto& u : unwanted) lu = std::max(lu, ellipse_level(u.re, u.im, d, c2));
      for (auto& w : wanted) lw = std::min(lw, ellipse_level(w.re, w.im, d, c2));
      const double rate = lu > 0.0 ? lw / lu : 1e300;
      if (rate > rate_any) {
        rate_any = rate;
        d_any = d;
        c2_any = c2;
      }
      if (ellipse_right_end(d, c2, lu) <= wleft && rate > rate_out) {
        rate_out = rate;
        d_out = d;
        c2_out = c2;
      }
    }
  }
  if (rate_out < 0.0) {
    rate_out = rate_any;
    d_out = d_any;
    c2_out = c2_any;
  }
}

}  // namespace fv
