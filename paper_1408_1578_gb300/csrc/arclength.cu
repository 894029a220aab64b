// Closed-form curves sampled at points equispaced in arclength (host code).
//
// Section 2 of the paper works on a boundary sampled at equispaced points in
// arclength: n = 4^q p points, p per wavelength, cut into segments of 2^l p
// consecutive points whose length is 2^l wavelengths.  The library's curves
// are given by a parameter t in [0, 2 pi) that is not arclength, so this file
// computes, for a curve z(t):
//
//   s(t) = int_0^t |z'(u)| du           composite Gauss-Legendre quadrature
//                                        (16 points on each of M panels)
//   t_j  with s(t_j) = L j / n          Newton's method on s(t) - s_j, kept
//                                        inside the panel that brackets s_j
//                                        (bisection when a step leaves it)
//
// and returns z and its first two derivatives with respect to the rescaled
// arclength sigma = 2 pi s / L (constant speed g = L / (2 pi)) at
// sigma_j = 2 pi j / n.  With dt/dsigma = g / |z'| and
// d2t/dsigma2 = -g^2 (z'.z'') / |z'|^4:
//
//   z_sigma = z' dt/dsigma,   z_sigmasigma = z'' (dt/dsigma)^2 + z' d2t/dsigma2.
//
// The curves and the arclength map are in host_curve.h.
#include "host_curve.h"

using namespace cfie_host;

extern "C" cfie_status cfie_arclength_samples(cfie_curve kind, const double* params, int nparams,
                                              int n, double* z, double* dz, double* ddz,
                                              double* perimeter) {
  if (!z || !dz || !ddz || n < 8 || n % 2 != 0 || n > (1 << 20)) return CFIE_EINVAL;
  host_curve C;
  if (C.set(kind, params, nparams) != CFIE_OK) return CFIE_EINVAL;
  try {
    arclength_map A;
    if (A.build(C, std::max(256, n / 8)) != CFIE_OK) return CFIE_EINVAL;
    const double g = A.L / kTwoPi;
    for (int j = 0; j < n; ++j) {
      const double t = A.t_of_s(A.L * j / n);
      const point q = C.at(t);
      const double u2 = q.d[0] * q.d[0] + q.d[1] * q.d[1];
      const double dt = g / std::sqrt(u2);                              // dt/dsigma
      const double ddt = -g * g * (q.d[0] * q.e[0] + q.d[1] * q.e[1]) / (u2 * u2);
      for (int c = 0; c < 2; ++c) {
        z[2 * j + c] = q.z[c];
        dz[2 * j + c] = q.d[c] * dt;
        ddz[2 * j + c] = q.e[c] * dt * dt + q.d[c] * ddt;
      }
    }
    if (perimeter) *perimeter = A.L;
    return CFIE_OK;
  } catch (...) {
    return CFIE_ENOMEM;
  }
}
