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
// The Gauss-Legendre nodes are computed here by Newton's method on the
// Legendre polynomial (three-term recurrence), not tabulated.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/cfie.h"

namespace {

constexpr int kGL = 16;                 // Gauss-Legendre points per panel
constexpr double kTwoPi = 6.283185307179586476925286766559;

struct gauss_legendre {
  double x[kGL], w[kGL];                // nodes and weights on [-1, 1]
  gauss_legendre() {
    const double pi = kTwoPi / 2;
    for (int i = 0; i < kGL; ++i) {
      double r = std::cos(pi * (i + 0.75) / (kGL + 0.5));
      double dp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = r;        // P_0, P_1, then P_k by the recurrence
        for (int k = 2; k <= kGL; ++k) {
          const double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = kGL * (r * p1 - p0) / (r * r - 1.0);
        const double step = p1 / dp;
        r -= step;
        if (std::fabs(step) < 1e-16) break;
      }
      x[i] = r;
      w[i] = 2.0 / ((1.0 - r * r) * dp * dp);
    }
  }
};

struct point { double z[2], d[2], e[2]; };   // z, z', z'' at one parameter

struct host_curve {
  cfie_curve kind;
  double p0 = 0, p1 = 0;
  std::vector<double> a, b;

  point at(double t) const {
    point q;
    const double c = std::cos(t), s = std::sin(t);
    switch (kind) {
      case CFIE_CURVE_CIRCLE:
        q = {{p0 * c, p0 * s}, {-p0 * s, p0 * c}, {-p0 * c, -p0 * s}};
        break;
      case CFIE_CURVE_ELLIPSE:
        q = {{p0 * c, p1 * s}, {-p0 * s, p1 * c}, {-p0 * c, -p1 * s}};
        break;
      case CFIE_CURVE_STAR: {
        double r = 1.0, dr = 0.0, ddr = 0.0;
        for (size_t k = 1; k <= a.size(); ++k) {
          const double ck = std::cos(k * t), sk = std::sin(k * t);
          r += a[k - 1] * ck + b[k - 1] * sk;
          dr += k * (b[k - 1] * ck - a[k - 1] * sk);
          ddr -= double(k * k) * (a[k - 1] * ck + b[k - 1] * sk);
        }
        q = {{r * c, r * s},
             {dr * c - r * s, dr * s + r * c},
             {ddr * c - 2 * dr * s - r * c, ddr * s + 2 * dr * c - r * s}};
        break;
      }
      default: {                        // kite
        const double c2 = std::cos(2 * t), s2 = std::sin(2 * t);
        q = {{c + 0.65 * c2 - 0.65, 1.5 * s},
             {-s - 1.3 * s2, 1.5 * c},
             {-c - 2.6 * c2, -1.5 * s}};
      }
    }
    return q;
  }
  double speed(double t) const {
    const point q = at(t);
    return std::hypot(q.d[0], q.d[1]);
  }
};

// int_lo^hi |z'| by one Gauss-Legendre rule
double arc(const host_curve& C, const gauss_legendre& G, double lo, double hi) {
  const double h = 0.5 * (hi - lo), m = 0.5 * (hi + lo);
  double acc = 0.0;
  for (int i = 0; i < kGL; ++i) acc += G.w[i] * C.speed(m + h * G.x[i]);
  return h * acc;
}

bool finite_all(const double* v, int count) {
  for (int i = 0; i < count; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

}  // namespace

extern "C" cfie_status cfie_arclength_samples(cfie_curve kind, const double* params, int nparams,
                                              int n, double* z, double* dz, double* ddz,
                                              double* perimeter) {
  if (!z || !dz || !ddz || n < 8 || n % 2 != 0 || n > (1 << 20)) return CFIE_EINVAL;
  if (nparams < 0 || (nparams > 0 && !params) || (params && !finite_all(params, nparams)))
    return CFIE_EINVAL;
  host_curve C;
  C.kind = kind;
  switch (kind) {
    case CFIE_CURVE_CIRCLE:
      if (nparams != 1 || !(params[0] > 0)) return CFIE_EINVAL;
      C.p0 = params[0];
      break;
    case CFIE_CURVE_ELLIPSE:
      if (nparams != 2 || !(params[0] > 0) || !(params[1] > 0)) return CFIE_EINVAL;
      C.p0 = params[0];
      C.p1 = params[1];
      break;
    case CFIE_CURVE_STAR:
      if (nparams < 2 || nparams % 2 != 0 || nparams > 128) return CFIE_EINVAL;
      C.a.assign(params, params + nparams / 2);
      C.b.assign(params + nparams / 2, params + nparams);
      break;
    case CFIE_CURVE_KITE:
      if (nparams != 0) return CFIE_EINVAL;
      break;
    default:
      return CFIE_EINVAL;
  }
  try {
    static const gauss_legendre G;
    // panels of the cumulative arclength table; the nodes also check that the
    // speed stays away from zero (and, for the star, that r stays positive)
    const int M = std::max(256, n / 8);
    const double hp = kTwoPi / M;
    std::vector<double> S(M + 1, 0.0);
    double run = 0.0, comp = 0.0;       // compensated (Neumaier) running sum
    double vmax = 0.0, vmin = INFINITY;
    for (int k = 0; k < M; ++k) {
      const double lo = k * hp;
      for (int i = 0; i < kGL; ++i) {
        const double t = lo + 0.5 * hp * (G.x[i] + 1.0);
        const double v = C.speed(t);
        vmax = std::max(vmax, v);
        vmin = std::min(vmin, v);
        if (kind == CFIE_CURVE_STAR) {          // r(t) = z(t) . (cos t, sin t) > 0
          const point q = C.at(t);
          if (!(q.z[0] * std::cos(t) + q.z[1] * std::sin(t) > 0)) return CFIE_EINVAL;
        }
      }
      const double piece = arc(C, G, lo, lo + hp), sum = run + piece;
      comp += std::fabs(run) >= std::fabs(piece) ? (run - sum) + piece : (piece - sum) + run;
      run = sum;
      S[k + 1] = run + comp;
    }
    if (!(vmin > 1e-12 * vmax) || !std::isfinite(S[M])) return CFIE_EINVAL;
    const double L = S[M];
    const double g = L / kTwoPi;
    for (int j = 0; j < n; ++j) {
      const double target = L * j / n;
      // panel k with S[k] <= target < S[k + 1]
      int k = int(std::upper_bound(S.begin(), S.end(), target) - S.begin()) - 1;
      k = std::min(std::max(k, 0), M - 1);
      double lo = k * hp, hi = (k + 1) * hp;
      double t = lo + (target - S[k]) / (S[k + 1] - S[k]) * hp;
      for (int it = 0; it < 60; ++it) {
        const double f = S[k] + arc(C, G, k * hp, t) - target;
        if (f == 0.0) break;
        if (f > 0) hi = t; else lo = t;
        double tn = t - f / C.speed(t);
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        const double step = std::fabs(tn - t);
        t = tn;
        if (step <= 1e-15 * kTwoPi) break;
      }
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
    if (perimeter) *perimeter = L;
    return CFIE_OK;
  } catch (...) {
    return CFIE_ENOMEM;
  }
}
