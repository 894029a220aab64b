// Host-side curves of the library and their arclength map (host code only).
//
// host_curve evaluates z, z', z'' of the curves the cfie_geometry_* calls
// build.  arclength_map tabulates s(t) = int_0^t |z'(u)| du with composite
// Gauss-Legendre quadrature (16 points on each of M panels, compensated panel
// sums) and inverts it by Newton's method kept inside the panel that brackets
// the target (bisection when a step leaves it).  The Gauss-Legendre nodes are
// computed by Newton's method on the Legendre polynomial (three-term
// recurrence), not tabulated.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/cfie.h"

namespace cfie_host {

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
  cfie_curve kind = CFIE_CURVE_KITE;
  double p0 = 0, p1 = 0;
  std::vector<double> a, b;

  // CFIE_OK, or CFIE_EINVAL for parameters the matching constructor refuses
  cfie_status set(cfie_curve k, const double* params, int nparams) {
    if (nparams < 0 || (nparams > 0 && !params)) return CFIE_EINVAL;
    for (int i = 0; i < nparams; ++i)
      if (!std::isfinite(params[i])) return CFIE_EINVAL;
    kind = k;
    switch (k) {
      case CFIE_CURVE_CIRCLE:
        if (nparams != 1 || !(params[0] > 0)) return CFIE_EINVAL;
        p0 = params[0];
        return CFIE_OK;
      case CFIE_CURVE_ELLIPSE:
        if (nparams != 2 || !(params[0] > 0) || !(params[1] > 0)) return CFIE_EINVAL;
        p0 = params[0];
        p1 = params[1];
        return CFIE_OK;
      case CFIE_CURVE_STAR:
        if (nparams < 2 || nparams % 2 != 0 || nparams > 128) return CFIE_EINVAL;
        a.assign(params, params + nparams / 2);
        b.assign(params + nparams / 2, params + nparams);
        return CFIE_OK;
      case CFIE_CURVE_KITE:
        return nparams == 0 ? CFIE_OK : CFIE_EINVAL;
      default:
        return CFIE_EINVAL;
    }
  }

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

struct arclength_map {
  const host_curve* C = nullptr;
  int M = 0;                            // panels
  double hp = 0;                        // panel width in t
  double L = 0;                         // perimeter
  std::vector<double> S;                // s at the panel boundaries

  static const gauss_legendre& rule() {
    static const gauss_legendre G;
    return G;
  }
  // int_lo^hi |z'| by one Gauss-Legendre rule
  double arc(double lo, double hi) const {
    const gauss_legendre& G = rule();
    const double h = 0.5 * (hi - lo), m = 0.5 * (hi + lo);
    double acc = 0.0;
    for (int i = 0; i < kGL; ++i) acc += G.w[i] * C->speed(m + h * G.x[i]);
    return h * acc;
  }
  // CFIE_EINVAL if the speed comes near zero (or a star's r does not stay positive)
  cfie_status build(const host_curve& curve, int panels) {
    C = &curve;
    M = panels;
    hp = kTwoPi / M;
    S.assign(M + 1, 0.0);
    const gauss_legendre& G = rule();
    double run = 0.0, comp = 0.0;       // compensated (Neumaier) running sum
    double vmax = 0.0, vmin = INFINITY;
    for (int k = 0; k < M; ++k) {
      const double lo = k * hp;
      for (int i = 0; i < kGL; ++i) {
        const double t = lo + 0.5 * hp * (G.x[i] + 1.0);
        const double v = C->speed(t);
        vmax = std::max(vmax, v);
        vmin = std::min(vmin, v);
        if (C->kind == CFIE_CURVE_STAR) {        // r(t) = z(t) . (cos t, sin t) > 0
          const point q = C->at(t);
          if (!(q.z[0] * std::cos(t) + q.z[1] * std::sin(t) > 0)) return CFIE_EINVAL;
        }
      }
      const double piece = arc(lo, lo + hp), sum = run + piece;
      comp += std::fabs(run) >= std::fabs(piece) ? (run - sum) + piece : (piece - sum) + run;
      run = sum;
      S[k + 1] = run + comp;
    }
    if (!(vmin > 1e-12 * vmax) || !std::isfinite(S[M])) return CFIE_EINVAL;
    L = S[M];
    return CFIE_OK;
  }
  // the parameter t in [0, 2 pi] with s(t) = target, 0 <= target <= L
  double t_of_s(double target) const {
    int k = int(std::upper_bound(S.begin(), S.end(), target) - S.begin()) - 1;
    k = std::min(std::max(k, 0), M - 1);
    double lo = k * hp, hi = (k + 1) * hp;
    double t = lo + (target - S[k]) / (S[k + 1] - S[k]) * hp;
    for (int it = 0; it < 60; ++it) {
      const double f = S[k] + arc(k * hp, t) - target;
      if (f == 0.0) break;
      if (f > 0) hi = t; else lo = t;
      double tn = t - f / C->speed(t);
      if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
      const double step = std::fabs(tn - t);
      t = tn;
      if (step <= 1e-15 * kTwoPi) break;
    }
    return t;
  }
};

}  // namespace cfie_host
