// Level blocks of the directional preconditioner (Section 2.2), host code.
//
// With the n nodes equispaced in arclength (spacing L / n, speed
// g = L / (2 pi) in the rescaled parameter), every segment of level l holds
// c = 2^l p nodes and all its blocks depend on l only:
//
//   B_l   the sound-soft operator restricted to a straight segment of c nodes
//         with that spacing and speed (Section 2.1): the Kress-Nystrom entries
//         R_|a-b| M1 + h (M - M1 log(4 sin^2(pi (a - b) / n))) of the
//         single-layer kernel on the line (the double-layer kernel and the
//         curvature term vanish there), B_l = 1/2 I - i eta S_l;
//   U_l   the partial Fourier matrix U(x, k) = exp(i k (rho(x) - rho(c))) on
//         the 2^(l+1) + 1 wave numbers k_m = -omega + m 2 omega / 2^(l+1),
//         rho(x) - rho(c) = (x - (c - 1) / 2) L / n;
//   T_l   (U_l^t B_l^-1 U_l)^-1, U^t the plain transpose (eq. fac).
//
// The Kress weights R_d = -(4 pi / n) sum_{m=1}^{n/2-1} cos(2 pi m d / n) / m
// - (4 pi / n^2) (-1)^d are summed with the index m d reduced mod n exactly;
// J0 and Y0 come from the C++17 special functions.  Inverses: Gaussian
// elimination with partial pivoting on [A | I].
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "../../include/cfie.h"

namespace {

using cplx = std::complex<double>;
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double kEulerGamma = 0.57721566490153286060651209008240243;

// y[c] -= f x[c] for c < len, in real arithmetic (std::complex products take
// the slow path that handles infinities and NaNs)
inline void axpy_neg(cplx f, const cplx* x, cplx* y, int len) {
  const double fr = f.real(), fi = f.imag();
  const double* xs = reinterpret_cast<const double*>(x);
  double* ys = reinterpret_cast<double*>(y);
  for (int c = 0; c < len; ++c) {
    const double xr = xs[2 * c], xi = xs[2 * c + 1];
    ys[2 * c] -= fr * xr - fi * xi;
    ys[2 * c + 1] -= fr * xi + fi * xr;
  }
}

// A^-1 of a k x k row-major matrix; false if a pivot vanishes
bool invert(std::vector<cplx>& A, int k, std::vector<cplx>& out) {
  out.assign((size_t)k * k, cplx(0.0));
  for (int i = 0; i < k; ++i) out[(size_t)i * k + i] = 1.0;
  for (int col = 0; col < k; ++col) {
    int piv = col;
    double best = std::abs(A[(size_t)col * k + col]);
    for (int r = col + 1; r < k; ++r) {
      const double v = std::abs(A[(size_t)r * k + col]);
      if (v > best) best = v, piv = r;
    }
    if (!(best > 0)) return false;
    if (piv != col) {
      for (int c = 0; c < k; ++c) {
        std::swap(A[(size_t)piv * k + c], A[(size_t)col * k + c]);
        std::swap(out[(size_t)piv * k + c], out[(size_t)col * k + c]);
      }
    }
    const cplx inv = 1.0 / A[(size_t)col * k + col];
    for (int c = 0; c < k; ++c) {
      A[(size_t)col * k + c] *= inv;
      out[(size_t)col * k + c] *= inv;
    }
    for (int r = 0; r < k; ++r) {
      if (r == col) continue;
      const cplx f = A[(size_t)r * k + col];
      if (f == 0.0) continue;
      axpy_neg(f, &A[(size_t)col * k], &A[(size_t)r * k], k);
      axpy_neg(f, &out[(size_t)col * k], &out[(size_t)r * k], k);
    }
  }
  return true;
}

void store(const std::vector<cplx>& a, double* dst) {
  if (!dst) return;
  for (size_t i = 0; i < a.size(); ++i) {
    dst[2 * i] = a[i].real();
    dst[2 * i + 1] = a[i].imag();
  }
}

}  // namespace

extern "C" cfie_status cfie_dirprec_level(int n, int p, int level, double omega, double eta,
                                          double L, double* B, double* Binv, double* U,
                                          double* T) {
  if (n < 8 || n % 2 != 0 || n > (1 << 20) || p < 1 || level < 0 || level > 20) return CFIE_EINVAL;
  const long long cl = (1LL << level) * p;
  if (cl > n / 2 || cl > 1024) return CFIE_EINVAL;
  if (!(omega > 0) || !(eta > 0) || !(L > 0) || !std::isfinite(omega) || !std::isfinite(eta) ||
      !std::isfinite(L))
    return CFIE_EINVAL;
  try {
    const int c = int(cl), K = (1 << (level + 1)) + 1;
    const double h = 2.0 * kPi / n, g = L / (2.0 * kPi);
    // Kress weights R_0 .. R_{c-1}
    std::vector<double> cosk(n), R(c);
    for (int k = 0; k < n; ++k) cosk[k] = std::cos(2.0 * kPi * k / n);
    for (int d = 0; d < c; ++d) {
      double acc = 0.0;
      long long idx = d % n;
      for (int m = 1; m < n / 2; ++m) {
        acc += cosk[idx] / m;
        idx += d;
        if (idx >= n) idx -= n;
      }
      R[d] = -(4.0 * kPi / n) * acc - (4.0 * kPi / ((double)n * n)) * ((d & 1) ? -1.0 : 1.0);
    }
    // B_l = 1/2 I - i eta S_l on the line
    std::vector<cplx> Bm((size_t)c * c);
    const cplx I(0.0, 1.0);
    const double m1d = -g / (4.0 * kPi);
    const cplx m2d = (cplx(0.0, 0.25) - kEulerGamma / (2.0 * kPi) -
                      std::log(omega * g / 2.0) / (2.0 * kPi)) * g;
    // the block is Toeplitz: one single-layer entry per distance d = |a - b|
    std::vector<cplx> srow(c);
    srow[0] = R[0] * m1d + h * m2d;
    for (int d = 1; d < c; ++d) {
      const double x = omega * d * h * g;
      const double j0 = std::cyl_bessel_j(0.0, x), y0 = std::cyl_neumann(0.0, x);
      const cplx M = cplx(0.0, 0.25) * cplx(j0, y0) * g;
      const double M1 = -j0 * g / (4.0 * kPi);
      const double sn = std::sin(kPi * d / n);
      srow[d] = R[d] * M1 + h * (M - M1 * std::log(4.0 * sn * sn));
    }
    for (int a = 0; a < c; ++a)
      for (int b = 0; b < c; ++b)
        Bm[(size_t)a * c + b] = (a == b ? 0.5 : 0.0) - I * eta * srow[std::abs(a - b)];
    store(Bm, B);
    std::vector<cplx> work = Bm, Bi;
    if (!invert(work, c, Bi)) return CFIE_EINVAL;
    store(Bi, Binv);
    // U_l and T_l = (U^t B^-1 U)^-1
    std::vector<cplx> Um((size_t)c * K);
    const double step = 2.0 * omega / (K - 1);
    for (int x = 0; x < c; ++x) {
      const double rho = (x - 0.5 * (c - 1)) * (L / n);
      for (int m = 0; m < K; ++m) {
        const double k = m == K - 1 ? omega : -omega + m * step;
        Um[(size_t)x * K + m] = std::polar(1.0, k * rho);
      }
    }
    store(Um, U);
    if (T) {
      std::vector<cplx> BU((size_t)c * K, cplx(0.0)), S((size_t)K * K, cplx(0.0)), Tm;
      for (int a = 0; a < c; ++a)
        for (int b = 0; b < c; ++b)
          axpy_neg(-Bi[(size_t)a * c + b], &Um[(size_t)b * K], &BU[(size_t)a * K], K);
      for (int x = 0; x < c; ++x)
        for (int r = 0; r < K; ++r)
          axpy_neg(-Um[(size_t)x * K + r], &BU[(size_t)x * K], &S[(size_t)r * K], K);
      if (!invert(S, K, Tm)) return CFIE_EINVAL;
      store(Tm, T);
    }
    return CFIE_OK;
  } catch (...) {
    return CFIE_ENOMEM;
  }
}

// T~: the `keep` largest entries of a K x K block in modulus, the rest zero
// (Section 2.2: T is numerically sparse; the number kept is proportional to K).
// Entries within a relative 2^-30 of the smallest modulus kept count as tied
// with it and are all kept: T is symmetric (and on a straight segment also
// symmetric about its anti-diagonal), so equal entries differ only by
// rounding, and the choice must not depend on it.
extern "C" cfie_status cfie_dirprec_threshold(int K, const double* T, int keep, double* Tt) {
  if (K < 1 || K > 4097 || !T || !Tt || keep < 0) return CFIE_EINVAL;
  try {
    const size_t total = (size_t)K * K;
    if ((size_t)keep >= total) {
      std::copy(T, T + 2 * total, Tt);
      return CFIE_OK;
    }
    std::vector<double> mag(total);
    for (size_t i = 0; i < total; ++i) mag[i] = std::hypot(T[2 * i], T[2 * i + 1]);
    double cut = INFINITY;
    if (keep > 0) {
      std::vector<double> sorted = mag;
      std::nth_element(sorted.begin(), sorted.begin() + (total - keep), sorted.end());
      cut = sorted[total - keep] * (1.0 - 0x1p-30);
    }
    for (size_t i = 0; i < total; ++i) {
      const bool in = keep > 0 && mag[i] >= cut;
      Tt[2 * i] = in ? T[2 * i] : 0.0;
      Tt[2 * i + 1] = in ? T[2 * i + 1] : 0.0;
    }
    return CFIE_OK;
  } catch (...) {
    return CFIE_ENOMEM;
  }
}
