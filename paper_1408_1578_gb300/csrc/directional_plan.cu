// Structure of the directional preconditioner (Section 2.1), host code.
//
// For a curve sampled at n = 4^q p points equispaced in arclength (p points
// per wavelength lambda = L p / n):
//
//   segments   the curve, from its point at t = 0, is cut into 2^q pieces of
//              2^q p points (length 2^q lambda); a piece of level l
//              (2^l p points) is kept when 2^l <= 2^q / sqrt(c), c the largest
//              |curvature| at its nodes (almost planar), or when 2^l <= m_leaf
//              (a non-planar leaf), and is halved otherwise;
//   centres    c_i, the curve point at the arclength halfway between the
//              segment's first and last node, and t_i the unit tangent there;
//   wave numbers  for i != j, a_ij = (c_i - c_j) / |c_i - c_j|,
//              k^i_ij = [omega a_ij . t_i]_i and k^j_ij = [-omega a_ij . t_j]_j,
//              [k]_l rounding to the nearest of the 2^(l+1) + 1 equispaced
//              points of [-omega, omega] (ties away from zero), returned as
//              grid indices.
//
// Curvature is kappa = (x' y'' - y' x'') / |z'|^3 at the nodes, which does not
// depend on the parametrisation.  The curves and the arclength map are in
// host_curve.h.
#include "host_curve.h"

using namespace cfie_host;

namespace {

// index of [k]_l among the 2^(l+1) + 1 grid points of [-omega, omega]
int round_to_grid(double k, int level, double omega) {
  const int m = 1 << (level + 1);
  const double v = (k + omega) * m / (2.0 * omega);
  const double idx = k >= 0 ? std::floor(v + 0.5) : std::ceil(v - 0.5);
  return int(std::min(std::max(idx, 0.0), double(m)));
}

}  // namespace

extern "C" cfie_status cfie_dirprec_plan(cfie_curve kind, const double* params, int nparams,
                                         int q, int p, double omega, int m_leaf, int capacity,
                                         int* m, int* first, int* level, int* kpair) {
  if (!m || q < 1 || q > 9 || p < 1 || m_leaf < 1 || !(omega > 0) || !std::isfinite(omega))
    return CFIE_EINVAL;
  const long long nl = (1LL << (2 * q)) * p;
  if (nl < 8 || nl % 2 != 0 || nl > (1 << 20)) return CFIE_EINVAL;
  const bool want = first || level || kpair;
  if (want && (!first || !level || !kpair || capacity < 1)) return CFIE_EINVAL;
  const int n = int(nl);
  host_curve C;
  if (C.set(kind, params, nparams) != CFIE_OK) return CFIE_EINVAL;
  try {
    arclength_map A;
    if (A.build(C, std::max(256, n / 8)) != CFIE_OK) return CFIE_EINVAL;
    const double L = A.L;
    std::vector<double> kappa(n);
    for (int j = 0; j < n; ++j) {
      const point z = C.at(A.t_of_s(L * j / n));
      const double sp = std::hypot(z.d[0], z.d[1]);
      kappa[j] = std::fabs(z.d[0] * z.e[1] - z.d[1] * z.e[0]) / (sp * sp * sp);
    }
    // the partition, in order along the curve
    std::vector<int> fst, lev;
    std::vector<std::pair<int, int>> stack;
    const double top = std::ldexp(1.0, q);
    for (int k = (1 << q) - 1; k >= 0; --k) stack.push_back({k * (1 << q) * p, q});
    while (!stack.empty()) {
      const auto [f, l] = stack.back();
      stack.pop_back();
      const int cnt = (1 << l) * p;
      const double c = *std::max_element(kappa.begin() + f, kappa.begin() + f + cnt);
      const double len = std::ldexp(1.0, l);
      if (len <= top / std::sqrt(c) || len <= m_leaf) {
        fst.push_back(f);
        lev.push_back(l);
      } else {                          // second half below the first: first half next
        stack.push_back({f + cnt / 2, l - 1});
        stack.push_back({f, l - 1});
      }
    }
    const int ms = int(fst.size());
    *m = ms;
    if (!want) return CFIE_OK;
    if (capacity < ms) return CFIE_EINVAL;
    // centres and unit tangents
    std::vector<double> cx(ms), cy(ms), tx(ms), ty(ms);
    for (int i = 0; i < ms; ++i) {
      const int cnt = (1 << lev[i]) * p;
      const double cs = L * fst[i] / n + 0.5 * (cnt - 1) * (L / n);
      const point z = C.at(A.t_of_s(cs));
      const double sp = std::hypot(z.d[0], z.d[1]);
      cx[i] = z.z[0];
      cy[i] = z.z[1];
      tx[i] = z.d[0] / sp;
      ty[i] = z.d[1] / sp;
      first[i] = fst[i];
      level[i] = lev[i];
    }
    for (int i = 0; i < ms; ++i) {
      for (int j = 0; j < ms; ++j) {
        int* out = kpair + 2 * ((size_t)i * ms + j);
        if (i == j) {
          out[0] = out[1] = 0;
          continue;
        }
        double ax = cx[i] - cx[j], ay = cy[i] - cy[j];
        const double r = std::hypot(ax, ay);
        ax /= r;
        ay /= r;
        out[0] = round_to_grid((omega * ax) * tx[i] + (omega * ay) * ty[i], lev[i], omega);
        out[1] = round_to_grid((-omega * ax) * tx[j] + (-omega * ay) * ty[j], lev[j], omega);
      }
    }
    return CFIE_OK;
  } catch (...) {
    return CFIE_ENOMEM;
  }
}

// Positions of W~ = E + antidiag(T) (Section 2.2) in the frequency unknowns:
// segment i owns K_i = 2^(level_i + 1) + 1 consecutive unknowns from
// koff[i].  Entries in this order: for every ordered pair i != j (i major),
// E's one entry (koff[i] + k^i_ij, koff[j] + k^j_ij); then for every segment
// the anti-diagonal of its T block, (koff[i] + r, koff[i] + K_i - 1 - r).
extern "C" cfie_status cfie_dirprec_w_pattern(int m, const int* level, const int* kpair,
                                              int capacity, int* koff, int* nnz, int* row,
                                              int* col) {
  if (m < 1 || !level || !kpair || !koff || !nnz) return CFIE_EINVAL;
  // every argument is checked before any output is written
  try {
    std::vector<int> ko((size_t)m + 1, 0);
    long long total = 0, count = (long long)m * (m - 1);
    for (int i = 0; i < m; ++i) {
      if (level[i] < 0 || level[i] > 20) return CFIE_EINVAL;
      const int K = (1 << (level[i] + 1)) + 1;
      total += K;
      count += K;
      if (total > (1LL << 30)) return CFIE_EINVAL;
      ko[i + 1] = int(total);
    }
    if (count > (1LL << 30)) return CFIE_EINVAL;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        if (i == j) continue;
        const int* kp = kpair + 2 * ((size_t)i * m + j);
        if (kp[0] < 0 || kp[0] >= ko[i + 1] - ko[i] || kp[1] < 0 || kp[1] >= ko[j + 1] - ko[j])
          return CFIE_EINVAL;
      }
    if ((row || col) && (!row || !col || capacity < count)) return CFIE_EINVAL;
    std::copy(ko.begin(), ko.end(), koff);
    *nnz = int(count);
    if (!row) return CFIE_OK;
    long long e = 0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        if (i == j) continue;
        const int* kp = kpair + 2 * ((size_t)i * m + j);
        row[e] = ko[i] + kp[0];
        col[e] = ko[j] + kp[1];
        ++e;
      }
    for (int i = 0; i < m; ++i) {
      const int K = ko[i + 1] - ko[i];
      for (int r = 0; r < K; ++r, ++e) {
        row[e] = ko[i] + r;
        col[e] = ko[i] + K - 1 - r;
      }
    }
    return CFIE_OK;
  } catch (...) {
    return CFIE_ENOMEM;
  }
}
