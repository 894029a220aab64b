// Directional preconditioner of Section 2 on the GPU: setup (E, W~^-1) and the
// apply of eq. (eapp), over every right-hand side at once.
//
// The operator is the sound-soft CFIE matrix M of eq. 1 on a curve sampled at
// n = 4^q p points equispaced in arclength.  Section 2.1 approximates
// M ~ B + U E U^t (segments P_i, flat diagonal blocks B, partial Fourier
// factors U_i, one coefficient e_ij per off-diagonal block), and Section 2.2
// applies the inverse of that approximation (eq. eapp):
//
//     b = B^-1 f,  p0 = -U^t b,  t = T~ p0,  r = W~^-1 t,
//     p = T~ r - t,  q = b - B^-1 U p,                       P f = q
//
// with T = (U^t B^-1 U)^-1 per segment, T~ its thresholded form and
// W~ = E + antidiag(T).  On arclength nodes B, U, T and T~ depend on the
// segment's level only; the host builds them (cfie_dirprec_level,
// cfie_dirprec_threshold), the GPU builds E and W~^-1:
//
//  * E: e_ij is the least-squares constant of the rank-1 form on the block
//    itself, the mean of M(x, y) / (U_i(x, k^i) U_j(y, k^j)) over x in P_i,
//    y in P_j (the quantity eq. entry approximates from Chebyshev samples):
//    one CTA per ordered pair of segments over the operator's own entries,
//    FP64 for the FP64 precision, FP32 for the refined ones (the fast
//    matvec's entries: one pass at FP32 speed instead of an FP64 matvec).
//  * W~^-1: W~ = A_T + E with A_T the block anti-diagonal of the T_i, one
//    entry per row, so every row a of W~ owns the unknown pi(a) (its
//    anti-diagonal partner) with coefficient D_a, and E has one entry per
//    ordered pair of segments in its rows R and columns C.  Rows outside R
//    give their unknown at once; the unknowns in C whose own row lies in R
//    (the set S, about half of W~'s size) couple through the |S| x |S|
//    system D_S + E_SS, inverted densely on the GPU (FP64 Gauss-Jordan with
//    row pivoting) and applied as a complex64 GEMM; the remaining rows of R
//    then give their unknowns from the known ones.  This is W~'s sparse
//    structure used exactly: the result equals W~^-1 t.
//
// The apply runs in complex64 (FP32 arithmetic): one batched GEMM kernel for
// the per-segment products B^-1, U^t, U, T~ (each segment's slice of every
// right-hand side against its level's matrix), four small kernels for W~.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <climits>

#include "hankel64.cuh"
#include "internal.h"
#include "pair32.cuh"

namespace {

// ---------------------------------------------------------------------------
// E: e_ij = mean over the block of M(x, y) exp(-i k^i rho_i(x)) exp(-i k^j rho_j(y))
// ---------------------------------------------------------------------------
constexpr int EMAX = 1024;   // largest segment (cfie_dirprec_level's bound)

// Entries in FP64 (the FP64 matvec's pair function), or for the refined
// precisions the operator's FP32 entries (near band from its table, the rest
// from the FP32 pair function, as the stored matrix is assembled), summed per
// thread in the entries' precision and across the block in FP64.
struct e32_args {
  omega32 W;
  geo32 g;
  const float* w32;
  const float2* band;
  int b;
};

template <bool F32>
__global__ void __launch_bounds__(256)
k_dirprec_e(int n, int m, double omega, double eta, double ds, geom_dev g,
            const double* __restrict__ wtab, e32_args f, const int* __restrict__ first,
            const int* __restrict__ count, const int* __restrict__ level,
            const int* __restrict__ kpair, double2* __restrict__ e) {
  __shared__ double2 phr[EMAX], phc[EMAX];
  __shared__ double2 red[8];
  const int i = blockIdx.x / m, j = blockIdx.x % m;
  if (i == j) {
    if (threadIdx.x == 0) e[blockIdx.x] = make_double2(0.0, 0.0);
    return;
  }
  const int fi = first[i], ci = count[i], fj = first[j], cj = count[j];
  const int* kp = kpair + 2 * ((size_t)i * m + j);
  // wave numbers k_m = -omega + m omega / 2^l on the 2^(l+1) + 1 points of each level
  const double ki = -omega + kp[0] * omega / (double)(1 << level[i]);
  const double kj = -omega + kp[1] * omega / (double)(1 << level[j]);
  for (int x = threadIdx.x; x < ci; x += blockDim.x) {
    double s, c;
    sincos(-ki * (x - 0.5 * (ci - 1)) * ds, &s, &c);
    phr[x] = make_double2(c, s);
  }
  for (int y = threadIdx.x; y < cj; y += blockDim.x) {
    double s, c;
    sincos(-kj * (y - 0.5 * (cj - 1)) * ds, &s, &c);
    phc[y] = make_double2(c, s);
  }
  __syncthreads();
  const double h = 2.0 * CFIE_PI / n;
  double ar = 0.0, ai = 0.0;
  float sr32 = 0.f, si32 = 0.f;
  const long long tot = (long long)ci * cj;
  for (long long idx = threadIdx.x; idx < tot; idx += blockDim.x) {
    const int x = (int)(idx / cj), y = (int)(idx % cj);
    const int gi = fi + x, gj = fj + y;
    int d = gi - gj;
    if (d < 0) d += n;
    const double2 u = phr[x], v = phc[y];
    const double pr = u.x * v.x - u.y * v.y, pim = u.x * v.y + u.y * v.x;
    if constexpr (F32) {
      float2 a, unused;
      const int dd = d <= f.b ? d : (d >= n - f.b ? d - n : INT_MAX);
      if (dd != INT_MAX)
        a = f.band[(size_t)gi * (2 * f.b + 1) + dd + f.b];
      else
        pair_entries_fp32<0>(f.W, f.g.xh[gi], f.g.xl[gi], f.g.yh[gi], f.g.yl[gi], f.g.nx[gi],
                             f.g.ny[gi], f.g.sp[gi], f.g.xh[gj], f.g.xl[gj], f.g.yh[gj],
                             f.g.yl[gj], f.g.nx[gj], f.g.ny[gj], f.g.sp[gj], f.w32[d], a, unused);
      const float p1 = (float)pr, p2 = (float)pim;
      sr32 = fmaf(a.x, p1, fmaf(-a.y, p2, sr32));
      si32 = fmaf(a.x, p2, fmaf(a.y, p1, si32));
    } else {
      double2 a, unused;
      pair_entries_fp64<0>(g.x[gi] - g.x[gj], g.y[gi] - g.y[gj], omega, eta, h, wtab[d], g.nx[gj],
                           g.ny[gj], g.sp[gj], g.nx[gi], g.ny[gi], g.sp[gi], a, unused);
      ar += a.x * pr - a.y * pim;
      ai += a.x * pim + a.y * pr;
    }
  }
  if constexpr (F32) {
    ar = sr32;
    ai = si32;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, o);
    ai += __shfl_xor_sync(0xffffffffu, ai, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(ar, ai);
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0.0, si = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sr += red[w].x;
      si += red[w].y;
    }
    const double inv = 1.0 / ((double)ci * cj);
    e[blockIdx.x] = make_double2(sr * inv, si * inv);
  }
}

// ---------------------------------------------------------------------------
// Dense inverse by Gauss-Jordan elimination with row pivoting (FP64, in place)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Step k, one CTA: pivot row p = argmax_{i >= k} |A_ik| (lowest index on
// ties), rows k and p swapped, row k divided by the pivot with A_kk replaced
// by its inverse; column k saved (row k as zero) and cleared for the update,
// and the rows whose saved entry is non-zero listed (rows[0 .. *cnt)): the
// coupled block of W~ is sparse and stays so under elimination (a few percent
// of the rows take part in a step), so the update touches only those rows.
__global__ void __launch_bounds__(1024)
k_gj_pivot(int N, int k, double2* __restrict__ A, int* __restrict__ piv,
           double2* __restrict__ col, double2* __restrict__ row, int* __restrict__ rows,
           int* __restrict__ cnt, int* __restrict__ err) {
  __shared__ double bv[32];
  __shared__ int bi[32];
  __shared__ int P, C;
  double best = -1.0;
  int arg = k;
  for (int i = k + threadIdx.x; i < N; i += blockDim.x) {
    const double2 v = A[(size_t)i * N + k];
    const double a = v.x * v.x + v.y * v.y;
    if (a > best) {
      best = a;
      arg = i;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
    if (ob > best || (ob == best && oa < arg)) {
      best = ob;
      arg = oa;
    }
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    bv[w] = best;
    bi[w] = arg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < nw; ++q)
      if (bv[q] > bv[0] || (bv[q] == bv[0] && bi[q] < bi[0])) {
        bv[0] = bv[q];
        bi[0] = bi[q];
      }
    P = bi[0];
    C = 0;
    piv[k] = bi[0];
    if (!(bv[0] > 0.0)) atomicExch(err, 1);   // singular
  }
  __syncthreads();
  const int p = P;
  if (p != k)
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      const double2 t = A[(size_t)k * N + j];
      A[(size_t)k * N + j] = A[(size_t)p * N + j];
      A[(size_t)p * N + j] = t;
    }
  __syncthreads();
  const double2 d = A[(size_t)k * N + k];
  const double dd = d.x * d.x + d.y * d.y;
  const double2 inv = dd > 0.0 ? make_double2(d.x / dd, -d.y / dd) : make_double2(0.0, 0.0);
  __syncthreads();
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const double2 v = j == k ? inv : cmul(A[(size_t)k * N + j], inv);
    A[(size_t)k * N + j] = v;
    row[j] = v;
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    if (i == k) {
      col[i] = make_double2(0.0, 0.0);
    } else {
      const double2 v = A[(size_t)i * N + k];
      col[i] = v;
      A[(size_t)i * N + k] = make_double2(0.0, 0.0);
      if (v.x != 0.0 || v.y != 0.0) rows[atomicAdd(&C, 1)] = i;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *cnt = C;
}

// A_ij -= col_i row_j for the listed rows i and every j (column k starts at 0,
// so it receives -A_ik / pivot); rows not listed have col_i = 0
__global__ void __launch_bounds__(256)
k_gj_update(int N, double2* __restrict__ A, const double2* __restrict__ col,
            const double2* __restrict__ row, const int* __restrict__ rows,
            const int* __restrict__ cnt) {
  const int nr = *cnt;
  for (int q = blockIdx.y; q < nr; q += gridDim.y) {
    const int i = rows[q];
    const double2 c = col[i];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
      const double2 r = row[j];
      double2 a = A[(size_t)i * N + j];
      a.x -= c.x * r.x - c.y * r.y;
      a.y -= c.x * r.y + c.y * r.x;
      A[(size_t)i * N + j] = a;
    }
  }
}

// the row interchanges undone as column interchanges (column c of the inverse
// is column perm[c] of A), stored as complex64
__global__ void k_gj_finish(int N, const double2* __restrict__ A, const int* __restrict__ perm,
                            float2* __restrict__ Z) {
  const int i = blockIdx.y;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const double2 v = A[(size_t)i * N + perm[c]];
    Z[(size_t)i * N + c] = make_float2((float)v.x, (float)v.y);
  }
}

// ---------------------------------------------------------------------------
// Apply: per-segment GEMMs  Y[y_off + r] = alpha sum_k A[r][k] X[x_off + k] + beta Z[y_off + r]
// ---------------------------------------------------------------------------
struct seg_desc {
  long long a_off;    // first element of the segment's level matrix in `mats`
  int rows, cols;     // matrix shape (row-major, leading dimension cols)
  int x_off, y_off;   // first row of the segment's slice in X and in Y / Z
};
constexpr int GBM = 64, GBN = 16, GBK = 32;

__global__ void __launch_bounds__(256)
k_seg_gemm(const int2* __restrict__ items, const seg_desc* __restrict__ descs,
           const float2* __restrict__ mats, const float2* __restrict__ X, int ldx,
           float2* __restrict__ Y, int ldy, const float2* __restrict__ Zb, float alpha,
           float beta, int nrhs) {
  __shared__ float2 As[GBM][GBK + 1];
  __shared__ float2 Xs[GBN][GBK + 1];
  const int2 it = items[blockIdx.x];          // (descriptor, first row)
  const seg_desc sd = descs[it.x];
  const int r0 = it.y, c0 = blockIdx.y * GBN;
  const int tid = threadIdx.x, col = tid & 15, rg = tid >> 4;
  const float2* A = mats + sd.a_off;
  float2 acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < sd.cols; k0 += GBK) {
    for (int e = tid; e < GBM * GBK; e += 256) {
      const int r = e / GBK, k = e % GBK;
      const int gr = r0 + r, gk = k0 + k;
      As[r][k] = (gr < sd.rows && gk < sd.cols) ? A[(size_t)gr * sd.cols + gk]
                                                 : make_float2(0.f, 0.f);
    }
    for (int e = tid; e < GBN * GBK; e += 256) {
      const int c = e / GBK, k = e % GBK;
      const int gc = c0 + c, gk = k0 + k;
      Xs[c][k] = (gc < nrhs && gk < sd.cols) ? X[(size_t)gc * ldx + sd.x_off + gk]
                                             : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GBK; ++k) {
      const float2 xv = Xs[col][k];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 a = As[rg + 16 * q][k];
        acc[q].x = fmaf(a.x, xv.x, fmaf(-a.y, xv.y, acc[q].x));
        acc[q].y = fmaf(a.x, xv.y, fmaf(a.y, xv.x, acc[q].y));
      }
    }
    __syncthreads();
  }
  const int gc = c0 + col;
  if (gc >= nrhs) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = r0 + rg + 16 * q;
    if (r >= sd.rows) continue;
    const size_t o = (size_t)gc * ldy + sd.y_off + r;
    float2 v = make_float2(alpha * acc[q].x, alpha * acc[q].y);
    if (Zb) {
      const float2 z = Zb[o];
      v.x = fmaf(beta, z.x, v.x);
      v.y = fmaf(beta, z.y, v.y);
    }
    Y[o] = v;
  }
}

// W~ solve data (one buffer): D (Ktot float2), pi (Ktot), inR (Ktot), rowptr
// (Ktot + 1), ecol (nnz), eval (nnz float2), sb (nS: the unknowns of S),
// sidx (Ktot: position in S or -1), rest (nRest: rows of R whose unknown is
// outside S)
struct wsolve_dev {
  const float2* D;
  const int *pi, *inR, *rowptr, *ecol, *sb, *sidx, *rest;
  const float2* eval;
};

__device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
  const float d = b.x * b.x + b.y * b.y;
  return make_float2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// rows outside R: r_{pi(a)} = t_a / D_a
__global__ void k_w_free(int K, int nrhs, wsolve_dev w, const float2* __restrict__ t,
                         float2* __restrict__ r) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)K * nrhs) return;
  const int a = (int)(e % K);
  const size_t c = e / K;
  if (w.inR[a]) return;
  r[c * K + w.pi[a]] = cdiv(t[c * K + a], w.D[a]);
}

// right-hand side of the S system: t at the row of each S unknown, less the
// E terms on unknowns outside S (known from k_w_free)
__global__ void k_w_rhs(int K, int nS, int nrhs, wsolve_dev w, const float2* __restrict__ t,
                        const float2* __restrict__ r, float2* __restrict__ rhs) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nS * nrhs) return;
  const int s = (int)(e % nS);
  const size_t c = e / nS;
  const int a = w.pi[w.sb[s]];
  float2 acc = t[c * K + a];
  for (int q = w.rowptr[a]; q < w.rowptr[a + 1]; ++q) {
    const int b = w.ecol[q];
    if (w.sidx[b] >= 0) continue;
    const float2 v = w.eval[q], x = r[c * K + b];
    acc.x -= v.x * x.x - v.y * x.y;
    acc.y -= v.x * x.y + v.y * x.x;
  }
  rhs[c * nS + s] = acc;
}

__global__ void k_w_scatter(int K, int nS, int nrhs, wsolve_dev w, const float2* __restrict__ rs,
                            float2* __restrict__ r) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nS * nrhs) return;
  const int s = (int)(e % nS);
  const size_t c = e / nS;
  r[c * K + w.sb[s]] = rs[c * nS + s];
}

// rows of R whose unknown lies outside S: r_{pi(a)} = (t_a - sum_b E_ab r_b) / D_a
__global__ void k_w_rest(int K, int nRest, int nrhs, wsolve_dev w, const float2* __restrict__ t,
                         float2* __restrict__ r) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)nRest * nrhs) return;
  const int a = w.rest[e % nRest];
  const size_t c = e / nRest;
  float2 acc = t[c * K + a];
  for (int q = w.rowptr[a]; q < w.rowptr[a + 1]; ++q) {
    const float2 v = w.eval[q], x = r[c * K + w.ecol[q]];
    acc.x -= v.x * x.x - v.y * x.y;
    acc.y -= v.x * x.y + v.y * x.x;
  }
  r[c * K + w.pi[a]] = cdiv(acc, w.D[a]);
}

// A[pos[q]] = val[q] (positions distinct)
__global__ void k_scatter_c128(size_t nz, const int* __restrict__ pos,
                               const double2* __restrict__ val, double2* __restrict__ A) {
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nz) A[pos[q]] = val[q];
}

__global__ void k_c128_to_c64(size_t len, const double2* __restrict__ x, float2* __restrict__ y) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < len) y[e] = make_float2((float)x[e].x, (float)x[e].y);
}
__global__ void k_c64_to_c128(size_t len, const float2* __restrict__ x, double2* __restrict__ y) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < len) y[e] = make_double2(x[e].x, x[e].y);
}

unsigned nblk(size_t len, int t = 256) { return (unsigned)((len + t - 1) / t); }

// Level blocks depend only on (n, p, level, omega, eta, L, t_keep): kept for
// the process so that preconditioners of the same discretisation (new
// operators at every solve, other right-hand sides) skip their host setup.
struct level_blocks {
  std::vector<double> Binv, U, T, Tt;
};
std::mutex g_level_mu;
std::map<std::tuple<int, int, int, double, double, double, int>, level_blocks> g_levels;

// The curve's n arclength samples (positions) and perimeter, kept for the
// process per (curve, parameters, n): setups of the same discretisation
// (a new operator at every solve) reuse them.
std::mutex g_arc_mu;
std::map<std::tuple<int, std::vector<double>, int>, std::pair<std::vector<double>, double>> g_arc;

void arclength_nodes(cfie_curve kind, const double* params, int nparams, int n,
                     std::vector<double>& z, double& L) {
  CFIE_REQUIRE(nparams >= 0 && nparams <= 128 && (nparams == 0 || params),
               "invalid curve parameters");
  const auto key = std::make_tuple((int)kind, std::vector<double>(params, params + nparams), n);
  {
    std::lock_guard<std::mutex> lock(g_arc_mu);
    auto it = g_arc.find(key);
    if (it != g_arc.end()) {
      z = it->second.first;
      L = it->second.second;
      return;
    }
  }
  z.assign(2 * (size_t)n, 0.0);
  std::vector<double> dz(2 * (size_t)n), ddz(2 * (size_t)n);
  CFIE_REQUIRE(cfie_arclength_samples(kind, params, nparams, n, z.data(), dz.data(), ddz.data(),
                                      &L) == CFIE_OK,
               "invalid curve for the arclength samples");
  std::lock_guard<std::mutex> lock(g_arc_mu);
  if (g_arc.size() >= 16) g_arc.clear();
  g_arc[key] = std::make_pair(z, L);
}

level_blocks level_setup(int n, int p, int l, double omega, double eta, double L, int t_keep) {
  const auto key = std::make_tuple(n, p, l, omega, eta, L, t_keep);
  {
    std::lock_guard<std::mutex> lock(g_level_mu);
    auto it = g_levels.find(key);
    if (it != g_levels.end()) return it->second;
  }
  const int c = (1 << l) * p, K = (1 << (l + 1)) + 1;
  level_blocks b;
  b.Binv.resize(2 * (size_t)c * c);
  b.U.resize(2 * (size_t)c * K);
  b.T.resize(2 * (size_t)K * K);
  b.Tt.resize(2 * (size_t)K * K);
  CFIE_REQUIRE(cfie_dirprec_level(n, p, l, omega, eta, L, nullptr, b.Binv.data(), b.U.data(),
                                  b.T.data()) == CFIE_OK,
               "cfie_dirprec_level failed (singular block?)");
  CFIE_REQUIRE(cfie_dirprec_threshold(K, b.T.data(), t_keep * K, b.Tt.data()) == CFIE_OK,
               "cfie_dirprec_threshold failed");
  std::lock_guard<std::mutex> lock(g_level_mu);
  if (g_levels.size() >= 32) g_levels.clear();   // bounded: a few MB per entry
  g_levels[key] = b;
  return b;
}

// GEMM kinds, in descriptor order: m descriptors each
enum { G_BINV = 0, G_UT = 1, G_TT = 2, G_U = 3, G_Z = 4 };

struct wsolve_host {
  size_t o_D, o_pi, o_inR, o_rowptr, o_ecol, o_eval, o_sb, o_sidx, o_rest, bytes;
};

wsolve_dev wsolve_at(const cfie_dirprec* P, const wsolve_host& h) {
  const char* b = P->wsolve.as<char>();
  wsolve_dev w;
  w.D = reinterpret_cast<const float2*>(b + h.o_D);
  w.pi = reinterpret_cast<const int*>(b + h.o_pi);
  w.inR = reinterpret_cast<const int*>(b + h.o_inR);
  w.rowptr = reinterpret_cast<const int*>(b + h.o_rowptr);
  w.ecol = reinterpret_cast<const int*>(b + h.o_ecol);
  w.eval = reinterpret_cast<const float2*>(b + h.o_eval);
  w.sb = reinterpret_cast<const int*>(b + h.o_sb);
  w.sidx = reinterpret_cast<const int*>(b + h.o_sidx);
  w.rest = reinterpret_cast<const int*>(b + h.o_rest);
  return w;
}

wsolve_host wsolve_layout(int K, int nnz, int nS, int nRest) {
  wsolve_host h{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 255) & ~size_t(255);
    return at;
  };
  h.o_D = take(sizeof(float2) * K);
  h.o_pi = take(sizeof(int) * K);
  h.o_inR = take(sizeof(int) * K);
  h.o_rowptr = take(sizeof(int) * (K + 1));
  h.o_ecol = take(sizeof(int) * std::max(1, nnz));
  h.o_eval = take(sizeof(float2) * std::max(1, nnz));
  h.o_sb = take(sizeof(int) * std::max(1, nS));
  h.o_sidx = take(sizeof(int) * K);
  h.o_rest = take(sizeof(int) * std::max(1, nRest));
  h.bytes = o;
  return h;
}

void launch_gemm(cfie_dirprec* P, int kind, const float2* mats, const float2* X, int ldx,
                 float2* Y, int ldy, const float2* Zb, float alpha, float beta, int nrhs) {
  if (!P->item_cnt[kind]) return;
  const dim3 grid((unsigned)P->item_cnt[kind], (unsigned)((nrhs + GBN - 1) / GBN));
  k_seg_gemm<<<grid, 256, 0, P->ctx->stream>>>(P->items.as<int2>() + P->item_off[kind],
                                                P->descs.as<seg_desc>(), mats, X, ldx, Y, ldy,
                                                Zb, alpha, beta, nrhs);
  CFIE_CHECK_LAUNCH();
}

}  // namespace

// ---------------------------------------------------------------------------
// host: setup
// ---------------------------------------------------------------------------
void dirprec_build(cfie_dirprec* P, cfie_op* op, cfie_curve kind, const double* params,
                   int nparams, int q, int p, int m_leaf, int t_keep) {
  CFIE_REQUIRE(op->bc == CFIE_SOUND_SOFT, "the directional preconditioner is built for the sound-soft operator");
  CFIE_REQUIRE(q >= 1 && q <= 9 && p >= 1, "q must be in [1, 9] and p positive");
  CFIE_REQUIRE(m_leaf >= 1 && t_keep >= 1, "m_leaf and t_keep must be positive");
  long long nn = p;
  for (int i = 0; i < q; ++i) nn *= 4;
  CFIE_REQUIRE(nn == op->n, "the operator must have n = 4^q p nodes");
  const int n = op->n;
  cudaStream_t st = op->ctx->stream;
  P->ctx = op->ctx;
  P->n = n;
  P->q = q;
  P->p = p;
  P->omega = op->omega;
  P->eta = op->eta;

  // the node set: the operator's nodes must be the curve's arclength samples
  std::vector<double> z;
  double L = 0;
  arclength_nodes(kind, params, nparams, n, z, L);
  P->L = L;
  {
    std::vector<double> gx(n), gy(n);
    CFIE_CHECK_CUDA(cudaMemcpyAsync(gx.data(), op->g.x, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    CFIE_CHECK_CUDA(cudaMemcpyAsync(gy.data(), op->g.y, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    CFIE_CHECK_CUDA(cudaStreamSynchronize(st));
    double dev = 0, scale = 0;
    for (int i = 0; i < n; ++i) {
      dev = std::max(dev, std::hypot(gx[i] - z[2 * i], gy[i] - z[2 * i + 1]));
      scale = std::max(scale, std::hypot(z[2 * i], z[2 * i + 1]));
    }
    CFIE_REQUIRE(dev <= 1e-9 * std::max(1.0, scale),
                 "the operator's nodes are not the curve's arclength samples (cfie_arclength_samples)");
  }

  // segments and wave-number pairs (Section 2.1)
  int m = 0;
  CFIE_REQUIRE(cfie_dirprec_plan(kind, params, nparams, q, p, op->omega, m_leaf, 0, &m, nullptr,
                                 nullptr, nullptr) == CFIE_OK,
               "cfie_dirprec_plan failed");
  P->m = m;
  P->first.assign(m, 0);
  P->level.assign(m, 0);
  std::vector<int> kpair(2 * (size_t)m * m);
  CFIE_REQUIRE(cfie_dirprec_plan(kind, params, nparams, q, p, op->omega, m_leaf, m, &m,
                                 P->first.data(), P->level.data(), kpair.data()) == CFIE_OK,
               "cfie_dirprec_plan failed");
  P->count.resize(m);
  P->koff.assign(m + 1, 0);
  for (int i = 0; i < m; ++i) {
    P->count[i] = (1 << P->level[i]) * p;
    CFIE_REQUIRE(P->count[i] <= EMAX, "a segment exceeds 1024 nodes");
    P->koff[i + 1] = P->koff[i] + (1 << (P->level[i] + 1)) + 1;
  }
  const int Ktot = P->koff[m];
  P->Ktot = Ktot;

  // level blocks (Section 2.2): B_l^-1, U_l, T_l, T~_l on the host, FP64
  std::vector<int> lv(P->level);
  std::sort(lv.begin(), lv.end());
  lv.erase(std::unique(lv.begin(), lv.end()), lv.end());
  struct lvl { int l, c, K; long long oBinv, oUt, oTt, oU; std::vector<double> T; };
  std::vector<lvl> lvls;
  long long mat_elems = 0;
  for (int l : lv) {
    lvl b;
    b.l = l;
    b.c = (1 << l) * p;
    b.K = (1 << (l + 1)) + 1;
    b.oBinv = mat_elems;
    mat_elems += (long long)b.c * b.c;
    b.oUt = mat_elems;
    mat_elems += (long long)b.K * b.c;
    b.oTt = mat_elems;
    mat_elems += (long long)b.K * b.K;
    b.oU = mat_elems;
    mat_elems += (long long)b.c * b.K;
    lvls.push_back(std::move(b));
  }
  std::vector<float2> mats_h((size_t)mat_elems);
  for (lvl& b : lvls) {
    level_blocks lb = level_setup(n, p, b.l, op->omega, op->eta, L, t_keep);
    const std::vector<double>& Binv = lb.Binv;
    const std::vector<double>& U = lb.U;
    const std::vector<double>& Tt = lb.Tt;
    std::vector<double>& T = lb.T;
    for (long long e = 0; e < (long long)b.c * b.c; ++e)
      mats_h[b.oBinv + e] = make_float2((float)Binv[2 * e], (float)Binv[2 * e + 1]);
    for (int x = 0; x < b.c; ++x)
      for (int k = 0; k < b.K; ++k) {
        const size_t s = (size_t)x * b.K + k;
        const float2 v = make_float2((float)U[2 * s], (float)U[2 * s + 1]);
        mats_h[b.oU + s] = v;
        mats_h[b.oUt + (size_t)k * b.c + x] = v;
      }
    for (long long e = 0; e < (long long)b.K * b.K; ++e)
      mats_h[b.oTt + e] = make_float2((float)Tt[2 * e], (float)Tt[2 * e + 1]);
    b.T = std::move(T);
  }
  auto lvl_of = [&](int l) -> const lvl& {
    for (const lvl& b : lvls)
      if (b.l == l) return b;
    throw cfie_error(CFIE_EINVAL, "level table");
  };

  // E on the GPU
  {
    dbuf tab;
    tab.reserve(sizeof(int) * (3 * (size_t)m + 2 * (size_t)m * m) + 64);
    int* t = tab.as<int>();
    CFIE_CHECK_CUDA(cudaMemcpyAsync(t, P->first.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st));
    CFIE_CHECK_CUDA(cudaMemcpyAsync(t + m, P->count.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st));
    CFIE_CHECK_CUDA(cudaMemcpyAsync(t + 2 * m, P->level.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st));
    CFIE_CHECK_CUDA(cudaMemcpyAsync(t + 3 * m, kpair.data(), sizeof(int) * 2 * (size_t)m * m,
                                    cudaMemcpyHostToDevice, st));
    dbuf eb;
    eb.reserve(sizeof(double2) * (size_t)m * m);
    e32_args f{};
    const bool f32 = op->prec == CFIE_FP32_REFINED && op->geo32.p && op->band_b >= 0;
    if (f32) {
      float* base = op->geo32.as<float>();
      f.W = omega32{(float)op->omega, (float)op->eta, (float)op->h};
      f.g = geo32_at(base, n);
      f.w32 = base + 7 * n;
      f.band = op->band.as<float2>();
      f.b = op->band_b;
      k_dirprec_e<true><<<(unsigned)m * m, 256, 0, st>>>(n, m, op->omega, op->eta, L / n, op->g,
                                                          op->wtab.as<double>(), f, t, t + m,
                                                          t + 2 * m, t + 3 * m, eb.as<double2>());
    } else {
      k_dirprec_e<false><<<(unsigned)m * m, 256, 0, st>>>(n, m, op->omega, op->eta, L / n, op->g,
                                                           op->wtab.as<double>(), f, t, t + m,
                                                           t + 2 * m, t + 3 * m, eb.as<double2>());
    }
    CFIE_CHECK_LAUNCH();
    P->e.assign(2 * (size_t)m * m, 0.0);
    CFIE_CHECK_CUDA(cudaMemcpyAsync(P->e.data(), eb.p, sizeof(double2) * (size_t)m * m,
                                    cudaMemcpyDeviceToHost, st));
    CFIE_CHECK_CUDA(cudaStreamSynchronize(st));
  }

  // W~ = A_T + E: the anti-diagonal partner pi(a) and coefficient D_a of every row
  std::vector<int> pi(Ktot), inR(Ktot, 0), inC(Ktot, 0);
  std::vector<double> D(2 * (size_t)Ktot);
  for (int i = 0; i < m; ++i) {
    const lvl& b = lvl_of(P->level[i]);
    for (int r = 0; r < b.K; ++r) {
      const int a = P->koff[i] + r;
      pi[a] = P->koff[i] + b.K - 1 - r;
      const size_t s = (size_t)r * b.K + (b.K - 1 - r);
      D[2 * a] = b.T[2 * s];
      D[2 * a + 1] = b.T[2 * s + 1];
      CFIE_REQUIRE(std::hypot(D[2 * a], D[2 * a + 1]) > 0, "zero anti-diagonal entry of T");
    }
  }
  // E's entries by row (CSR), one per ordered pair of segments
  std::vector<std::vector<std::pair<int, int>>> rows(Ktot);   // (column, pair index)
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      if (i == j) continue;
      const int* kp = kpair.data() + 2 * ((size_t)i * m + j);
      const int a = P->koff[i] + kp[0], bcol = P->koff[j] + kp[1];
      rows[a].push_back({bcol, i * m + j});
      inR[a] = 1;
      inC[bcol] = 1;
    }
  std::vector<int> rowptr(Ktot + 1, 0), ecol;
  std::vector<float2> evalf;
  std::vector<double> evald;
  for (int a = 0; a < Ktot; ++a) {
    for (auto& pr : rows[a]) {
      ecol.push_back(pr.first);
      const double er = P->e[2 * (size_t)pr.second], ei = P->e[2 * (size_t)pr.second + 1];
      evalf.push_back(make_float2((float)er, (float)ei));
      evald.push_back(er);
      evald.push_back(ei);
    }
    rowptr[a + 1] = (int)ecol.size();
  }
  // S: unknowns in C whose own row is in R; the rest of R
  std::vector<int> sb, sidx(Ktot, -1), rest;
  for (int b = 0; b < Ktot; ++b)
    if (inC[b] && inR[pi[b]]) {
      sidx[b] = (int)sb.size();
      sb.push_back(b);
    }
  for (int a = 0; a < Ktot; ++a)
    if (inR[a] && sidx[pi[a]] < 0) rest.push_back(a);
  const int nS = (int)sb.size(), nRest = (int)rest.size();
  P->nS = nS;
  P->nRest = nRest;

  // M_S = D_S + E_SS (row of unknown b is pi(b)), inverted on the GPU in FP64
  if (nS > 0) {
    // its non-zeros: the diagonal D and E's entries on S x S (one per segment
    // pair at most, so no two share a position), scattered into a zeroed matrix
    std::vector<int> mpos;
    std::vector<double2> mval;
    for (int s = 0; s < nS; ++s) {
      const int a = pi[sb[s]];
      mpos.push_back(s * nS + s);
      mval.push_back(make_double2(D[2 * a], D[2 * a + 1]));
      for (int qq = rowptr[a]; qq < rowptr[a + 1]; ++qq) {
        const int t2 = sidx[ecol[qq]];
        if (t2 < 0) continue;
        mpos.push_back(s * nS + t2);
        mval.push_back(make_double2(evald[2 * qq], evald[2 * qq + 1]));
      }
    }
    dbuf A, aux, sp;
    A.reserve(sizeof(double2) * (size_t)nS * nS);
    aux.reserve(sizeof(double2) * 2 * (size_t)nS + sizeof(int) * (2 * (size_t)nS + 8) + 64);
    double2* col = aux.as<double2>();
    double2* row = col + nS;
    int* piv = reinterpret_cast<int*>(row + nS);
    int* rows = piv + nS;
    int* cnt = rows + nS;
    int* err = cnt + 1;
    const size_t nz = mpos.size();
    sp.reserve((sizeof(double2) + sizeof(int)) * nz + 64);
    double2* spv = sp.as<double2>();
    int* spp = reinterpret_cast<int*>(spv + nz);
    CFIE_CHECK_CUDA(cudaMemcpyAsync(spv, mval.data(), sizeof(double2) * nz, cudaMemcpyHostToDevice, st));
    CFIE_CHECK_CUDA(cudaMemcpyAsync(spp, mpos.data(), sizeof(int) * nz, cudaMemcpyHostToDevice, st));
    CFIE_CHECK_CUDA(cudaMemsetAsync(A.p, 0, sizeof(double2) * (size_t)nS * nS, st));
    k_scatter_c128<<<nblk(nz), 256, 0, st>>>(nz, spp, spv, A.as<double2>());
    CFIE_CHECK_LAUNCH();
    CFIE_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    const unsigned gx = (unsigned)std::max(1, std::min(8, (nS + 255) / 256));
    const unsigned gy = (unsigned)std::min(nS, 256);
    for (int k = 0; k < nS; ++k) {
      k_gj_pivot<<<1, 1024, 0, st>>>(nS, k, A.as<double2>(), piv, col, row, rows, cnt, err);
      CFIE_CHECK_LAUNCH();
      k_gj_update<<<dim3(gx, gy), 256, 0, st>>>(nS, A.as<double2>(), col, row, rows, cnt);
      CFIE_CHECK_LAUNCH();
    }
    int bad = 0;
    std::vector<int> pv(nS), perm(nS);
    CFIE_CHECK_CUDA(cudaMemcpyAsync(&bad, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CFIE_CHECK_CUDA(cudaMemcpyAsync(pv.data(), piv, sizeof(int) * nS, cudaMemcpyDeviceToHost, st));
    CFIE_CHECK_CUDA(cudaStreamSynchronize(st));
    CFIE_REQUIRE(!bad, "the coupled block of W~ is singular");
    // column interchanges in reverse order of the row interchanges
    for (int c = 0; c < nS; ++c) perm[c] = c;
    for (int k = nS - 1; k >= 0; --k) std::swap(perm[k], perm[pv[k]]);
    CFIE_CHECK_CUDA(cudaMemcpyAsync(piv, perm.data(), sizeof(int) * nS, cudaMemcpyHostToDevice, st));
    P->Z.reserve(sizeof(float2) * (size_t)nS * nS);
    k_gj_finish<<<dim3(gx, (unsigned)nS), 256, 0, st>>>(nS, A.as<double2>(), piv, P->Z.as<float2>());
    CFIE_CHECK_LAUNCH();
    CFIE_CHECK_CUDA(cudaStreamSynchronize(st));   // perm dies on return
  }

  // W~ solve tables
  const int nnz = (int)ecol.size();
  P->nnz = nnz;
  const wsolve_host wl = wsolve_layout(Ktot, nnz, nS, nRest);
  std::vector<char> wh(wl.bytes, 0);
  std::vector<float2> Df(Ktot);
  for (int a = 0; a < Ktot; ++a) Df[a] = make_float2((float)D[2 * a], (float)D[2 * a + 1]);
  std::memcpy(wh.data() + wl.o_D, Df.data(), sizeof(float2) * Ktot);
  std::memcpy(wh.data() + wl.o_pi, pi.data(), sizeof(int) * Ktot);
  std::memcpy(wh.data() + wl.o_inR, inR.data(), sizeof(int) * Ktot);
  std::memcpy(wh.data() + wl.o_rowptr, rowptr.data(), sizeof(int) * (Ktot + 1));
  if (nnz) std::memcpy(wh.data() + wl.o_ecol, ecol.data(), sizeof(int) * nnz);
  if (nnz) std::memcpy(wh.data() + wl.o_eval, evalf.data(), sizeof(float2) * nnz);
  if (nS) std::memcpy(wh.data() + wl.o_sb, sb.data(), sizeof(int) * nS);
  std::memcpy(wh.data() + wl.o_sidx, sidx.data(), sizeof(int) * Ktot);
  if (nRest) std::memcpy(wh.data() + wl.o_rest, rest.data(), sizeof(int) * nRest);
  P->wsolve.reserve(wl.bytes);
  CFIE_CHECK_CUDA(cudaMemcpyAsync(P->wsolve.p, wh.data(), wl.bytes, cudaMemcpyHostToDevice, st));

  // GEMM descriptors: per kind, one per segment (B^-1, U^t, T~, U), then Z
  std::vector<seg_desc> descs;
  std::vector<int2> items;
  for (int kind = 0; kind < 5; ++kind) {
    P->item_off[kind] = (int)items.size();
    const int nd = kind == G_Z ? (nS > 0 ? 1 : 0) : m;
    for (int i = 0; i < nd; ++i) {
      seg_desc d{};
      if (kind == G_Z) {
        d.a_off = 0;
        d.rows = d.cols = nS;
        d.x_off = d.y_off = 0;
      } else {
        const lvl& b = lvl_of(P->level[i]);
        const int c = b.c, K = b.K, f = P->first[i], ko = P->koff[i];
        switch (kind) {
          case G_BINV: d = seg_desc{b.oBinv, c, c, f, f}; break;
          case G_UT: d = seg_desc{b.oUt, K, c, f, ko}; break;
          case G_TT: d = seg_desc{b.oTt, K, K, ko, ko}; break;
          default: d = seg_desc{b.oU, c, K, ko, f}; break;
        }
      }
      const int di = (int)descs.size();
      descs.push_back(d);
      for (int r0 = 0; r0 < d.rows; r0 += GBM) items.push_back(make_int2(di, r0));
    }
    P->item_cnt[kind] = (int)items.size() - P->item_off[kind];
  }
  P->mats.reserve(sizeof(float2) * (size_t)mat_elems);
  CFIE_CHECK_CUDA(cudaMemcpyAsync(P->mats.p, mats_h.data(), sizeof(float2) * (size_t)mat_elems,
                                  cudaMemcpyHostToDevice, st));
  P->descs.reserve(sizeof(seg_desc) * descs.size());
  CFIE_CHECK_CUDA(cudaMemcpyAsync(P->descs.p, descs.data(), sizeof(seg_desc) * descs.size(),
                                  cudaMemcpyHostToDevice, st));
  P->items.reserve(sizeof(int2) * items.size());
  CFIE_CHECK_CUDA(cudaMemcpyAsync(P->items.p, items.data(), sizeof(int2) * items.size(),
                                  cudaMemcpyHostToDevice, st));
  CFIE_CHECK_CUDA(cudaStreamSynchronize(st));   // host tables die on return
}

// ---------------------------------------------------------------------------
// host: apply y = P x for nrhs right-hand sides (complex128 in and out)
// ---------------------------------------------------------------------------
void dirprec_apply(cfie_dirprec* P, const double2* x, double2* y, int nrhs) {
  const int n = P->n, K = P->Ktot, nS = P->nS;
  cudaStream_t st = P->ctx->stream;
  const size_t vn = (size_t)n * nrhs, vk = (size_t)K * nrhs, vs = (size_t)std::max(1, nS) * nrhs;
  // work: f, b, u, q (n each); p0, t, r, p (K each); rhs_S, r_S
  const size_t need = sizeof(float2) * (4 * vn + 4 * vk + 2 * vs);
  P->work.reserve(need);
  float2* f = P->work.as<float2>();
  float2* b = f + vn;
  float2* u = b + vn;
  float2* qv = u + vn;
  float2* p0 = qv + vn;
  float2* t = p0 + vk;
  float2* r = t + vk;
  float2* pp = r + vk;
  float2* rs_in = pp + vk;
  float2* rs_out = rs_in + vs;
  const float2* mats = P->mats.as<float2>();
  k_c128_to_c64<<<nblk(vn), 256, 0, st>>>(vn, x, f);
  CFIE_CHECK_LAUNCH();
  launch_gemm(P, G_BINV, mats, f, n, b, n, nullptr, 1.f, 0.f, nrhs);        // b = B^-1 f
  launch_gemm(P, G_UT, mats, b, n, p0, K, nullptr, -1.f, 0.f, nrhs);        // p0 = -U^t b
  launch_gemm(P, G_TT, mats, p0, K, t, K, nullptr, 1.f, 0.f, nrhs);         // t = T~ p0
  // r = W~^-1 t
  const wsolve_dev w = wsolve_at(P, wsolve_layout(K, P->nnz, nS, P->nRest));
  k_w_free<<<nblk(vk), 256, 0, st>>>(K, nrhs, w, t, r);
  CFIE_CHECK_LAUNCH();
  if (nS > 0) {
    k_w_rhs<<<nblk((size_t)nS * nrhs), 256, 0, st>>>(K, nS, nrhs, w, t, r, rs_in);
    CFIE_CHECK_LAUNCH();
    launch_gemm(P, G_Z, P->Z.as<float2>(), rs_in, nS, rs_out, nS, nullptr, 1.f, 0.f, nrhs);
    k_w_scatter<<<nblk((size_t)nS * nrhs), 256, 0, st>>>(K, nS, nrhs, w, rs_out, r);
    CFIE_CHECK_LAUNCH();
  }
  if (P->nRest > 0) {
    k_w_rest<<<nblk((size_t)P->nRest * nrhs), 256, 0, st>>>(K, P->nRest, nrhs, w, t, r);
    CFIE_CHECK_LAUNCH();
  }
  launch_gemm(P, G_TT, mats, r, K, pp, K, t, 1.f, -1.f, nrhs);              // p = T~ r - t
  launch_gemm(P, G_U, mats, pp, K, u, n, nullptr, 1.f, 0.f, nrhs);          // u = U p
  launch_gemm(P, G_BINV, mats, u, n, qv, n, b, -1.f, 1.f, nrhs);            // q = b - B^-1 u
  k_c64_to_c128<<<nblk(vn), 256, 0, st>>>(vn, qv, y);
  CFIE_CHECK_LAUNCH();
}

int dirprec_n(const cfie_dirprec* P) { return P->n; }

// e_ij of the m segments (m x m complex128 interleaved) to e unless NULL; returns m
int dirprec_segments(const cfie_dirprec* P, double* e) {
  if (e) std::memcpy(e, P->e.data(), sizeof(double) * P->e.size());
  return P->m;
}
