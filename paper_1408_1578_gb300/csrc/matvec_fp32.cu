// FP32 fused matrix-free Nystrom matvec: H0^(1), H1^(1)(omega |x - y|) evaluated on
// the fly in FP32, Kress log-split correction applied per pair, FP32 sums.
//
// Operators: paper Section 1 (eq. 1 sound soft, eq. 2 sound hard); the per-pair
// entry formulas are those of the FP64 kernel (hankel64.cuh), evaluated here in
// FP32 with two safeguards:
//
//  * Phase.  omega r reaches ~6e3 on the largest workloads, where one FP32
//    rounding of r is a ~4e-4 rad phase error.  Coordinates are stored
//    times omega as hi + lo FP32 pairs, the hi parts on a common grid on
//    which their differences and the sum of two squared differences are
//    exact, so the node distance is x = omega r itself; x^2 and x are
//    carried as two-float numbers (error-free transformations built from
//    fmaf), and chi = x - pi/4 is reduced modulo 2 pi with a three-part
//    Cody-Waite constant whose first part has 10 significant bits (k * C1
//    exact for x < 1e5).  The phase error grows with the scaled coordinates
//    (lo parts and their cross terms in FP32): ~2^(e - 33) rad for
//    omega |z| < 2^e, 6.5e-7 rad at most on the kite at omega = 2048 (e = 12),
//    1.3e-6 at e = 13; below the bf16 hi + lo split of the tensor-core sums.
//  * Small arguments.  Hankel's asymptotic expansion (A&S 9.2.5, 9.2.9, 9.2.10;
//    three terms of P and of Q, truncation error < 4.1e-8 for x >= 16) is used for
//    every pair with omega r >= 16.  Pairs closer than that form a band
//    |i - j| <= b around the diagonal (b found by an O(n^2) scan at set-up);
//    their entries are evaluated once in FP64 and stored as complex64.
//
// Layout: a CTA owns TI = 128 targets and a range of source tiles (TJ = 32).
// Per tile, warp w evaluates the entries of rows w, w+8, ... (lane = source)
// into shared memory, source-major; then the tile is contracted with the staged
// right-hand sides, each thread accumulating 4 targets x R/8 right-hand sides in
// registers (complex multiply-add on the FP32 pipe).  Source ranges are split
// across CTAs to fill the GPU; partial sums (complex64) are added in FP64 in a
// fixed order by the reduction kernel.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "hankel64.cuh"
#include "internal.h"
#include "pair32.cuh"

namespace {

constexpr int TI = 128;
constexpr int TJ = 32;
constexpr int NT = 256;
struct pair_params : omega32 {
  int n, b, splits, tiles_per_split, nrhs;
  geo32 g;
  const float* w32;
  const float2* band;    // soft: A ; hard: S
  const float2* band2;   // hard: D'
  const float2* xin;     // [k][j] complex64 (hard: x)
  const float2* uin;     // hard: (1/s) Dt x
  float2* part;          // [o][split][k][i]
};

__device__ __forceinline__ float2 cmul_add(float2 acc, float2 a, float2 x) {
  acc.x = fmaf(a.x, x.x, acc.x);
  acc.x = fmaf(-a.y, x.y, acc.x);
  acc.y = fmaf(a.x, x.y, acc.y);
  acc.y = fmaf(a.y, x.x, acc.y);
  return acc;
}

template <int BC, int R>
struct smem32 {
  float txh[TI], txl[TI], tyh[TI], tyl[TI], tnx[TI], tny[TI], tsp[TI];
  float2 A[TJ][TI + 1];
  float2 B[BC ? TJ : 1][TI + 1];
  float2 X[BC ? 4 : 1][TJ][R];
};

template <int BC, int R>
__global__ void __launch_bounds__(NT, 2) k_pair_fp32(pair_params P) {
  extern __shared__ __align__(16) unsigned char raw[];
  smem32<BC, R>& S = *reinterpret_cast<smem32<BC, R>*>(raw);
  constexpr int RQ = R / 8;
  const int n = P.n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = blockIdx.x * TI;
  const int split = blockIdx.y;
  const int rb0 = blockIdx.z * R;
  const int rbn = min(R, P.nrhs - rb0);
  const int ntiles = (n + TJ - 1) / TJ;
  const int t_begin = split * P.tiles_per_split;
  const int t_end = min(ntiles, t_begin + P.tiles_per_split);
  const int bw = 2 * P.b + 1;

  for (int q = tid; q < TI; q += NT) {
    const int i = i0 + q;
    const bool ok = i < n;
    S.txh[q] = ok ? P.g.xh[i] : 0.f;
    S.txl[q] = ok ? P.g.xl[i] : 0.f;
    S.tyh[q] = ok ? P.g.yh[i] : 0.f;
    S.tyl[q] = ok ? P.g.yl[i] : 0.f;
    S.tnx[q] = ok ? P.g.nx[i] : 0.f;
    S.tny[q] = ok ? P.g.ny[i] : 0.f;
    S.tsp[q] = ok ? P.g.sp[i] : 1.f;
  }

  float2 acc[BC ? 4 : 1][4][RQ];
#pragma unroll
  for (int o = 0; o < (BC ? 4 : 1); ++o)
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < RQ; ++q) acc[o][p][q] = make_float2(0.f, 0.f);

  for (int t = t_begin; t < t_end; ++t) {
    const int j0 = t * TJ;
    const int j = j0 + lane;
    const bool jok = j < n;
    __syncthreads();
    // stage right-hand sides of this source tile
    for (int e = tid; e < TJ * R; e += NT) {
      const int jl = e / R, r = e % R;
      const int jj = j0 + jl;
      float2 xv = make_float2(0.f, 0.f), uv = xv;
      if (jj < n && r < rbn) {
        xv = P.xin[(size_t)(rb0 + r) * n + jj];
        if (BC) uv = P.uin[(size_t)(rb0 + r) * n + jj];
      }
      if constexpr (BC == 1) {
        const float inv = jj < n ? 1.0f / P.g.sp[jj] : 0.f;
        const float n1 = jj < n ? P.g.nx[jj] * inv : 0.f;
        const float n2 = jj < n ? P.g.ny[jj] * inv : 0.f;
        S.X[0][jl][r] = uv;
        S.X[1][jl][r] = make_float2(n1 * xv.x, n1 * xv.y);
        S.X[2][jl][r] = make_float2(n2 * xv.x, n2 * xv.y);
        S.X[3][jl][r] = xv;
      } else {
        S.X[0][jl][r] = xv;
      }
    }
    // this lane's source
    const float sxh = jok ? P.g.xh[j] : 0.f, sxl = jok ? P.g.xl[j] : 0.f;
    const float syh = jok ? P.g.yh[j] : 0.f, syl = jok ? P.g.yl[j] : 0.f;
    const float snx = jok ? P.g.nx[j] : 0.f, sny = jok ? P.g.ny[j] : 0.f;
    const float ssp = jok ? P.g.sp[j] : 1.f;
    __syncthreads();  // target geometry (first tile) and X are in place

    // ---- entries: warp handles rows warp + 8 q, lane = source
#pragma unroll 2
    for (int q = 0; q < TI / 8; ++q) {
      const int il = warp + 8 * q;
      const int i = i0 + il;
      float2 a = make_float2(0.f, 0.f), b = a;
      if (i < n && jok) {
        int d = i - j;
        if (d < 0) d += n;
        int dd = d <= P.b ? d : (d >= n - P.b ? d - n : INT_MAX);
        if (dd != INT_MAX) {
          a = P.band[(size_t)i * bw + dd + P.b];
          if (BC) b = P.band2[(size_t)i * bw + dd + P.b];
        } else {
          pair_entries_fp32<BC>(P, S.txh[il], S.txl[il], S.tyh[il], S.tyl[il], S.tnx[il],
                                S.tny[il], S.tsp[il], sxh, sxl, syh, syl, snx, sny, ssp,
                                P.w32[d], a, b);
        }
      }
      S.A[lane][il] = a;
      if constexpr (BC == 1) S.B[lane][il] = b;
    }
    __syncthreads();

    // ---- contraction: lane -> targets lane + 32 p, warp -> right-hand sides warp*RQ + q
    const int jn = min(TJ, n - j0);
    for (int jl = 0; jl < jn; ++jl) {
      float2 av[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) av[p] = S.A[jl][lane + 32 * p];
      if constexpr (BC == 0) {
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
          const float2 xv = S.X[0][jl][warp * RQ + q];
#pragma unroll
          for (int p = 0; p < 4; ++p) acc[0][p][q] = cmul_add(acc[0][p][q], av[p], xv);
        }
      } else {
        float2 bv[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) bv[p] = S.B[jl][lane + 32 * p];
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
          const int r = warp * RQ + q;
          const float2 x0 = S.X[0][jl][r], x1 = S.X[1][jl][r], x2 = S.X[2][jl][r],
                       x3 = S.X[3][jl][r];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            acc[0][p][q] = cmul_add(acc[0][p][q], av[p], x0);
            acc[1][p][q] = cmul_add(acc[1][p][q], av[p], x1);
            acc[2][p][q] = cmul_add(acc[2][p][q], av[p], x2);
            acc[3 * BC][p][q] = cmul_add(acc[3 * BC][p][q], bv[p], x3);
          }
        }
      }
    }
  }

#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = i0 + lane + 32 * p;
    if (i >= n) continue;
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
      const int r = warp * RQ + q;
      if (r >= rbn) continue;
#pragma unroll
      for (int o = 0; o < (BC ? 4 : 1); ++o)
        P.part[(((size_t)o * P.splits + split) * P.nrhs + rb0 + r) * n + i] = acc[o][p][q];
    }
  }
}

// y = sum of split partials in FP64; hard: t = S u (complex64 for the
// derivative) and y = 1/2 x - D' x - i (omega^2/eta)(n1 S n1 x + n2 S n2 x)
template <int BC>
__global__ void k_reduce32(int n, int nrhs, int splits, double omega, double eta, geom_dev g,
                           const float2* __restrict__ part, const double2* __restrict__ x,
                           float2* __restrict__ t_out, double2* __restrict__ y) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t tot = (size_t)n * nrhs;
  if (e >= tot) return;
  const size_t so = (size_t)splits * tot;
  double2 s[4] = {};
  for (int o = 0; o < (BC ? 4 : 1); ++o) {
    double2 v = make_double2(0.0, 0.0);
    for (int sp = 0; sp < splits; ++sp) {
      const float2 p = part[o * so + (size_t)sp * tot + e];
      v.x += p.x;
      v.y += p.y;
    }
    s[o] = v;
  }
  if (BC == 0) {
    y[e] = s[0];
  } else {
    const int i = (int)(e % n);
    const double inv = 1.0 / g.sp[i];
    const double n1 = g.nx[i] * inv, n2 = g.ny[i] * inv;
    const double2 m = make_double2(n1 * s[1].x + n2 * s[2].x, n1 * s[1].y + n2 * s[2].y);
    const double k = omega * omega / eta;
    const double2 xv = x[e];
    y[e] = make_double2(0.5 * xv.x - s[3].x + k * m.y, 0.5 * xv.y - s[3].y - k * m.x);
    t_out[e] = make_float2((float)s[0].x, (float)s[0].y);
  }
}

__global__ void k_to32(size_t len, const double2* __restrict__ in, float2* __restrict__ out) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < len) out[e] = make_float2((float)in[e].x, (float)in[e].y);
}

// out[k][i] (+)= (scale / s_i) sum_j c_{(i-j) mod n} in[k][j] in FP32 with
// blocked accumulation (256-source partial sums); out complex64 or complex128
constexpr int SPT = 256;
template <bool OUT64>
__global__ void __launch_bounds__(SPT)
k_spectral32(int n, const float* __restrict__ ct, const double* __restrict__ sp,
             const float2* __restrict__ in, double2 scale, float2* __restrict__ out32,
             double2* __restrict__ out64) {
  __shared__ float2 xs[SPT];
  const int i = blockIdx.x * SPT + threadIdx.x;
  const int k = blockIdx.y;
  const float2* ink = in + (size_t)k * n;
  float2 outer = make_float2(0.f, 0.f);
  for (int j0 = 0; j0 < n; j0 += SPT) {
    __syncthreads();
    const int jj = j0 + threadIdx.x;
    xs[threadIdx.x] = jj < n ? ink[jj] : make_float2(0.f, 0.f);
    __syncthreads();
    if (i < n) {
      const int jn = min(SPT, n - j0);
      int idx = i - j0;
      if (idx < 0) idx += n;
      float2 acc = make_float2(0.f, 0.f);
      for (int q = 0; q < jn; ++q) {
        const float c = ct[idx];
        acc.x = fmaf(c, xs[q].x, acc.x);
        acc.y = fmaf(c, xs[q].y, acc.y);
        idx = idx == 0 ? n - 1 : idx - 1;
      }
      outer.x += acc.x;
      outer.y += acc.y;
    }
  }
  if (i < n) {
    const double inv = 1.0 / sp[i];
    const double sx = scale.x * inv, sy = scale.y * inv;
    const double2 v = make_double2(sx * outer.x - sy * outer.y, sx * outer.y + sy * outer.x);
    const size_t e = (size_t)k * n + i;
    if (OUT64) {
      out64[e] = make_double2(out64[e].x + v.x, out64[e].y + v.y);
    } else {
      out32[e] = make_float2((float)v.x, (float)v.y);
    }
  }
}

// ---------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------
// Largest |x|, |y| over the nodes, as the bit pattern of a non-negative float
// (ordered like the values), for the coordinate grid below
__global__ void k_coord_bound(int n, geom_dev g, unsigned* __restrict__ bound) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float m = 0.f;
  if (i < n) m = fmaxf(fabsf((float)g.x[i]), fabsf((float)g.y[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(bound, __float_as_uint(m));
}

// FP32 geometry.  Coordinates scaled by omega and split as hi + lo with hi on
// the grid 2^-g, g = 10 - e where every omega |x|, omega |y| < 2^e: then a hi
// difference is a multiple of 2^-g below 2^(e+1) (+ one grid step), exact in
// FP32, and the sum of two squared hi differences a multiple of 2^-2g below
// 2^23.1 of them, exact as well; the lo parts (|lo| <= 2^(e-11)) keep the rest
// to ~2^(e-35).
__global__ void k_geo32(int n, geom_dev g, geo32 o, const double* __restrict__ w,
                        const double* __restrict__ ct, const unsigned* __restrict__ bound,
                        double omega, double eta, double h, float* __restrict__ w32,
                        float* __restrict__ c32, float4* __restrict__ pk,
                        float2* __restrict__ wkt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 8) wkt[2 * n + i] = make_float2(0.f, 0.f);
  if (i >= n) return;
  int e = 0;
  const double m = omega * (double)__uint_as_float(*bound);
  if (m > 0.0) frexp(m, &e);
  const double q = ldexp(1.0, 10 - e), qi = ldexp(1.0, e - 10);
  const double x = omega * g.x[i], y = omega * g.y[i];
  const double xhd = rint(x * q) * qi, yhd = rint(y * q) * qi;
  const float xh = (float)xhd, yh = (float)yhd;
  const float xl = (float)(x - xhd), yl = (float)(y - yhd);
  o.xh[i] = xh;
  o.xl[i] = xl;
  o.yh[i] = yh;
  o.yl[i] = yl;
  o.nx[i] = (float)g.nx[i];
  o.ny[i] = (float)g.ny[i];
  o.sp[i] = (float)g.sp[i];
  w32[i] = (float)w[i];
  c32[i] = (float)ct[i];
  // the Kress table twice over, divided by pi h, indexed by i - j + n (no
  // cyclic wrap), paired with the weight of the next source; the zero tail is
  // written above
  const double ph = 3.141592653589793 * h;
  const float2 wk = make_float2((float)(w[i] / ph), (float)(w[i == 0 ? n - 1 : i - 1] / ph));
  wkt[i] = wk;
  wkt[n + i] = wk;
  const double f = 0.25 * h * 0.7978845608028654;   // hq c0
  const double nx = g.nx[i], ny = g.ny[i], sp = g.sp[i];
  pk[i] = make_float4(xh, xl, yh, yl);
  pk[n + i] = make_float4((float)(omega * f * nx), (float)(omega * f * ny),
                          (float)(f * eta * sp), (float)(f * sp));
  pk[2 * n + i] = make_float4((float)(omega * nx / sp), (float)(omega * ny / sp), 0.f, 0.f);
}

// Largest cyclic index distance |i - j| of a pair with omega r < X0 (with a
// 1% margin), and the largest omega r over all pairs.
__global__ void __launch_bounds__(256)
k_band_scan(int n, double omega, geom_dev g, int* __restrict__ bmax, float* __restrict__ xmax) {
  __shared__ float sx[256], sy[256];
  const int i = blockIdx.x * 256 + threadIdx.x;
  const float xi = i < n ? (float)g.x[i] : 0.f, yi = i < n ? (float)g.y[i] : 0.f;
  const float lim = (float)((kX0 * 1.01) / omega);
  const float lim2 = lim * lim;
  int best = 0;
  float far2 = 0.f;
  for (int j0 = 0; j0 < n; j0 += 256) {
    __syncthreads();
    const int jj = j0 + threadIdx.x;
    sx[threadIdx.x] = jj < n ? (float)g.x[jj] : 0.f;
    sy[threadIdx.x] = jj < n ? (float)g.y[jj] : 0.f;
    __syncthreads();
    if (i < n) {
      const int jn = min(256, n - j0);
      for (int q = 0; q < jn; ++q) {
        const float dx = xi - sx[q], dy = yi - sy[q];
        const float r2 = dx * dx + dy * dy;
        far2 = fmaxf(far2, r2);
        if (r2 < lim2) {
          int d = i - (j0 + q);
          if (d < 0) d = -d;
          d = min(d, n - d);
          best = max(best, d);
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    far2 = fmaxf(far2, __shfl_xor_sync(0xffffffffu, far2, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(bmax, best);
    atomicMax(reinterpret_cast<int*>(xmax), __float_as_int((float)(omega * sqrt((double)far2))));
  }
}

// FP32 band entries (offsets |dd| <= b) from the double-float band of width
// bd >= b: the high parts (the FP32 rounding of the FP64 entries); `ops`
// bands of each kind (sound hard: S, then D')
__global__ void k_band_from_df(int n, int b, int bd, int ops, const float4* __restrict__ dfb,
                               float2* __restrict__ band) {
  const int bw = 2 * b + 1, bwd = 2 * bd + 1;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * bw) return;
  const int i = (int)(e / bw);
  const int dd = (int)(e % bw) - b;
  for (int o = 0; o < ops; ++o) {
    const float4 v = dfb[(size_t)o * n * bwd + (size_t)i * bwd + dd + bd];
    band[(size_t)o * n * bw + e] = make_float2(v.x, v.z);
  }
}

template <int BC>
__global__ void k_band_fill(int n, int b, double omega, double eta, geom_dev g,
                            const double* __restrict__ wtab, const double2* __restrict__ diag,
                            float2* __restrict__ band, float2* __restrict__ band2) {
  const int bw = 2 * b + 1;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * bw) return;
  const int i = (int)(e / bw);
  const int dd = (int)(e % bw) - b;
  int j = i - dd;
  j %= n;
  if (j < 0) j += n;
  double2 a, bb = make_double2(0.0, 0.0);
  if (j == i) {
    if (BC) {
      a = diag[2 * i];
      bb = diag[2 * i + 1];
    } else {
      a = diag[i];
    }
  } else {
    int d = i - j;
    if (d < 0) d += n;
    const double h = 2.0 * CFIE_PI / n;
    pair_entries_fp64<BC>(g.x[i] - g.x[j], g.y[i] - g.y[j], omega, eta, h, wtab[d], g.nx[j],
                          g.ny[j], g.sp[j], g.nx[i], g.ny[i], g.sp[i], a, bb);
  }
  band[e] = make_float2((float)a.x, (float)a.y);
  if (BC) band2[e] = make_float2((float)bb.x, (float)bb.y);
}

unsigned nblk(size_t len, int t = 256) { return (unsigned)((len + t - 1) / t); }

template <int BC, int R>
int launch32(cfie_op* op, pair_params P, int rowtiles, int slices) {
  size_t smem = sizeof(smem32<BC, R>);
  CFIE_CHECK_CUDA(cudaFuncSetAttribute(k_pair_fp32<BC, R>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 1;
  CFIE_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_fp32<BC, R>, NT,
                                                                smem));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, op->ctx->device);
  const int slots = std::max(1, per_sm) * sms;
  const int ntiles = (P.n + TJ - 1) / TJ;
  // source splits: pick the count (<= 16) whose grid best fills whole waves
  int best_s = 1;
  double best_eff = -1.0;
  for (int s = 1; s <= std::min(16, ntiles); ++s) {
    const double ctas = (double)rowtiles * slices * s;
    const double waves = std::ceil(ctas / slots);
    const double eff = ctas / (waves * slots) - 0.002 * s;  // prefer fewer splits on ties
    if (eff > best_eff) {
      best_eff = eff;
      best_s = s;
    }
  }
  int tps = (ntiles + best_s - 1) / best_s;
  P.splits = (ntiles + tps - 1) / tps;
  P.tiles_per_split = tps;
  const int ops = BC ? 4 : 1;
  op->partial.reserve(sizeof(float2) * (size_t)ops * P.splits * P.nrhs * P.n);
  P.part = op->partial.as<float2>();
  dim3 grid(rowtiles, P.splits, slices);
  {
    prof_scope ps(op->ctx, CFIE_K_MATVEC_FP32);
    k_pair_fp32<BC, R><<<grid, NT, smem, op->ctx->stream>>>(P);
    CFIE_CHECK_LAUNCH();
  }
  return P.splits;
}

}  // namespace

void fp32_prepare(cfie_op* op) {
  const int n = op->n;
  cudaStream_t st = op->ctx->stream;
  op->geo32.reserve(sizeof(float) * geo32_floats(n));
  // band width and argument range
  dbuf scan;
  scan.reserve(16);
  CFIE_CHECK_CUDA(cudaMemsetAsync(scan.p, 0, 16, st));
  k_band_scan<<<nblk(n), 256, 0, st>>>(n, op->omega, op->g, scan.as<int>(),
                                        reinterpret_cast<float*>(scan.as<int>() + 1));
  CFIE_CHECK_LAUNCH();
  int hb[2];
  CFIE_CHECK_CUDA(cudaMemcpyAsync(hb, scan.p, 8, cudaMemcpyDeviceToHost, st));
  CFIE_CHECK_CUDA(cudaStreamSynchronize(st));
  float xmax;
  std::memcpy(&xmax, &hb[1], 4);
  if (!(xmax < 1.0e5f))
    throw cfie_error(CFIE_EINVAL, "FP32 path needs omega * diameter < 1e5");
  int b = std::max(1, hb[0]);
  b = std::min(b, n / 2);
  const size_t bw = 2 * (size_t)b + 1;
  const int ops = op->bc == CFIE_SOUND_HARD ? 2 : 1;
  if ((size_t)n * bw * ops * sizeof(float2) > ((size_t)4 << 30))
    throw cfie_error(CFIE_EINVAL,
                     "FP32 near-field band too wide (curve too close to itself or too few "
                     "points per wavelength); use CFIE_FP64");
  op->band_b = b;
  op->band.reserve(sizeof(float2) * (size_t)n * bw * ops);
  float* base = op->geo32.as<float>();
  geo32 o{base, base + n, base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n, base + 6 * n};
  float* w32 = base + 7 * n;
  float* c32 = base + 8 * n;
  unsigned* bound = reinterpret_cast<unsigned*>(scan.as<int>() + 2);
  CFIE_CHECK_CUDA(cudaMemsetAsync(bound, 0, sizeof(unsigned), st));
  k_coord_bound<<<nblk(n), 256, 0, st>>>(n, op->g, bound);
  CFIE_CHECK_LAUNCH();
  k_geo32<<<nblk(n), 256, 0, st>>>(n, op->g, o, op->wtab.as<double>(), op->ctab.as<double>(),
                                    bound, op->omega, op->eta, op->h, w32, c32,
                                    reinterpret_cast<float4*>(base + geo32_pack_offset(n)),
                                    reinterpret_cast<float2*>(base + geo32_wk_offset(n)));
  CFIE_CHECK_LAUNCH();
}

// The FP32 near band (omega r < 16), after df_prepare: rounded from the
// FP64-evaluated double-float band when that one is at least as wide (it holds
// the same entries), else evaluated in FP64 here.
void fp32_band(cfie_op* op) {
  const int n = op->n, b = op->band_b;
  const size_t bw = 2 * (size_t)b + 1;
  cudaStream_t st = op->ctx->stream;
  float2* band = op->band.as<float2>();
  const bool hard = op->bc == CFIE_SOUND_HARD;
  if (op->df_b >= b) {
    k_band_from_df<<<nblk((size_t)n * bw), 256, 0, st>>>(n, b, op->df_b, hard ? 2 : 1,
                                                          op->df_band.as<float4>(), band);
  } else if (!hard) {
    k_band_fill<0><<<nblk((size_t)n * bw), 256, 0, st>>>(n, b, op->omega, op->eta, op->g,
                                                          op->wtab.as<double>(),
                                                          op->diag.as<double2>(), band, nullptr);
  } else {
    k_band_fill<1><<<nblk((size_t)n * bw), 256, 0, st>>>(
        n, b, op->omega, op->eta, op->g, op->wtab.as<double>(), op->diag.as<double2>(), band,
        band + (size_t)n * bw);
  }
  CFIE_CHECK_LAUNCH();
  CFIE_CHECK_CUDA(cudaStreamSynchronize(st));
}

void k_to32_fp32(cfie_op* op, const double2* x, float2* x32, size_t tot) {
  k_to32<<<nblk(tot), 256, 0, op->ctx->stream>>>(tot, x, x32);
  CFIE_CHECK_LAUNCH();
}

void spectral32_apply(cfie_op* op, const float2* x32, float2* u32, int nrhs) {
  spectral_fft32_apply(op, x32, u32, nrhs);
}

void spectral32_accumulate(cfie_op* op, const float2* t32, double2* y, int nrhs) {
  spectral_fft32_accumulate(op, t32, y, make_double2(0.0, -1.0 / op->eta), nrhs);
}

void matvec_fp32(cfie_op* op, const double2* x, double2* y, int nrhs) {
  const int n = op->n;
  const bool hard = op->bc == CFIE_SOUND_HARD;
  cudaStream_t st = op->ctx->stream;
  const size_t tot = (size_t)n * nrhs;
  float* base = op->geo32.as<float>();
  pair_params P{};
  P.n = n;
  P.b = op->band_b;
  P.nrhs = nrhs;
  P.wh = (float)op->omega;
  P.eta = (float)op->eta;
  P.h = (float)op->h;
  P.g = geo32{base, base + n, base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n, base + 6 * n};
  P.w32 = base + 7 * n;
  const size_t bw = 2 * (size_t)op->band_b + 1;
  P.band = op->band.as<float2>();
  P.band2 = hard ? P.band + (size_t)n * bw : nullptr;
  op->xin32.reserve(sizeof(float2) * tot * (hard ? 3 : 1));
  float2* x32 = op->xin32.as<float2>();
  k_to32<<<nblk(tot), 256, 0, st>>>(tot, x, x32);
  CFIE_CHECK_LAUNCH();
  P.xin = x32;
  const int rowtiles = (n + TI - 1) / TI;
  if (!hard) {
    int splits;
    if (nrhs > 16)
      splits = launch32<0, 64>(op, P, rowtiles, (nrhs + 63) / 64);
    else if (nrhs > 8)
      splits = launch32<0, 16>(op, P, rowtiles, 1);
    else
      splits = launch32<0, 8>(op, P, rowtiles, 1);
    k_reduce32<0><<<nblk(tot), 256, 0, st>>>(n, nrhs, splits, op->omega, op->eta, op->g,
                                             op->partial.as<float2>(), x, nullptr, y);
    CFIE_CHECK_LAUNCH();
    return;
  }
  float2* u32 = x32 + tot;
  float2* t32 = x32 + 2 * tot;
  spectral32_apply(op, x32, u32, nrhs);
  P.uin = u32;
  int splits;
  if (nrhs > 8)
    splits = launch32<1, 16>(op, P, rowtiles, (nrhs + 15) / 16);
  else
    splits = launch32<1, 8>(op, P, rowtiles, 1);
  k_reduce32<1><<<nblk(tot), 256, 0, st>>>(n, nrhs, splits, op->omega, op->eta, op->g,
                                           op->partial.as<float2>(), x, t32, y);
  CFIE_CHECK_LAUNCH();
  // y += (1/(i eta)) (1/s) Dt t
  spectral32_accumulate(op, t32, y, nrhs);
}
