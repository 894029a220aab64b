// Off-surface scattered field from the boundary density (step after the solve;
// Section 1 of the paper evaluates u through a boundary integral without
// writing it out).  Representations whose boundary limits give eq. 1 and
// eq. 2 through the jump relations (outward normal):
//
//     sound soft:  u(x) = (D q)(x) - i eta (S q)(x)
//     sound hard:  u(x) = -(S q)(x) + (D q)(x) / (i eta)
//
//     (S q)(x) = h sum_j (i/4) H0(omega r_j) |z'_j| q_j
//     (D q)(x) = h sum_j (i/4) omega H1(omega r_j) ((x - z_j) . nu~_j / r_j) q_j
//
// discretised by the plain trapezoidal rule (spectrally accurate a few node
// spacings away from the curve), FP64 throughout with the library's own
// Hankel evaluation.  One thread per (point, quarter of the sources), sources
// staged in shared memory a tile at a time, the quarters added at the end.
#include <algorithm>

#include "hankel64.cuh"
#include "internal.h"

namespace {

constexpr int FPT = 64;      // points per CTA
constexpr int FSPL = 4;      // source quarters (threads per point)
constexpr int FNT = FPT * FSPL;
constexpr int FTJ = 128;     // sources per shared-memory tile
constexpr int FRB = 8;       // right-hand sides per CTA

template <int BC>
__global__ void __launch_bounds__(FNT)
k_field(int n, int npts, int nrhs, double omega, double eta, double h, geom_dev g,
        const double2* __restrict__ pts, const double2* __restrict__ q,
        double2* __restrict__ u) {
  __shared__ double sx[FTJ], sy[FTJ], snx[FTJ], sny[FTJ], ssp[FTJ];
  // densities of the tile during the loop, the quarters' sums after it
  constexpr int BUF = FTJ * FRB > FSPL * FPT * FRB ? FTJ * FRB : FSPL * FPT * FRB;
  __shared__ double2 buf[BUF];
  double2 (*sq)[FRB] = reinterpret_cast<double2 (*)[FRB]>(buf);
  double2 (*red)[FPT][FRB] = reinterpret_cast<double2 (*)[FPT][FRB]>(buf);
  const int tid = threadIdx.x;
  const int pl = tid % FPT, quarter = tid / FPT;
  const int p = blockIdx.x * FPT + pl;
  const int r0 = blockIdx.y * FRB;
  const int rn = min(FRB, nrhs - r0);
  const double2 xp = p < npts ? pts[p] : make_double2(0.0, 0.0);
  double2 acc[FRB];
#pragma unroll
  for (int k = 0; k < FRB; ++k) acc[k] = make_double2(0.0, 0.0);
  for (int j0 = 0; j0 < n; j0 += FTJ) {
    __syncthreads();
    for (int e = tid; e < FTJ; e += FNT) {
      const int j = j0 + e;
      const bool ok = j < n;
      sx[e] = ok ? g.x[j] : 0.0;
      sy[e] = ok ? g.y[j] : 0.0;
      snx[e] = ok ? g.nx[j] : 0.0;
      sny[e] = ok ? g.ny[j] : 0.0;
      ssp[e] = ok ? g.sp[j] : 0.0;
    }
    for (int e = tid; e < FTJ * FRB; e += FNT) {
      const int jl = e / FRB, k = e % FRB, j = j0 + jl;
      sq[jl][k] = (j < n && k < rn) ? q[(size_t)(r0 + k) * n + j] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (p >= npts) continue;
    const int jn = min(FTJ, n - j0);
    for (int jl = quarter; jl < jn; jl += FSPL) {
      const double dx = xp.x - sx[jl], dy = xp.y - sy[jl];
      const double r = sqrt(dx * dx + dy * dy);
      double J0, Y0, J1, Y1;
      h64::bessel01(omega * r, J0, Y0, J1, Y1);
      // S kernel (i/4) H0 |z'|, D kernel (i/4) omega H1 c; H = J + i Y
      const double sk = 0.25 * ssp[jl];
      const double dk = 0.25 * omega * (dx * snx[jl] + dy * sny[jl]) / r;
      const double2 S = make_double2(-sk * Y0, sk * J0);
      const double2 D = make_double2(-dk * Y1, dk * J1);
      double2 c;
      if constexpr (BC == 0) {
        c = make_double2(D.x + eta * S.y, D.y - eta * S.x);           // D - i eta S
      } else {
        c = make_double2(-S.x + D.y / eta, -S.y - D.x / eta);         // -S + D / (i eta)
      }
#pragma unroll
      for (int k = 0; k < FRB; ++k) {
        const double2 qq = sq[jl][k];
        acc[k].x += c.x * qq.x - c.y * qq.y;
        acc[k].y += c.x * qq.y + c.y * qq.x;
      }
    }
  }
  __syncthreads();   // every thread is done with the last tile's densities
#pragma unroll
  for (int k = 0; k < FRB; ++k) red[quarter][pl][k] = acc[k];
  __syncthreads();
  if (quarter == 0 && p < npts) {
    for (int k = 0; k < rn; ++k) {
      double2 s = make_double2(0.0, 0.0);
      for (int t = 0; t < FSPL; ++t) {
        s.x += red[t][pl][k].x;
        s.y += red[t][pl][k].y;
      }
      u[(size_t)(r0 + k) * npts + p] = make_double2(h * s.x, h * s.y);
    }
  }
}

}  // namespace

void field_eval(cfie_op* op, const double2* q, int nrhs, int npts, const double2* pts,
                double2* u) {
  const dim3 grid((npts + FPT - 1) / FPT, (nrhs + FRB - 1) / FRB);
  cudaStream_t st = op->ctx->stream;
  if (op->bc == CFIE_SOUND_SOFT)
    k_field<0><<<grid, FNT, 0, st>>>(op->n, npts, nrhs, op->omega, op->eta, op->h, op->g, pts, q,
                                     u);
  else
    k_field<1><<<grid, FNT, 0, st>>>(op->n, npts, nrhs, op->omega, op->eta, op->h, op->g, pts, q,
                                     u);
  CFIE_CHECK_LAUNCH();
}
