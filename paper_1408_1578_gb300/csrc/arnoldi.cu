// Restarted GMRES (Section 3 of the paper: GMRES with a relative tolerance and
// a restart length) for nrhs independent right-hand sides, with the Arnoldi
// orthogonalisation, Givens rotations, Hessenberg least-squares solve and the
// solution update all in FP64 on the GPU, and mixed-precision iterative
// refinement on the outer FP64 residual for the FP32 / tensor precisions.
//
// Arnoldi step j (per right-hand side k, V_k = [v_0 .. v_j]):
//   w = A v_j
//   classical Gram-Schmidt twice (CGS2):  h = V^H w, w -= V h   (two passes)
//   H(0:j, j) = h_1 + h_2,  H(j+1, j) = ||w||,  v_{j+1} = w / ||w||
//   rotate column j of H by the previous Givens rotations, build rotation j,
//   g(j+1) = -conj(s_j) g(j), g(j) = c_j g(j); |g(j+1)| is the residual norm.
// After a cycle: R y = g (back substitution), x += V y, then the true residual.
//
// Memory layout: V is [(m+1)][nrhs][n] complex128, so basis vector j of all
// right-hand sides is a column-major n x nrhs block that the matvec reads
// directly.  H is [nrhs][m+1][m].  The orthogonalisation kernels stream V once
// per pass (HBM-bound); a CTA owns a chunk of 2048 nodes of one right-hand side.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace {

constexpr int AT = 256;          // threads per CTA
constexpr int AE = 8;            // nodes per thread
constexpr int CH = AT * AE;      // nodes per chunk
constexpr int MAXJ = 512;        // largest restart length

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partial[k][jj][chunk] = sum_{i in chunk} conj(V[jj][k][i]) w[k][i], jj = 0..J
__global__ void __launch_bounds__(AT)
k_dots(int n, int nrhs, int J, const double2* __restrict__ V, const double2* __restrict__ w,
       const int* __restrict__ act, int nchunks, double2* __restrict__ partial) {
  extern __shared__ double2 red[];  // [J+1][AT/32]
  const int k = blockIdx.y;
  if (!act[k]) return;
  const int chunk = blockIdx.x;
  const int base = chunk * CH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double2 wr[AE];
#pragma unroll
  for (int e = 0; e < AE; ++e) {
    int i = base + e * AT + threadIdx.x;
    wr[e] = i < n ? w[(size_t)k * n + i] : make_double2(0.0, 0.0);
  }
  for (int jj = 0; jj <= J; ++jj) {
    const double2* v = V + ((size_t)jj * nrhs + k) * n;
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int e = 0; e < AE; ++e) {
      int i = base + e * AT + threadIdx.x;
      if (i < n) {
        double2 a = v[i];
        re = fma(a.x, wr[e].x, fma(a.y, wr[e].y, re));
        im = fma(a.x, wr[e].y, fma(-a.y, wr[e].x, im));
      }
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) red[jj * (AT / 32) + warp] = make_double2(re, im);
  }
  __syncthreads();
  for (int jj = threadIdx.x; jj <= J; jj += AT) {
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < AT / 32; ++q) {
      s.x += red[jj * (AT / 32) + q].x;
      s.y += red[jj * (AT / 32) + q].y;
    }
    partial[((size_t)k * (J + 1) + jj) * nchunks + chunk] = s;
  }
}

// h[k][jj] = sum over chunks; H[k][jj][col] += h (first pass sets, second adds)
__global__ void k_dots_reduce(int nrhs, int J, int nchunks, int m, int col, int first,
                              const int* __restrict__ act, const double2* __restrict__ partial,
                              double2* __restrict__ hbuf, double2* __restrict__ H) {
  const int k = blockIdx.x;
  if (!act[k]) return;
  for (int jj = threadIdx.x; jj <= J; jj += blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    const double2* p = partial + ((size_t)k * (J + 1) + jj) * nchunks;
    for (int c = 0; c < nchunks; ++c) {
      s.x += p[c].x;
      s.y += p[c].y;
    }
    hbuf[(size_t)k * (J + 1) + jj] = s;
    double2* hk = H + ((size_t)k * (m + 1) + jj) * m + col;
    if (first) {
      *hk = s;
    } else {
      hk->x += s.x;
      hk->y += s.y;
    }
  }
}

// w[k][i] -= sum_jj V[jj][k][i] h[k][jj]; optional |w|^2 partial per chunk
__global__ void __launch_bounds__(AT)
k_update(int n, int nrhs, int J, const double2* __restrict__ V, const double2* __restrict__ hbuf,
         const int* __restrict__ act, double2* __restrict__ w, int nchunks,
         double* __restrict__ nrm_partial) {
  extern __shared__ double2 hs[];
  const int k = blockIdx.y;
  if (!act[k]) return;
  const int chunk = blockIdx.x;
  const int base = chunk * CH;
  for (int jj = threadIdx.x; jj <= J; jj += AT) hs[jj] = hbuf[(size_t)k * (J + 1) + jj];
  __syncthreads();
  double2 acc[AE];
#pragma unroll
  for (int e = 0; e < AE; ++e) {
    int i = base + e * AT + threadIdx.x;
    acc[e] = i < n ? w[(size_t)k * n + i] : make_double2(0.0, 0.0);
  }
  for (int jj = 0; jj <= J; ++jj) {
    const double2* v = V + ((size_t)jj * nrhs + k) * n;
    const double2 hh = hs[jj];
#pragma unroll
    for (int e = 0; e < AE; ++e) {
      int i = base + e * AT + threadIdx.x;
      if (i < n) {
        double2 a = v[i];
        acc[e].x -= a.x * hh.x - a.y * hh.y;
        acc[e].y -= a.x * hh.y + a.y * hh.x;
      }
    }
  }
  double ss = 0.0;
#pragma unroll
  for (int e = 0; e < AE; ++e) {
    int i = base + e * AT + threadIdx.x;
    if (i < n) {
      w[(size_t)k * n + i] = acc[e];
      ss += acc[e].x * acc[e].x + acc[e].y * acc[e].y;
    }
  }
  if (nrm_partial) {
    __shared__ double red[AT / 32];
    ss = warp_sum(ss);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < AT / 32; ++q) t += red[q];
      nrm_partial[(size_t)k * nchunks + chunk] = t;
    }
  }
}

// One thread per right-hand side: ||w||, Givens rotations, residual estimate.
__global__ void k_givens(int nrhs, int m, int j, int nchunks, const int* __restrict__ act,
                         const double* __restrict__ nrm_partial, double2* __restrict__ H,
                         double* __restrict__ cs, double2* __restrict__ sn,
                         double2* __restrict__ gv, double* __restrict__ hnorm,
                         double* __restrict__ res) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nrhs || !act[k]) return;
  double s2 = 0.0;
  for (int c = 0; c < nchunks; ++c) s2 += nrm_partial[(size_t)k * nchunks + c];
  double hn = sqrt(s2);
  hnorm[k] = hn;
  double2* Hk = H + (size_t)k * (m + 1) * m;
  Hk[(size_t)(j + 1) * m + j] = make_double2(hn, 0.0);
  // previous rotations on column j
  for (int q = 0; q < j; ++q) {
    double2 a = Hk[(size_t)q * m + j], b = Hk[(size_t)(q + 1) * m + j];
    double c = cs[(size_t)k * m + q];
    double2 s = sn[(size_t)k * m + q];
    // [c s; -conj(s) c]
    double2 na = make_double2(c * a.x + s.x * b.x - s.y * b.y, c * a.y + s.x * b.y + s.y * b.x);
    double2 nb = make_double2(-(s.x * a.x + s.y * a.y) + c * b.x, -(s.x * a.y - s.y * a.x) + c * b.y);
    Hk[(size_t)q * m + j] = na;
    Hk[(size_t)(q + 1) * m + j] = nb;
  }
  double2 a = Hk[(size_t)j * m + j];
  double bn = hn;  // b = hn (real)
  double c;
  double2 s;
  double aa = hypot(a.x, a.y);
  if (bn == 0.0) {
    c = 1.0;
    s = make_double2(0.0, 0.0);
  } else if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);  // conj(b)/|b| with b real positive
  } else {
    double t = hypot(aa, bn);
    c = aa / t;
    // s = (a/|a|) conj(b) / t
    s = make_double2(a.x / aa * bn / t, a.y / aa * bn / t);
  }
  cs[(size_t)k * m + j] = c;
  sn[(size_t)k * m + j] = s;
  // H(j,j) = c a + s b
  Hk[(size_t)j * m + j] = make_double2(c * a.x + s.x * bn, c * a.y + s.y * bn);
  Hk[(size_t)(j + 1) * m + j] = make_double2(0.0, 0.0);
  double2 gj = gv[(size_t)k * (m + 1) + j];
  // g(j+1) = -conj(s) g(j); g(j) = c g(j)
  double2 g1 = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
  gv[(size_t)k * (m + 1) + j + 1] = g1;
  gv[(size_t)k * (m + 1) + j] = make_double2(c * gj.x, c * gj.y);
  res[k] = hypot(g1.x, g1.y);
}

// v_{j+1} = w / ||w|| (0 on breakdown)
__global__ void k_scale(int n, int nrhs, const int* __restrict__ act, const double* __restrict__ hn,
                        const double2* __restrict__ w, double2* __restrict__ vout) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * nrhs) return;
  int k = (int)(e / n);
  if (!act[k]) return;
  double h = hn[k];
  double inv = h > 0.0 ? 1.0 / h : 0.0;
  double2 v = w[e];
  vout[e] = make_double2(v.x * inv, v.y * inv);
}

// per right-hand side: y = R^{-1} g on the leading kd x kd triangle
__global__ void k_lsq(int nrhs, int m, const int* __restrict__ kd, const double2* __restrict__ H,
                      const double2* __restrict__ gv, double2* __restrict__ y) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nrhs) return;
  int K = kd[k];
  const double2* Hk = H + (size_t)k * (m + 1) * m;
  double2* yk = y + (size_t)k * m;
  for (int i = K - 1; i >= 0; --i) {
    double2 s = gv[(size_t)k * (m + 1) + i];
    for (int q = i + 1; q < K; ++q) {
      double2 h = Hk[(size_t)i * m + q], yq = yk[q];
      s.x -= h.x * yq.x - h.y * yq.y;
      s.y -= h.x * yq.y + h.y * yq.x;
    }
    double2 d = Hk[(size_t)i * m + i];
    double den = d.x * d.x + d.y * d.y;
    yk[i] = den > 0.0 ? make_double2((s.x * d.x + s.y * d.y) / den, (s.y * d.x - s.x * d.y) / den)
                      : make_double2(0.0, 0.0);
  }
}

// x[k][i] += sum_{jj < kd[k]} V[jj][k][i] y[k][jj]
__global__ void k_xupdate(int n, int nrhs, int m, const int* __restrict__ kd,
                          const double2* __restrict__ V, const double2* __restrict__ y,
                          double2* __restrict__ x) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * nrhs) return;
  int k = (int)(e / n);
  int i = (int)(e % n);
  int K = kd[k];
  if (K == 0) return;
  double2 acc = x[e];
  for (int jj = 0; jj < K; ++jj) {
    double2 v = V[((size_t)jj * nrhs + k) * n + i];
    double2 yy = y[(size_t)k * m + jj];
    acc.x += v.x * yy.x - v.y * yy.y;
    acc.y += v.x * yy.y + v.y * yy.x;
  }
  x[e] = acc;
}

// r = f - ax (ax may be null: r = f); per-rhs ||r||^2 and ||f||^2 partials
__global__ void __launch_bounds__(AT)
k_residual(int n, int nrhs, const double2* __restrict__ f, const double2* __restrict__ ax,
           double2* __restrict__ r, int nchunks, double* __restrict__ rr, double* __restrict__ ff) {
  const int k = blockIdx.y, chunk = blockIdx.x, base = chunk * CH;
  double sr = 0.0, sf = 0.0;
#pragma unroll
  for (int e = 0; e < AE; ++e) {
    int i = base + e * AT + threadIdx.x;
    if (i < n) {
      size_t idx = (size_t)k * n + i;
      double2 fv = f[idx];
      double2 v = fv;
      if (ax) {
        double2 a = ax[idx];
        v.x -= a.x;
        v.y -= a.y;
      }
      if (r) r[idx] = v;
      sr += v.x * v.x + v.y * v.y;
      sf += fv.x * fv.x + fv.y * fv.y;
    }
  }
  __shared__ double red[2][AT / 32];
  sr = warp_sum(sr);
  sf = warp_sum(sf);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sr;
    red[1][threadIdx.x >> 5] = sf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < AT / 32; ++q) {
      a += red[0][q];
      b += red[1][q];
    }
    rr[(size_t)k * nchunks + chunk] = a;
    ff[(size_t)k * nchunks + chunk] = b;
  }
}

__global__ void k_sum_chunks(int nrhs, int nchunks, const double* __restrict__ a,
                             const double* __restrict__ b, double* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nrhs) return;
  double s = 0.0, t = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    s += a[(size_t)k * nchunks + c];
    t += b[(size_t)k * nchunks + c];
  }
  out[k] = sqrt(s);
  out[nrhs + k] = sqrt(t);
}

// v0[k] = r[k] / beta[k]; g[k] = (beta, 0, ...)
__global__ void k_start(int n, int nrhs, int m, const int* __restrict__ act,
                        const double* __restrict__ beta, const double2* __restrict__ r,
                        double2* __restrict__ v0, double2* __restrict__ gv) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < (size_t)nrhs * (m + 1)) {
    int k = (int)(e / (m + 1));
    int q = (int)(e % (m + 1));
    gv[e] = make_double2(q == 0 && act[k] ? beta[k] : 0.0, 0.0);
  }
  if (e >= (size_t)n * nrhs) return;
  int k = (int)(e / n);
  double b = beta[k];
  double inv = (act[k] && b > 0.0) ? 1.0 / b : 0.0;
  double2 v = r[e];
  v0[e] = make_double2(v.x * inv, v.y * inv);
}

__global__ void k_axpy(size_t len, const double2* __restrict__ d, double2* __restrict__ x) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  double2 a = x[e], b = d[e];
  x[e] = make_double2(a.x + b.x, a.y + b.y);
}

__global__ void k_zero(size_t len, double2* __restrict__ x) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < len) x[e] = make_double2(0.0, 0.0);
}

unsigned blocks_for(size_t len, int t = 256) { return (unsigned)((len + t - 1) / t); }

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
using matvec_t = void (*)(cfie_op*, const double2*, double2*, int);

struct ws {
  double2 *V, *H, *gv, *sn, *w, *hbuf, *y, *part;
  double *cs, *hn, *res, *nrmp, *rr, *ff, *norms;
  int *act, *kd;
  int nchunks;
};

ws workspace(cfie_op* op, int nrhs, int m) {
  const int n = op->n;
  const int nchunks = (n + CH - 1) / CH;
  const size_t nv = (size_t)n * nrhs;
  op->V.reserve(sizeof(double2) * nv * (m + 1));
  op->wv.reserve(sizeof(double2) * nv);
  op->H.reserve(sizeof(double2) * (size_t)nrhs * (m + 1) * m);
  size_t sm = 0;
  auto take = [&](size_t bytes) { size_t o = sm; sm += (bytes + 255) & ~size_t(255); return o; };
  size_t o_gv = take(sizeof(double2) * nrhs * (m + 1));
  size_t o_sn = take(sizeof(double2) * nrhs * m);
  size_t o_hb = take(sizeof(double2) * nrhs * (m + 1));
  size_t o_y = take(sizeof(double2) * nrhs * m);
  size_t o_part = take(sizeof(double2) * nrhs * (m + 1) * nchunks);
  size_t o_cs = take(sizeof(double) * nrhs * m);
  size_t o_hn = take(sizeof(double) * nrhs);
  size_t o_res = take(sizeof(double) * nrhs);
  size_t o_nrmp = take(sizeof(double) * nrhs * nchunks);
  size_t o_rr = take(sizeof(double) * nrhs * nchunks);
  size_t o_ff = take(sizeof(double) * nrhs * nchunks);
  size_t o_norms = take(sizeof(double) * 2 * nrhs);
  size_t o_act = take(sizeof(int) * nrhs);
  size_t o_kd = take(sizeof(int) * nrhs);
  op->small.reserve(sm);
  char* b = op->small.as<char>();
  ws W;
  W.V = op->V.as<double2>();
  W.H = op->H.as<double2>();
  W.w = op->wv.as<double2>();
  W.gv = (double2*)(b + o_gv);
  W.sn = (double2*)(b + o_sn);
  W.hbuf = (double2*)(b + o_hb);
  W.y = (double2*)(b + o_y);
  W.part = (double2*)(b + o_part);
  W.cs = (double*)(b + o_cs);
  W.hn = (double*)(b + o_hn);
  W.res = (double*)(b + o_res);
  W.nrmp = (double*)(b + o_nrmp);
  W.rr = (double*)(b + o_rr);
  W.ff = (double*)(b + o_ff);
  W.norms = (double*)(b + o_norms);
  W.act = (int*)(b + o_act);
  W.kd = (int*)(b + o_kd);
  W.nchunks = nchunks;
  if (op->host_res_cap < 2 * nrhs + 8) {
    if (op->host_res) cudaFreeHost(op->host_res);
    op->host_res = nullptr;
    CFIE_CHECK_CUDA(cudaMallocHost(&op->host_res, sizeof(double) * (2 * nrhs + 8)));
    op->host_res_cap = 2 * nrhs + 8;
  }
  return W;
}

// ||r_k|| and ||f_k|| to host (synchronous); r = f - ax (ax may be null)
void residual_norms(cfie_op* op, const ws& W, const double2* f, const double2* ax, double2* r,
                    int nrhs, std::vector<double>& rn, std::vector<double>& fn) {
  cudaStream_t st = op->ctx->stream;
  dim3 grid(W.nchunks, nrhs);
  k_residual<<<grid, AT, 0, st>>>(op->n, nrhs, f, ax, r, W.nchunks, W.rr, W.ff);
  CFIE_CHECK_LAUNCH();
  k_sum_chunks<<<blocks_for(nrhs, 64), 64, 0, st>>>(nrhs, W.nchunks, W.rr, W.ff, W.norms);
  CFIE_CHECK_LAUNCH();
  CFIE_CHECK_CUDA(cudaMemcpyAsync(op->host_res, W.norms, sizeof(double) * 2 * nrhs,
                                  cudaMemcpyDeviceToHost, st));
  CFIE_CHECK_CUDA(cudaStreamSynchronize(st));
  rn.assign(op->host_res, op->host_res + nrhs);
  fn.assign(op->host_res + nrhs, op->host_res + 2 * nrhs);
}

// One GMRES cycle per call: starting residual r (device), basis built with `mv`,
// x += V y.  active[k] on entry says which right-hand sides take part; tol[k]
// is the absolute residual-norm target.  Returns steps taken per rhs.
void gmres_cycle(cfie_op* op, const ws& W, matvec_t mv, const double2* r,
                 const std::vector<double>& beta, const std::vector<double>& tol,
                 std::vector<int>& active, int nrhs, int m, std::vector<int>& steps_left,
                 double2* x, std::vector<int>& its) {
  cudaStream_t st = op->ctx->stream;
  const int n = op->n;
  const size_t nv = (size_t)n * nrhs;
  std::vector<int> act = active, kd(nrhs, 0);
  int nact = 0;
  for (int k = 0; k < nrhs; ++k) nact += act[k];
  if (!nact) return;
  CFIE_CHECK_CUDA(cudaMemcpyAsync(W.act, act.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
  CFIE_CHECK_CUDA(cudaMemcpyAsync(W.norms, beta.data(), sizeof(double) * nrhs,
                                  cudaMemcpyHostToDevice, st));
  k_start<<<blocks_for(std::max(nv, (size_t)nrhs * (m + 1))), 256, 0, st>>>(n, nrhs, m, W.act,
                                                                           W.norms, r, W.V, W.gv);
  CFIE_CHECK_LAUNCH();
  op->stats.cycles++;
  for (int j = 0; j < m; ++j) {
    double2* vj = W.V + (size_t)j * nv;
    mv(op, vj, W.w, nrhs);
    {
      prof_scope ps(op->ctx, CFIE_K_ARNOLDI);
      dim3 grid(W.nchunks, nrhs);
      size_t red_smem = sizeof(double2) * (j + 1) * (AT / 32);
      for (int pass = 0; pass < 2; ++pass) {
        k_dots<<<grid, AT, red_smem, st>>>(n, nrhs, j, W.V, W.w, W.act, W.nchunks, W.part);
        CFIE_CHECK_LAUNCH();
        k_dots_reduce<<<nrhs, 128, 0, st>>>(nrhs, j, W.nchunks, m, j, pass == 0, W.act, W.part,
                                            W.hbuf, W.H);
        CFIE_CHECK_LAUNCH();
        k_update<<<grid, AT, sizeof(double2) * (j + 1), st>>>(
            n, nrhs, j, W.V, W.hbuf, W.act, W.w, W.nchunks, pass == 1 ? W.nrmp : nullptr);
        CFIE_CHECK_LAUNCH();
      }
      k_givens<<<blocks_for(nrhs, 64), 64, 0, st>>>(nrhs, m, j, W.nchunks, W.act, W.nrmp, W.H,
                                                     W.cs, W.sn, W.gv, W.hn, W.res);
      CFIE_CHECK_LAUNCH();
      k_scale<<<blocks_for(nv), 256, 0, st>>>(n, nrhs, W.act, W.hn, W.w, W.V + (size_t)(j + 1) * nv);
      CFIE_CHECK_LAUNCH();
    }
    CFIE_CHECK_CUDA(cudaMemcpyAsync(op->host_res, W.res, sizeof(double) * nrhs,
                                    cudaMemcpyDeviceToHost, st));
    CFIE_CHECK_CUDA(cudaStreamSynchronize(st));
    op->stats.arnoldi_steps++;
    bool changed = false;
    nact = 0;
    for (int k = 0; k < nrhs; ++k) {
      if (!act[k]) continue;
      kd[k] = j + 1;
      its[k]++;
      steps_left[k]--;
      if (op->host_res[k] <= tol[k] || steps_left[k] <= 0) {
        act[k] = 0;
        changed = true;
      } else {
        nact++;
      }
    }
    if (!nact) break;
    if (changed)
      CFIE_CHECK_CUDA(cudaMemcpyAsync(W.act, act.data(), sizeof(int) * nrhs,
                                      cudaMemcpyHostToDevice, st));
  }
  CFIE_CHECK_CUDA(cudaMemcpyAsync(W.kd, kd.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, st));
  k_lsq<<<blocks_for(nrhs, 64), 64, 0, st>>>(nrhs, m, W.kd, W.H, W.gv, W.y);
  CFIE_CHECK_LAUNCH();
  k_xupdate<<<blocks_for(nv), 256, 0, st>>>(n, nrhs, m, W.kd, W.V, W.y, x);
  CFIE_CHECK_LAUNCH();
  // the temporaries copied from host must stay alive until the copies ran
  CFIE_CHECK_CUDA(cudaStreamSynchronize(st));
}

void fp64_mv(cfie_op* op, const double2* x, double2* y, int nrhs) {
  op->stats.fp64_matvecs++;
  matvec_fp64(op, x, y, nrhs);
}
void inner_mv(cfie_op* op, const double2* x, double2* y, int nrhs) {
  op->stats.inner_matvecs++;
  apply_inner(op, x, y, nrhs);
}

}  // namespace

void gmres_solve(cfie_op* op, const double2* f, double2* x, int nrhs, double rtol, int restart,
                 int maxit, int* iters, double* relres, cfie_status* status) {
  op->stats = cfie_solve_stats{};
  const int n = op->n;
  const size_t nv = (size_t)n * nrhs;
  int m = restart > 0 ? restart : maxit;
  m = std::max(1, std::min(m, std::min(maxit, MAXJ)));
  ws W = workspace(op, nrhs, m);
  cudaStream_t st = op->ctx->stream;
  op->rv.reserve(sizeof(double2) * nv);
  double2* r = op->rv.as<double2>();
  double2* ax = W.w;  // matvec output scratch (free between cycles)

  std::vector<double> rn, fn, xn, dummy;
  std::vector<int> its(nrhs, 0), steps_left(nrhs, maxit), active(nrhs, 1);
  // true residual of the initial guess (no matvec when x0 = 0)
  residual_norms(op, W, x, nullptr, nullptr, nrhs, xn, dummy);
  bool x_zero = true;
  for (int k = 0; k < nrhs; ++k) x_zero = x_zero && xn[k] == 0.0;
  if (x_zero) {
    residual_norms(op, W, f, nullptr, r, nrhs, rn, fn);
  } else {
    fp64_mv(op, x, ax, nrhs);
    residual_norms(op, W, f, ax, r, nrhs, rn, fn);
  }

  const bool refined = op->prec != CFIE_FP64;
  if (!refined) {
    for (;;) {
      std::vector<double> tol(nrhs);
      int nact = 0;
      for (int k = 0; k < nrhs; ++k) {
        tol[k] = rtol * fn[k];
        active[k] = (rn[k] > tol[k] && steps_left[k] > 0) ? 1 : 0;
        nact += active[k];
      }
      if (!nact) break;
      gmres_cycle(op, W, fp64_mv, r, rn, tol, active, nrhs, m, steps_left, x, its);
      fp64_mv(op, x, ax, nrhs);
      residual_norms(op, W, f, ax, r, nrhs, rn, fn);
    }
  } else {
    // mixed-precision iterative refinement: inner GMRES on A d = r with the
    // operator's fast matvec, x += d, r = f - A64 x (FP64)
    op->dv.reserve(sizeof(double2) * nv);
    op->rin.reserve(sizeof(double2) * nv);
    double2* d = op->dv.as<double2>();
    double2* rin = op->rin.as<double2>();
    const double tau_min = 1e-4;
    for (int outer = 0; outer < 12; ++outer) {
      std::vector<double> tol(nrhs);
      int nact = 0;
      for (int k = 0; k < nrhs; ++k) {
        active[k] = (rn[k] > rtol * fn[k] && steps_left[k] > 0) ? 1 : 0;
        nact += active[k];
        double tau = rn[k] > 0 ? 0.3 * rtol * fn[k] / rn[k] : 1.0;
        tau = std::min(0.5, std::max(tau_min, tau));
        tol[k] = tau * rn[k];
      }
      if (!nact) break;
      op->stats.refinements++;
      k_zero<<<blocks_for(nv), 256, 0, st>>>(nv, d);
      CFIE_CHECK_LAUNCH();
      // inner restarted GMRES on A32 d = r
      std::vector<double> irn = rn, ifn;
      std::vector<int> iact = active;
      CFIE_CHECK_CUDA(cudaMemcpyAsync(rin, r, sizeof(double2) * nv, cudaMemcpyDeviceToDevice, st));
      for (int cyc = 0; cyc < 64; ++cyc) {
        gmres_cycle(op, W, inner_mv, rin, irn, tol, iact, nrhs, m, steps_left, d, its);
        // inner true residual r - A32 d
        inner_mv(op, d, ax, nrhs);
        residual_norms(op, W, r, ax, rin, nrhs, irn, ifn);
        int left = 0;
        for (int k = 0; k < nrhs; ++k) {
          iact[k] = active[k] && irn[k] > tol[k] && steps_left[k] > 0 ? 1 : 0;
          left += iact[k];
        }
        if (!left) break;
      }
      k_axpy<<<blocks_for(nv), 256, 0, st>>>(nv, d, x);
      CFIE_CHECK_LAUNCH();
      fp64_mv(op, x, ax, nrhs);
      residual_norms(op, W, f, ax, r, nrhs, rn, fn);
    }
  }
  *status = CFIE_OK;
  for (int k = 0; k < nrhs; ++k) {
    double rel = fn[k] > 0 ? rn[k] / fn[k] : 0.0;
    if (relres) relres[k] = rel;
    if (iters) iters[k] = its[k];
    if (!(rel <= rtol)) *status = CFIE_ENOCONV;
  }
}
