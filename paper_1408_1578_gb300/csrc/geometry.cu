// Geometry sampling, Kress weight tables, diagonal limits and plane-wave data.
//
// Section 1 of the paper: Nystrom discretisation of the CFIE on a smooth
// boundary; Section 2: n equispaced boundary points.  The quadrature is Kress's
// logarithmic-split trapezoidal rule on the parameter nodes t_j = 2 pi j / n:
// an entry of the discrete operator is R_{(i-j) mod n} K1_ij + h K2_ij, with
// K = K1 ln(4 sin^2((t-tau)/2)) + K2.  For i != j this is h K_ij + w_d K1_ij with
// the table w_d = R_d - h ln(4 sin^2(pi d / n)), which is what the matvec
// kernels read.
#include <cmath>

#include "internal.h"

namespace {

struct curve_params {
  int kind;
  int K;
  double p0, p1;
  double a[64], b[64];
};

// One thread per node: z, z', z'' from the closed-form parametrisation, then the
// per-node quantities the kernels need.
__global__ void k_sample(curve_params P, int n, const double* __restrict__ zs,
                         const double* __restrict__ dzs, const double* __restrict__ ddzs,
                         geom_dev g) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s, c;
  sincospi(2.0 * j / n, &s, &c);  // t_j = 2 pi j / n
  double z1, z2, d1, d2, e1, e2;   // z, z', z''
  switch (P.kind) {
    case G_CIRCLE:
      z1 = P.p0 * c; z2 = P.p0 * s;
      d1 = -P.p0 * s; d2 = P.p0 * c;
      e1 = -P.p0 * c; e2 = -P.p0 * s;
      break;
    case G_ELLIPSE:
      z1 = P.p0 * c; z2 = P.p1 * s;
      d1 = -P.p0 * s; d2 = P.p1 * c;
      e1 = -P.p0 * c; e2 = -P.p1 * s;
      break;
    case G_STAR: {
      double r = 1.0, dr = 0.0, ddr = 0.0;
      for (int k = 1; k <= P.K; ++k) {
        double sk, ck;
        long long kj = ((long long)k * j) % n;    // exact reduction of k t_j
        sincospi(2.0 * (double)kj / n, &sk, &ck);
        double a = P.a[k - 1], b = P.b[k - 1];
        r += a * ck + b * sk;
        dr += k * (-a * sk + b * ck);
        ddr += -(double)k * k * (a * ck + b * sk);
      }
      z1 = r * c; z2 = r * s;
      d1 = dr * c - r * s; d2 = dr * s + r * c;
      e1 = ddr * c - 2.0 * dr * s - r * c;
      e2 = ddr * s + 2.0 * dr * c - r * s;
      break;
    }
    case G_KITE: {
      double s2, c2;
      long long j2 = (2LL * j) % n;
      sincospi(2.0 * (double)j2 / n, &s2, &c2);
      z1 = c + 0.65 * c2 - 0.65; z2 = 1.5 * s;
      d1 = -s - 1.3 * s2; d2 = 1.5 * c;
      e1 = -c - 2.6 * c2; e2 = -1.5 * s;
      break;
    }
    default:  // caller samples
      z1 = zs[2 * j]; z2 = zs[2 * j + 1];
      d1 = dzs[2 * j]; d2 = dzs[2 * j + 1];
      e1 = ddzs[2 * j]; e2 = ddzs[2 * j + 1];
      break;
  }
  double sp = sqrt(d1 * d1 + d2 * d2);
  g.x[j] = z1;
  g.y[j] = z2;
  g.nx[j] = d2;
  g.ny[j] = -d1;
  g.sp[j] = sp;
  g.kap[j] = (d2 * e1 - d1 * e2) / (4.0 * CFIE_PI * sp * sp);
}

// cos(2 pi k / n) and 1/m tables for the weight sums
__global__ void k_tables(int n, double* __restrict__ cosk, double* __restrict__ invm) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  cosk[k] = cospi(2.0 * k / n);
  invm[k] = k ? 1.0 / k : 0.0;
}

// R_d = -(4 pi / n) sum_{m=1}^{n/2-1} cos(2 pi m d / n) / m - (4 pi / n^2) (-1)^d,
// one block per d in [0, n/2]; the index (m d) mod n is stepped exactly.
__global__ void k_kress(int n, const double* __restrict__ cosk, const double* __restrict__ invm,
                        double* __restrict__ R) {
  int d = blockIdx.x;
  int N = n / 2;
  double acc = 0.0;
  long long idx = ((long long)(threadIdx.x + 1) * d) % n;
  long long step = ((long long)blockDim.x * d) % n;
  for (int m = threadIdx.x + 1; m < N; m += blockDim.x) {
    acc += cosk[idx] * invm[m];
    idx += step;
    if (idx >= n) idx -= n;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      double sgn = (d & 1) ? -1.0 : 1.0;
      R[d] = -(4.0 * CFIE_PI / n) * v - (4.0 * CFIE_PI / ((double)n * n)) * sgn;
    }
  }
}

// w_d for all d (R_d = R_{n-d}); spectral-derivative circulant c_d; diagonal entries.
__global__ void k_finish(int n, double omega, double eta, int bc, const double* __restrict__ R,
                         double* __restrict__ w, double* __restrict__ ct, geom_dev g,
                         double2* __restrict__ diag) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= n) return;
  double h = 2.0 * CFIE_PI / n;
  int dd = d <= n / 2 ? d : n - d;
  double Rd = R[dd];
  if (d == 0) {
    w[0] = Rd;
    ct[0] = 0.0;
  } else {
    double sn, cs;
    sincospi((double)d / n, &sn, &cs);
    w[d] = Rd - h * log(4.0 * sn * sn);
    ct[d] = 0.5 * ((d & 1) ? -1.0 : 1.0) * cs / sn;
  }
  // diagonal limits (node i = d)
  int i = d;
  double s = g.sp[i];
  double lg = CFIE_EULER + log(omega * s / 2.0);
  double R0 = R[0];
  if (bc == CFIE_SOUND_SOFT) {
    // A_ii = 1/2 + R_0 K1_ii + h K2_ii,  K = L - i eta M
    double re = 0.5 + h * g.kap[i] + h * eta * s / 4.0;
    double im = R0 * eta * s / (4.0 * CFIE_PI) + h * eta * s * lg / (2.0 * CFIE_PI);
    diag[i] = make_double2(re, im);
  } else {
    // S_ii = R_0 M1_ii + h M2_ii,  D'_ii = h L2_ii
    double sre = -R0 * s / (4.0 * CFIE_PI) - h * s * lg / (2.0 * CFIE_PI);
    double sim = h * s / 4.0;
    diag[2 * i] = make_double2(sre, sim);
    diag[2 * i + 1] = make_double2(h * g.kap[i], 0.0);
  }
}

__global__ void k_plane_waves(int n, int nrhs, double omega, int bc,
                              const double* __restrict__ theta, geom_dev g,
                              double2* __restrict__ f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int k = blockIdx.y;
  if (i >= n || k >= nrhs) return;
  double st, ct;
  sincos(theta[k], &st, &ct);
  double ph = omega * (ct * g.x[i] + st * g.y[i]);
  double sp, cp;
  sincos(ph, &sp, &cp);
  double2 v;
  if (bc == CFIE_SOUND_SOFT) {
    v = make_double2(-cp, -sp);                       // -exp(i ph)
  } else {
    double dn = (ct * g.nx[i] + st * g.ny[i]) / g.sp[i];
    v = make_double2(omega * dn * sp, -omega * dn * cp);  // -i omega dn exp(i ph)
  }
  f[(size_t)k * n + i] = v;
}

}  // namespace

void geometry_sample(cfie_op* op, const cfie_geom* geom) {
  int n = op->n;
  op->geo.reserve(sizeof(double) * 6 * n);
  double* base = op->geo.as<double>();
  op->g = geom_dev{base, base + n, base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n};
  curve_params P{};
  P.kind = geom->kind;
  P.p0 = geom->p0;
  P.p1 = geom->p1;
  P.K = (int)geom->a.size();
  for (int k = 0; k < P.K; ++k) {
    P.a[k] = geom->a[k];
    P.b[k] = geom->b[k];
  }
  dbuf samp;
  const double *zs = nullptr, *dzs = nullptr, *ddzs = nullptr;
  if (geom->kind == G_SAMPLES) {
    samp.reserve(sizeof(double) * 6 * n);
    double* s = samp.as<double>();
    cudaStream_t st = op->ctx->stream;
    CFIE_CHECK_CUDA(cudaMemcpyAsync(s, geom->z.data(), sizeof(double) * 2 * n,
                                    cudaMemcpyHostToDevice, st));
    CFIE_CHECK_CUDA(cudaMemcpyAsync(s + 2 * n, geom->dz.data(), sizeof(double) * 2 * n,
                                    cudaMemcpyHostToDevice, st));
    CFIE_CHECK_CUDA(cudaMemcpyAsync(s + 4 * n, geom->ddz.data(), sizeof(double) * 2 * n,
                                    cudaMemcpyHostToDevice, st));
    zs = s;
    dzs = s + 2 * n;
    ddzs = s + 4 * n;
  }
  k_sample<<<(n + 255) / 256, 256, 0, op->ctx->stream>>>(P, n, zs, dzs, ddzs, op->g);
  CFIE_CHECK_LAUNCH();
  if (samp.p) CFIE_CHECK_CUDA(cudaStreamSynchronize(op->ctx->stream));
}

void kress_tables(cfie_op* op) {
  int n = op->n;
  cudaStream_t st = op->ctx->stream;
  dbuf tmp;
  tmp.reserve(sizeof(double) * (3 * (size_t)n + 2));
  double* cosk = tmp.as<double>();
  double* invm = cosk + n;
  double* R = invm + n;
  op->wtab.reserve(sizeof(double) * n);
  op->ctab.reserve(sizeof(double) * n);
  op->diag.reserve(sizeof(double2) * 2 * (size_t)n);
  k_tables<<<(n + 255) / 256, 256, 0, st>>>(n, cosk, invm);
  CFIE_CHECK_LAUNCH();
  k_kress<<<n / 2 + 1, 256, 0, st>>>(n, cosk, invm, R);
  CFIE_CHECK_LAUNCH();
  k_finish<<<(n + 255) / 256, 256, 0, st>>>(n, op->omega, op->eta, op->bc, R,
                                             op->wtab.as<double>(), op->ctab.as<double>(), op->g,
                                             op->diag.as<double2>());
  CFIE_CHECK_LAUNCH();
  CFIE_CHECK_CUDA(cudaMemcpyAsync(&op->R0, R, sizeof(double), cudaMemcpyDeviceToHost, st));
  CFIE_CHECK_CUDA(cudaStreamSynchronize(st));
}

void rhs_plane_waves(cfie_op* op, int nrhs, const double* theta_host, double2* f) {
  dbuf th;
  th.reserve(sizeof(double) * nrhs);
  cudaStream_t st = op->ctx->stream;
  CFIE_CHECK_CUDA(cudaMemcpyAsync(th.p, theta_host, sizeof(double) * nrhs,
                                  cudaMemcpyHostToDevice, st));
  dim3 grid((op->n + 255) / 256, nrhs);
  k_plane_waves<<<grid, 256, 0, st>>>(op->n, nrhs, op->omega, op->bc, th.as<double>(), op->g, f);
  CFIE_CHECK_LAUNCH();
  CFIE_CHECK_CUDA(cudaStreamSynchronize(st));  // the angle buffer is freed on return
}
