// FP64 matrix-free Nystrom matvec (the plain FP64 comparison form) and the
// spectral tangential derivative used by Maue's identity.
//
// Operators (paper, Section 1): soft  A = 1/2 I + D - i eta S        (eq. 1)
//                               hard  A = 1/2 I - D' + N / (i eta)   (eq. 2)
// Per pair (i != j), r = |z_i - z_j|, x = omega r, s_j = |z'_j|, h = 2 pi / n,
// w = w_{(i-j) mod n} (Kress table):
//   soft:  A_ij = h K_ij + w K1_ij,  K = L - i eta M, K1 = L1 - i eta M1 with
//          L  = (i omega/4) H1(x) c,      L1 = -(omega/4pi) J1(x) c,  c = (z_i - z_j).nu~_j / r
//          M  = (i/4) H0(x) s_j,          M1 = -(1/4pi) J0(x) s_j
//   hard:  S_ij  = h M_ij + w M1_ij
//          D'_ij = h L'_ij + w L'1_ij with c' = (z_j - z_i).nu~_i / r * s_j / s_i
//          A x = 1/2 x - D' x + (1/(i eta)) [ (1/s) Dt S (1/s) Dt x
//                                            + omega^2 (n1 S (n1 x) + n2 S (n2 x)) ]
//          (Maue's identity; Dt = spectral derivative, Nyquist mode zeroed)
// Diagonal entries come precomputed (geometry.cu).
//
// Layout: a CTA owns TI = 64 targets and walks a contiguous range of source
// tiles (TJ = 32 sources each).  For every tile it evaluates the TI x TJ block
// of entries into shared memory (one warp per target row, lanes over sources),
// then contracts it with the staged block of up to 16 right-hand sides, each
// thread holding 4 right-hand sides of one target.  Source ranges are split
// across CTAs when the row tiles alone do not fill the GPU; the per-split
// partial sums go to a scratch buffer and a second kernel adds them in a fixed
// order (deterministic results) and applies the hard-path epilogue.
#include <algorithm>
#include <mutex>
#include <string>

#include <cuda.h>

#include "internal.h"
#include "hankel64.cuh"

namespace {

constexpr int TI = 64;
constexpr int TJ = 32;
constexpr int NT = 256;
constexpr int RB = 16;  // right-hand sides per launch slice (soft with many RHS: 64)

__device__ __forceinline__ double2 cmad(double2 acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}

template <int BC, int RBT = RB>
struct pair_smem {
  double tx[TI], ty[TI], tnx[TI], tny[TI], tsp[TI];
  double sx[TJ], sy[TJ], snx[TJ], sny[TJ], ssp[TJ];
  double2 A[TI][TJ + 1];
  double2 B[BC ? TI : 1][TJ + 1];        // hard: D' entries
  double2 X[BC ? 4 : 1][TJ][RBT];        // soft: x ; hard: u, n1 x, n2 x, x
};

template <int BC, int RBT = RB>
__global__ void __launch_bounds__(NT)
k_pair_fp64(int n, double omega, double eta, geom_dev g, const double* __restrict__ wtab,
            const double2* __restrict__ diag, const double2* __restrict__ xin,
            const double2* __restrict__ uin, int nrhs, int splits, int tiles_per_split,
            double2* __restrict__ part) {
  constexpr int RQ = RBT / (NT / TI);  // right-hand sides per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pair_smem<BC, RBT>& S = *reinterpret_cast<pair_smem<BC, RBT>*>(smem_raw);
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * TI;
  const int split = blockIdx.y;
  const int rb0 = blockIdx.z * RBT;
  const int rbn = min(RBT, nrhs - rb0);
  const int ntiles = (n + TJ - 1) / TJ;
  const int t_begin = split * tiles_per_split;
  const int t_end = min(ntiles, t_begin + tiles_per_split);
  const double h = 2.0 * CFIE_PI / n;

  if (tid < TI) {
    int i = i0 + tid;
    bool ok = i < n;
    S.tx[tid] = ok ? g.x[i] : 0.0;
    S.ty[tid] = ok ? g.y[i] : 0.0;
    S.tnx[tid] = ok ? g.nx[i] : 0.0;
    S.tny[tid] = ok ? g.ny[i] : 0.0;
    S.tsp[tid] = ok ? g.sp[i] : 1.0;
  }

  const int il2 = tid % TI;     // contraction: target row
  const int rg = tid / TI;      // contraction: right-hand-side group
  double2 acc[BC ? 4 : 1][RQ];
#pragma unroll
  for (int o = 0; o < (BC ? 4 : 1); ++o)
#pragma unroll
    for (int q = 0; q < RQ; ++q) acc[o][q] = make_double2(0.0, 0.0);

  for (int t = t_begin; t < t_end; ++t) {
    const int j0 = t * TJ;
    __syncthreads();
    if (tid < TJ) {
      int j = j0 + tid;
      bool ok = j < n;
      S.sx[tid] = ok ? g.x[j] : 0.0;
      S.sy[tid] = ok ? g.y[j] : 0.0;
      S.snx[tid] = ok ? g.nx[j] : 0.0;
      S.sny[tid] = ok ? g.ny[j] : 0.0;
      S.ssp[tid] = ok ? g.sp[j] : 1.0;
    }
    for (int e = tid; e < TJ * RBT; e += NT) {
      int jl = e / RBT, r = e % RBT;
      int j = j0 + jl;
      double2 xv = make_double2(0.0, 0.0), uv = xv;
      if (j < n && r < rbn) {
        xv = xin[(size_t)(rb0 + r) * n + j];
        if (BC) uv = uin[(size_t)(rb0 + r) * n + j];
      }
      if constexpr (BC == 1) {
        double inv = (j < n) ? 1.0 / g.sp[j] : 0.0;
        double n1 = (j < n) ? g.nx[j] * inv : 0.0;
        double n2 = (j < n) ? g.ny[j] * inv : 0.0;
        S.X[0][jl][r] = uv;
        S.X[1][jl][r] = make_double2(n1 * xv.x, n1 * xv.y);
        S.X[2][jl][r] = make_double2(n2 * xv.x, n2 * xv.y);
        S.X[3][jl][r] = xv;
      } else {
        S.X[0][jl][r] = xv;
      }
    }
    __syncthreads();

    // ---- entries of the TI x TJ block: warp w handles rows w, w+8, ...; lane = source
    for (int e = tid; e < TI * TJ; e += NT) {
      const int il = e / TJ, jl = e % TJ;
      const int i = i0 + il, j = j0 + jl;
      double2 a = make_double2(0.0, 0.0), b = a;
      if (i < n && j < n) {
        int d = i - j;
        if (d < 0) d += n;
        if (d == 0) {
          if (BC) {
            a = diag[2 * i];
            b = diag[2 * i + 1];
          } else {
            a = diag[i];
          }
        } else {
          pair_entries_fp64<BC>(S.tx[il] - S.sx[jl], S.ty[il] - S.sy[jl], omega, eta, h,
                                wtab[d], S.snx[jl], S.sny[jl], S.ssp[jl], S.tnx[il],
                                S.tny[il], S.tsp[il], a, b);
        }
      }
      S.A[il][jl] = a;
      if constexpr (BC == 1) S.B[il][jl] = b;
    }
    __syncthreads();

    // ---- contraction
    const int jn = min(TJ, n - j0);
    for (int jl = 0; jl < jn; ++jl) {
      const double2 a = S.A[il2][jl];
      if constexpr (BC == 0) {
#pragma unroll
        for (int q = 0; q < RQ; ++q) acc[0][q] = cmad(acc[0][q], a, S.X[0][jl][rg + 4 * q]);
      } else {
        const double2 b = S.B[il2][jl];
#pragma unroll
        for (int q = 0; q < RQ; ++q) {
          const int r = rg + 4 * q;
          acc[0][q] = cmad(acc[0][q], a, S.X[0][jl][r]);
          acc[1][q] = cmad(acc[1][q], a, S.X[1][jl][r]);
          acc[2][q] = cmad(acc[2][q], a, S.X[2][jl][r]);
          acc[3][q] = cmad(acc[3][q], b, S.X[3][jl][r]);
        }
      }
    }
  }

  const int i = i0 + il2;
  if (i < n) {
#pragma unroll
    for (int q = 0; q < RQ; ++q) {
      const int r = rg + 4 * q;
      if (r < rbn) {
#pragma unroll
        for (int o = 0; o < (BC ? 4 : 1); ++o)
          part[(((size_t)o * splits + split) * nrhs + rb0 + r) * n + i] = acc[o][q];
      }
    }
  }
}

// Sum split partials (fixed order).  Soft: y = sum.  Hard: t = S u,
// y = 1/2 x - D' x - i (omega^2 / eta) (n1 S(n1 x) + n2 S(n2 x)).
template <int BC>
__global__ void k_reduce_fp64(int n, int nrhs, int splits, double omega, double eta, geom_dev g,
                              const double2* __restrict__ part, const double2* __restrict__ x,
                              double2* __restrict__ t_out, double2* __restrict__ y) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)n * nrhs;
  if (e >= tot) return;
  const size_t stride_o = (size_t)splits * tot;
  double2 s[4] = {};
  for (int o = 0; o < (BC ? 4 : 1); ++o) {
    double2 v = make_double2(0.0, 0.0);
    for (int sp = 0; sp < splits; ++sp) {
      double2 p = part[o * stride_o + (size_t)sp * tot + e];
      v.x += p.x;
      v.y += p.y;
    }
    s[o] = v;
  }
  if (BC == 0) {
    y[e] = s[0];
  } else {
    int i = (int)(e % n);
    double inv = 1.0 / g.sp[i];
    double n1 = g.nx[i] * inv, n2 = g.ny[i] * inv;
    double2 m = make_double2(n1 * s[1].x + n2 * s[2].x, n1 * s[1].y + n2 * s[2].y);
    double k = omega * omega / eta;
    double2 xv = x[e];
    // -i k m = (k m.y, -k m.x)
    y[e] = make_double2(0.5 * xv.x - s[3].x + k * m.y, 0.5 * xv.y - s[3].y - k * m.x);
    t_out[e] = s[0];
  }
}

// out[k][i] = base[k][i] + (scale / s_i) sum_j c_{(i-j) mod n} in[k][j]
// (spectral derivative as a circulant; c_d = (-1)^d cot(pi d / n) / 2)
constexpr int SPT = 256;
__global__ void __launch_bounds__(SPT)
k_spectral_fp64(int n, const double* __restrict__ ct, const double* __restrict__ sp,
                const double2* __restrict__ in, const double2* __restrict__ base, double2 scale,
                double2* __restrict__ out) {
  __shared__ double2 xs[SPT];
  const int i = blockIdx.x * SPT + threadIdx.x;
  const int k = blockIdx.y;
  const double2* ink = in + (size_t)k * n;
  double2 acc = make_double2(0.0, 0.0);
  for (int j0 = 0; j0 < n; j0 += SPT) {
    __syncthreads();
    int jj = j0 + threadIdx.x;
    xs[threadIdx.x] = jj < n ? ink[jj] : make_double2(0.0, 0.0);
    __syncthreads();
    if (i < n) {
      int jn = min(SPT, n - j0);
      int idx = i - j0;
      if (idx < 0) idx += n;
      for (int q = 0; q < jn; ++q) {
        double c = ct[idx];
        acc.x = fma(c, xs[q].x, acc.x);
        acc.y = fma(c, xs[q].y, acc.y);
        idx = idx == 0 ? n - 1 : idx - 1;
      }
    }
  }
  if (i < n) {
    double inv = 1.0 / sp[i];
    double2 sc = make_double2(scale.x * inv, scale.y * inv);
    double2 v = make_double2(sc.x * acc.x - sc.y * acc.y, sc.x * acc.y + sc.y * acc.x);
    if (base) {
      double2 b = base[(size_t)k * n + i];
      v.x += b.x;
      v.y += b.y;
    }
    out[(size_t)k * n + i] = v;
  }
}

template <int BC, int RBT = RB>
void launch_pair(cfie_op* op, const double2* x, const double2* u, int nrhs, int splits, int tps,
                 double2* part) {
  const int n = op->n;
  size_t smem = sizeof(pair_smem<BC, RBT>);
  CFIE_CHECK_CUDA(cudaFuncSetAttribute(k_pair_fp64<BC, RBT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((n + TI - 1) / TI, splits, (nrhs + RBT - 1) / RBT);
  prof_scope ps(op->ctx, CFIE_K_MATVEC_FP64);
  k_pair_fp64<BC, RBT><<<grid, NT, smem, op->ctx->stream>>>(
      n, op->omega, op->eta, op->g, op->wtab.as<double>(), op->diag.as<double2>(), x, u, nrhs,
      splits, tps, part);
  CFIE_CHECK_LAUNCH();
}

}  // namespace

// out = base + scale (1/|z'|) d/dt in: by FFT (O(n log n) per column); the
// allocation-free variant below keeps the circulant kernel
void spectral_apply(cfie_op* op, const double2* in, double2* out, const double2* base,
                    double2 scale, int nrhs) {
  spectral_fft64(op, in, out, base, scale, nrhs);
}

void reduce_hard_fp64(cfie_op* op, const double2* part, int splits, const double2* x,
                      double2* t, double2* y, int nrhs) {
  const size_t tot = (size_t)op->n * nrhs;
  k_reduce_fp64<1><<<(unsigned)((tot + 255) / 256), 256, 0, op->ctx->stream>>>(
      op->n, nrhs, splits, op->omega, op->eta, op->g, part, x, t, y);
  CFIE_CHECK_LAUNCH();
}

void matvec_fp64(cfie_op* op, const double2* x, double2* y, int nrhs) {
  const int n = op->n;
  const int hard = op->bc == CFIE_SOUND_HARD;
  const int rowtiles = (n + TI - 1) / TI;
  const bool wide = !hard && nrhs > RB;  // one pass of pair evaluations for up to 64 RHS
  const int rb = wide ? 64 : RB;
  const int rhsblocks = (nrhs + rb - 1) / rb;
  const int ntiles = (n + TJ - 1) / TJ;
  int dev_sms = 152;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, op->ctx->device);
  const int target = 4 * dev_sms;
  int splits = std::max(1, std::min(ntiles, (target + rowtiles * rhsblocks - 1) /
                                                (rowtiles * rhsblocks)));
  int tps = (ntiles + splits - 1) / splits;
  splits = (ntiles + tps - 1) / tps;
  const int ops = hard ? 4 : 1;
  op->partial.reserve(sizeof(double2) * (size_t)ops * splits * nrhs * n);
  double2* part = op->partial.as<double2>();
  const size_t tot = (size_t)n * nrhs;
  if (!hard) {
    if (wide)
      launch_pair<0, 64>(op, x, nullptr, nrhs, splits, tps, part);
    else
      launch_pair<0>(op, x, nullptr, nrhs, splits, tps, part);
    k_reduce_fp64<0><<<(unsigned)((tot + 255) / 256), 256, 0, op->ctx->stream>>>(
        n, nrhs, splits, op->omega, op->eta, op->g, part, x, nullptr, y);
    CFIE_CHECK_LAUNCH();
    return;
  }
  op->tmp1.reserve(sizeof(double2) * tot);
  op->tmp2.reserve(sizeof(double2) * tot);
  double2* u = op->tmp1.as<double2>();
  double2* t = op->tmp2.as<double2>();
  // u = (1/s) Dt x
  spectral_apply(op, x, u, nullptr, make_double2(1.0, 0.0), nrhs);
  launch_pair<1>(op, x, u, nrhs, splits, tps, part);
  k_reduce_fp64<1><<<(unsigned)((tot + 255) / 256), 256, 0, op->ctx->stream>>>(
      n, nrhs, splits, op->omega, op->eta, op->g, part, x, t, y);
  CFIE_CHECK_LAUNCH();
  // y += (1/(i eta)) (1/s) Dt t
  spectral_apply(op, t, y, y, make_double2(0.0, -1.0 / op->eta), nrhs);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the FP64 matvec (cfie_apply_fp64_static).
//
// The split-source partial sums (and, for the sound-hard operator, the two
// derivative vectors) live in one file-scope device array instead of buffers
// the operator grows with cudaMalloc.  Every GPU that loads the library holds
// this array until the process exits.  Its device address is looked up once
// per device (cudaGetSymbolAddress, with that device current) on the first
// call there, and again if the device's context has been replaced since;
// host code never hands the array's name itself to a kernel.
// Each call overwrites every scratch element it later reads, so nothing has to
// start at zero; calls that overlap on the GPU share the array and race.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// The address is cached per device together with the device's current CUDA
// context: a context torn down and created again (cudaDeviceReset) reloads the
// module, so a cached address from the old context is looked up afresh.
using ctx_get_fn = CUresult (*)(CUcontext*);
ctx_get_fn driver_ctx_get_current() {
  static ctx_get_fn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<ctx_get_fn>(p);
  }();
  return fn;
}

std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};
CUcontext g_static_ctx[kMaxDevices] = {};

void* static_scratch_address(int device) {
  if (device < 0 || device >= kMaxDevices)
    throw cfie_error(CFIE_EINVAL, "device index out of range for the static scratch table");
  ctx_get_fn get = driver_ctx_get_current();
  CUcontext cur = nullptr;
  if (!get || get(&cur) != CUDA_SUCCESS || !cur)
    throw cfie_error(CFIE_ECUDA, "cuCtxGetCurrent: no current CUDA context for the static scratch");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[device] || g_static_ctx[device] != cur) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      throw cfie_error(CFIE_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") +
                                       cudaGetErrorString(e));
    g_static_addr[device] = p;
    g_static_ctx[device] = cur;
  }
  return g_static_addr[device];
}

}  // namespace

size_t static_scratch_capacity() { return kStaticScratchBytes; }

void matvec_fp64_static(cfie_op* op, const double2* x, double2* y, int nrhs) {
  const int n = op->n;
  const int hard = op->bc == CFIE_SOUND_HARD;
  const int ops = hard ? 4 : 1;
  const size_t tot = (size_t)n * nrhs;
  const size_t vec_bytes = sizeof(double2) * tot;
  const size_t fixed = hard ? 2 * vec_bytes : 0;          // u and t
  const size_t per_split = sizeof(double2) * (size_t)ops * tot;
  if (fixed + per_split > kStaticScratchBytes)
    throw cfie_error(CFIE_EINVAL,
                     "cfie_apply_fp64_static: n * nrhs too large for the 32 MiB static scratch "
                     "(needs " + std::to_string(fixed + per_split) + " bytes)");
  // device address of the array on the context's (current) device
  unsigned char* base = static_cast<unsigned char*>(static_scratch_address(op->ctx->device));

  const int rowtiles = (n + TI - 1) / TI;
  const int rhsblocks = (nrhs + RB - 1) / RB;
  const int ntiles = (n + TJ - 1) / TJ;
  int dev_sms = 152;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, op->ctx->device);
  const int target = 4 * dev_sms;
  int splits = std::max(1, std::min(ntiles, (target + rowtiles * rhsblocks - 1) /
                                                (rowtiles * rhsblocks)));
  const int fit = (int)std::min<size_t>((kStaticScratchBytes - fixed) / per_split, ntiles);
  splits = std::max(1, std::min(splits, fit));
  int tps = (ntiles + splits - 1) / splits;
  splits = (ntiles + tps - 1) / tps;

  double2* part = reinterpret_cast<double2*>(base + fixed);
  double2* u = hard ? reinterpret_cast<double2*>(base) : nullptr;
  double2* t = hard ? reinterpret_cast<double2*>(base + vec_bytes) : nullptr;
  cudaStream_t st = op->ctx->stream;
  const dim3 grid(rowtiles, splits, rhsblocks);
  const dim3 sgrid((n + SPT - 1) / SPT, nrhs);
  if (!hard) {
    const size_t smem = sizeof(pair_smem<0>);
    CFIE_CHECK_CUDA(cudaFuncSetAttribute(k_pair_fp64<0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_pair_fp64<0><<<grid, NT, smem, st>>>(n, op->omega, op->eta, op->g, op->wtab.as<double>(),
                                           op->diag.as<double2>(), x, nullptr, nrhs, splits, tps,
                                           part);
    CFIE_CHECK_LAUNCH();
    k_reduce_fp64<0><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
        n, nrhs, splits, op->omega, op->eta, op->g, part, x, nullptr, y);
    CFIE_CHECK_LAUNCH();
    return;
  }
  k_spectral_fp64<<<sgrid, SPT, 0, st>>>(n, op->ctab.as<double>(), op->g.sp, x, nullptr,
                                          make_double2(1.0, 0.0), u);
  CFIE_CHECK_LAUNCH();
  const size_t smem = sizeof(pair_smem<1>);
  CFIE_CHECK_CUDA(cudaFuncSetAttribute(k_pair_fp64<1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_pair_fp64<1><<<grid, NT, smem, st>>>(n, op->omega, op->eta, op->g, op->wtab.as<double>(),
                                         op->diag.as<double2>(), x, u, nrhs, splits, tps, part);
  CFIE_CHECK_LAUNCH();
  k_reduce_fp64<1><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
      n, nrhs, splits, op->omega, op->eta, op->g, part, x, t, y);
  CFIE_CHECK_LAUNCH();
  k_spectral_fp64<<<sgrid, SPT, 0, st>>>(n, op->ctab.as<double>(), op->g.sp, t, y,
                                          make_double2(0.0, -1.0 / op->eta), y);
  CFIE_CHECK_LAUNCH();
}
