// Stored-matrix path: the sound-soft Nystrom matrix A (eq. 1 of the paper,
// entries exactly as the FP32 fused matvec evaluates them, near band from FP64)
// is assembled once per operator and kept in HBM as four bf16 planes
//     A = (Ahi_re + Alo_re) + i (Ahi_im + Alo_im),   hi = bf16(a), lo = bf16(a - hi),
// 8 bytes per complex entry, i.e. the bytes of complex64 with ~16 significant
// bits per component.  Each block matvec Y = A X (up to 32 right-hand sides per
// pass) is a split-complex contraction on the 5th-generation tensor cores:
//
//     [Yr | Yi] = Ar [Xr | Xi] + Ai [-Xi | Xr]
//
// with every real product expanded as hi*hi + hi*lo + lo*hi (bf16 inputs, FP32
// accumulation in tensor memory).  Operand tiles are moved by TMA
// (cp.async.bulk.tensor, 128-byte swizzle, no multicast) into a two-stage
// shared-memory ring; one thread issues tcgen05.mma (M = 128, N = 2 * 32,
// K = 16 per instruction, kind::f16 with bf16 operands), tcgen05.commit frees
// the stage; after the last K tile the four warps read the 128 x N accumulator
// back with tcgen05.ld and write FP32 partial sums.  Source ranges are split
// across CTAs; a reduction kernel adds the partials in FP64 in a fixed order.
// Every mbarrier wait is bounded: on timeout the kernel records an error code,
// stops issuing work, drains its own copies (bounded), frees its tensor memory
// and returns.
//
// The path is HBM-bound: 8 bytes per entry per block matvec against
// 6 (products) x 4 x 2 flops x 32 right-hand sides.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"
#include "pair32.cuh"

namespace {

constexpr int BM = 128;     // rows (targets) per CTA tile = UMMA M
constexpr int BK = 64;      // sources per K tile (64 bf16 = one 128-byte swizzle row)
constexpr int STAGES = 2;
constexpr int NT = 128;     // 4 warps
constexpr long long kTimeoutCycles = 4000000000LL;  // ~2 s at 2 GHz

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on the phase of parity `parity`; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kTimeoutCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, both K-major
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 TMEM lanes x 16 consecutive 32-bit columns into 16 registers per thread
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Shared-memory matrix descriptor: K-major operand in 128-byte-swizzled rows,
// 8-row core groups 1024 bytes apart (SBO), descriptor version 1 (sm_100 family).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset
  d |= (uint64_t)1 << 46;                      // version
  d |= (uint64_t)2 << 61;                      // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int NP>
struct gemm_smem {
  __nv_bfloat16 A[STAGES][4][BM * BK];   // planes: hi_re, hi_im, lo_re, lo_im
  __nv_bfloat16 B[STAGES][4][NP * BK];   // planes: B1 hi, B1 lo, B2 hi, B2 lo
  uint64_t full[STAGES], empty[STAGES], done;
  uint32_t tmem_base;
  int abort;
  int issued[STAGES];                    // last issued phase parity per stage, -1 = none
};

template <int NP>
constexpr size_t gemm_smem_bytes() {
  return sizeof(gemm_smem<NP>) + 1024;   // + alignment slack for the 1024-byte swizzle atoms
}

// grid (m tiles, splits); NP = 2 * NR output columns (NR right-hand sides)
template <int NP>
__global__ void __launch_bounds__(NT, 1)
k_stored_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int n, int nr, int ktiles, int tiles_per_split, float2* __restrict__ part,
              int* __restrict__ err) {
  constexpr int NR = NP / 2;
  constexpr uint32_t TMEM_COLS = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);
  constexpr uint32_t STAGE_BYTES = 4u * BM * BK * 2u + 4u * NP * BK * 2u;
  extern __shared__ unsigned char raw[];
  gemm_smem<NP>& S = *reinterpret_cast<gemm_smem<NP>*>(
      (reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM;
  const int split = blockIdx.y;
  const int kt0 = split * tiles_per_split;
  const int kt1 = min(ktiles, kt0 + tiles_per_split);
  const int nk = kt1 - kt0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
      S.issued[s] = -1;
    }
    mbar_init(&S.done, 1);
    S.abort = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(&S.tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      if (it >= STAGES && !mbar_wait(&S.empty[s], ((it / STAGES) - 1) & 1)) {
        atomicExch(err, 1);
        S.abort = 1;
        break;
      }
      if (*(volatile int*)&S.abort) break;
      mbar_arrive_expect_tx(&S.full[s], STAGE_BYTES);
      S.issued[s] = (it / STAGES) & 1;
      const int kc = (kt0 + it) * BK;
#pragma unroll
      for (int p = 0; p < 4; ++p) tma_load_2d(S.A[s][p], &tmA, &S.full[s], kc, p * n + m0);
#pragma unroll
      for (int p = 0; p < 4; ++p) tma_load_2d(S.B[s][p], &tmB, &S.full[s], kc, p * NP);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    constexpr uint32_t idesc = make_idesc(BM, NP);
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES;
      if (!mbar_wait(&S.full[s], (it / STAGES) & 1)) {
        atomicExch(err, 2);
        S.abort = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(S.A[s][0]), a1 = smem_u32(S.A[s][1]);
      const uint32_t a2 = smem_u32(S.A[s][2]), a3 = smem_u32(S.A[s][3]);
      const uint32_t b0 = smem_u32(S.B[s][0]), b1 = smem_u32(S.B[s][1]);
      const uint32_t b2 = smem_u32(S.B[s][2]), b3 = smem_u32(S.B[s][3]);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint32_t off = kk * 32;   // 16 bf16 = 32 bytes along K inside the swizzle row
        const uint32_t acc0 = (it > 0 || kk > 0) ? 1u : 0u;
        umma_bf16(tmem, smem_desc(a0 + off), smem_desc(b0 + off), idesc, acc0);  // hr * B1 hi
        umma_bf16(tmem, smem_desc(a0 + off), smem_desc(b1 + off), idesc, 1u);    // hr * B1 lo
        umma_bf16(tmem, smem_desc(a2 + off), smem_desc(b0 + off), idesc, 1u);    // lr * B1 hi
        umma_bf16(tmem, smem_desc(a1 + off), smem_desc(b2 + off), idesc, 1u);    // hi * B2 hi
        umma_bf16(tmem, smem_desc(a1 + off), smem_desc(b3 + off), idesc, 1u);    // hi * B2 lo
        umma_bf16(tmem, smem_desc(a3 + off), smem_desc(b2 + off), idesc, 1u);    // li * B2 hi
      }
      umma_commit(&S.empty[s]);
    }
    umma_commit(&S.done);   // arrives once every MMA issued above has completed
  }

  // ---- epilogue: warp w owns TMEM lanes (rows) 32 w .. 32 w + 31
  __syncwarp();
  const bool ok = mbar_wait(&S.done, 0);
  if (!ok && lane == 0) {
    atomicExch(err, 3);
    S.abort = 1;
  }
  __syncwarp();
  tc_fence_after();
  float v[NP];
#pragma unroll
  for (int c0 = 0; c0 < NP; c0 += 16)
    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v + c0);
  const int i = m0 + 32 * warp + lane;
  if (ok && i < n && nk > 0) {
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nr) part[((size_t)split * nr + r) * n + i] = make_float2(v[r], v[NR + r]);
  }
  tc_fence_before();
  __syncthreads();
  // drain copies still in flight after an abort (bounded), then free TMEM
  if (threadIdx.x == 0 && *(volatile int*)&S.abort) {
    for (int s = 0; s < STAGES; ++s)
      if (S.issued[s] >= 0) mbar_wait(&S.full[s], (uint32_t)S.issued[s]);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// assembly and operand preparation
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// planes [4][n][pitch]: hi_re, hi_im, lo_re, lo_im; grid (ceil(pitch / 256), n)
__global__ void __launch_bounds__(256)
k_assemble(int n, int pitch, int b, omega32 W, geo32 g, const float* __restrict__ w32,
           const float2* __restrict__ band, __nv_bfloat16* __restrict__ planes) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * 256 + threadIdx.x;
  if (j >= pitch) return;
  float2 a = make_float2(0.f, 0.f), unused;
  if (j < n) {
    int d = i - j;
    if (d < 0) d += n;
    const int dd = d <= b ? d : (d >= n - b ? d - n : INT_MAX);
    if (dd != INT_MAX) {
      a = band[(size_t)i * (2 * b + 1) + dd + b];
    } else {
      pair_entries_fp32<0>(W, g.xh[i], g.xl[i], g.yh[i], g.yl[i], g.nx[i], g.ny[i], g.sp[i],
                           g.xh[j], g.xl[j], g.yh[j], g.yl[j], g.nx[j], g.ny[j], g.sp[j], w32[d],
                           a, unused);
    }
  }
  __nv_bfloat16 hr, lr, hi, li;
  split_bf16(a.x, hr, lr);
  split_bf16(a.y, hi, li);
  const size_t plane = (size_t)n * pitch;
  const size_t e = (size_t)i * pitch + j;
  planes[e] = hr;
  planes[plane + e] = hi;
  planes[2 * plane + e] = lr;
  planes[3 * plane + e] = li;
}

// B operand planes [4][NP][pitch] for right-hand sides r0 .. r0 + nr - 1:
// B1 = [Xr | Xi], B2 = [-Xi | Xr] (rows = output columns), hi / lo split.
__global__ void k_prep_b(int n, int pitch, int NP, int nr, const double2* __restrict__ x,
                         __nv_bfloat16* __restrict__ bt) {
  const int c = blockIdx.y;
  const int j = blockIdx.x * 256 + threadIdx.x;
  if (j >= pitch) return;
  const int NR = NP / 2;
  const int r = c < NR ? c : c - NR;
  double w1 = 0.0, w2 = 0.0;
  if (j < n && r < nr) {
    const double2 xv = x[(size_t)r * n + j];
    w1 = c < NR ? xv.x : xv.y;
    w2 = c < NR ? -xv.y : xv.x;
  }
  const __nv_bfloat16 h1 = __float2bfloat16_rn((float)w1), h2 = __float2bfloat16_rn((float)w2);
  const __nv_bfloat16 l1 = __float2bfloat16_rn((float)(w1 - (double)__bfloat162float(h1)));
  const __nv_bfloat16 l2 = __float2bfloat16_rn((float)(w2 - (double)__bfloat162float(h2)));
  const size_t plane = (size_t)NP * pitch;
  const size_t e = (size_t)c * pitch + j;
  bt[e] = h1;
  bt[plane + e] = l1;
  bt[2 * plane + e] = h2;
  bt[3 * plane + e] = l2;
}

// y[r0 + r][i] = sum over splits (fixed order, FP64)
__global__ void k_reduce_stored(int n, int nr, int splits, const float2* __restrict__ part,
                                double2* __restrict__ y) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t tot = (size_t)n * nr;
  if (e >= tot) return;
  double sx = 0.0, sy = 0.0;
  for (int s = 0; s < splits; ++s) {
    const float2 p = part[(size_t)s * tot + e];
    sx += p.x;
    sy += p.y;
  }
  y[e] = make_double2(sx, sy);
}

// ---------------------------------------------------------------------------
// host: tensor maps
// ---------------------------------------------------------------------------
using encode_fn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                               const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                               const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                               CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_fn get_encode() {
  static std::mutex mu;
  static encode_fn fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    CFIE_CHECK_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q));
    if (!p || q != cudaDriverEntryPointSuccess)
      throw cfie_error(CFIE_ECUDA, "cuTensorMapEncodeTiled is not available");
    fn = reinterpret_cast<encode_fn>(p);
  }
  return fn;
}

// bf16 matrix of `rows` x `cols` (row pitch `pitch` elements), box box_rows x 64
CUtensorMap make_map(void* base, uint64_t rows, uint64_t cols, uint64_t pitch, uint32_t box_rows) {
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {pitch * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = get_encode()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw cfie_error(CFIE_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

unsigned nblk(size_t len, int t = 256) { return (unsigned)((len + t - 1) / t); }

template <int NP>
void run_gemm(cfie_op* op, const CUtensorMap& ta, const CUtensorMap& tb, int nr, float2* part,
              int splits, int tps, int* err) {
  const size_t smem = gemm_smem_bytes<NP>();
  CFIE_CHECK_CUDA(cudaFuncSetAttribute(k_stored_gemm<NP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int n = op->n;
  const dim3 grid((n + BM - 1) / BM, splits);
  prof_scope ps(op->ctx, CFIE_K_MATVEC_TENSOR);
  k_stored_gemm<NP><<<grid, NT, smem, op->ctx->stream>>>(ta, tb, n, nr, (n + BK - 1) / BK, tps,
                                                         part, err);
  CFIE_CHECK_LAUNCH();
}

}  // namespace

int stored_pitch(int n) { return (n + 63) / 64 * 64; }

void stored_prepare(cfie_op* op) {
  if (op->bc != CFIE_SOUND_SOFT)
    throw cfie_error(CFIE_EINVAL, "the stored layout supports the sound-soft operator");
  const int n = op->n;
  const int pitch = stored_pitch(n);
  const size_t plane = (size_t)n * pitch;
  op->stored.reserve(sizeof(__nv_bfloat16) * 4 * plane);
  float* base = op->geo32.as<float>();
  omega32 W{};
  W.wh = (float)op->omega;
  W.wl = (float)(op->omega - (double)W.wh);
  W.winv = (float)(1.0 / op->omega);
  W.eta = (float)op->eta;
  W.h = (float)op->h;
  const dim3 grid(nblk(pitch), n);
  k_assemble<<<grid, 256, 0, op->ctx->stream>>>(n, pitch, op->band_b, W, geo32_at(base, n),
                                                base + 7 * n, op->band.as<float2>(),
                                                op->stored.as<__nv_bfloat16>());
  CFIE_CHECK_LAUNCH();
  op->err_flag.reserve(sizeof(int));
  CFIE_CHECK_CUDA(cudaMemsetAsync(op->err_flag.p, 0, sizeof(int), op->ctx->stream));
  CFIE_CHECK_CUDA(cudaStreamSynchronize(op->ctx->stream));
}

void matvec_stored(cfie_op* op, const double2* x, double2* y, int nrhs) {
  const int n = op->n;
  const int pitch = stored_pitch(n);
  cudaStream_t st = op->ctx->stream;
  constexpr int NP = 64;           // 32 right-hand sides per pass
  constexpr int NR = NP / 2;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, op->ctx->device);
  const int mtiles = (n + BM - 1) / BM;
  const int ktiles = (n + BK - 1) / BK;
  // source splits: fill the SMs (one CTA per SM), at least 4 K tiles each
  int splits = std::max(1, std::min((sms + mtiles - 1) / mtiles, std::max(1, ktiles / 4)));
  const int tps = (ktiles + splits - 1) / splits;
  splits = (ktiles + tps - 1) / tps;
  op->bt.reserve(sizeof(__nv_bfloat16) * 4 * (size_t)NP * pitch);
  op->partial.reserve(sizeof(float2) * (size_t)splits * NR * n);
  const CUtensorMap ta = make_map(op->stored.p, 4 * (uint64_t)n, (uint64_t)pitch, pitch, BM);
  const CUtensorMap tb = make_map(op->bt.p, 4 * (uint64_t)NP, (uint64_t)pitch, pitch, NP);
  int* err = op->err_flag.as<int>();
  for (int r0 = 0; r0 < nrhs; r0 += NR) {
    const int nr = std::min(NR, nrhs - r0);
    k_prep_b<<<dim3(nblk(pitch), NP), 256, 0, st>>>(n, pitch, NP, nr, x + (size_t)r0 * n,
                                                    op->bt.as<__nv_bfloat16>());
    CFIE_CHECK_LAUNCH();
    run_gemm<NP>(op, ta, tb, nr, op->partial.as<float2>(), splits, tps, err);
    k_reduce_stored<<<nblk((size_t)n * nr), 256, 0, st>>>(n, nr, splits, op->partial.as<float2>(),
                                                          y + (size_t)r0 * n);
    CFIE_CHECK_LAUNCH();
  }
}

// error code left by the bounded waits of the tensor-core kernel (0 = none);
// resets it.  Synchronises the stream.
int stored_take_error(cfie_op* op) {
  if (!op->err_flag.p) return 0;
  int e = 0;
  CFIE_CHECK_CUDA(cudaMemcpyAsync(&e, op->err_flag.p, sizeof(int), cudaMemcpyDeviceToHost,
                                  op->ctx->stream));
  CFIE_CHECK_CUDA(cudaStreamSynchronize(op->ctx->stream));
  if (e) CFIE_CHECK_CUDA(cudaMemsetAsync(op->err_flag.p, 0, sizeof(int), op->ctx->stream));
  return e;
}
