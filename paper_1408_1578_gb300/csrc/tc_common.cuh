// Shared pieces of the tensor-core kernels (stored-matrix contraction and the
// fused matrix-free contraction): inline-PTX wrappers for mbarriers, TMA,
// tcgen05 (TMEM allocation, MMA, commit, loads), shared-memory matrix and
// instruction descriptors, tensor-map encoding, the stream-K work split, and
// the preparation of the right-hand-side operand planes.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace {

constexpr long long kTimeoutCycles = 4000000000LL;  // ~2 s at 2 GHz

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

// try_wait may suspend the waiting thread until the phase completes or this
// many nanoseconds pass, instead of returning at once: waiting roles then stop
// taking issue slots from the warps that do the work
constexpr uint32_t kSuspendNs = 1000000;

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
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

// untiled bulk copy global -> shared, completing on an mbarrier: both
// addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// L2 policies for streamed operands (read once: evict first) and reused ones
// (evict last)
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// tiled 2-D TMA load with an L2 cache policy
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, uint64_t* bar,
                                                 int c0, int c1, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "l"(policy)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d_hint(void* dst, const CUtensorMap* map, uint64_t* bar,
                                                 int c0, int c1, int c2, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%3, %4, %5}], [%2], %6;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2),
      "l"(policy)
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

// 16 registers per thread into 32 TMEM lanes x 16 consecutive 32-bit columns
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 32 TMEM lanes x 8 consecutive 32-bit columns into 8 registers per thread
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
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
// 64-byte-swizzle variant (rows of 64 bytes, 8-row groups 512 bytes apart)
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;                      // 64-byte swizzle
  return d;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}


// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
using encode_fn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                               const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                               const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                               CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline encode_fn get_encode() {
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

// bf16 matrix of `rows` x `cols` (row pitch `pitch` elements), box box_rows x box_k
inline CUtensorMap tc_make_map(void* base, uint64_t rows, uint64_t cols, uint64_t pitch,
                               uint32_t box_rows, uint32_t box_k, CUtensorMapSwizzle swz) {
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {pitch * 2};
  const cuuint32_t box[2] = {box_k, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = get_encode()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw cfie_error(CFIE_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

// bf16 tiles stored one after another, each `rows` x `cols` row-major
// (`cols` x 2 bytes a multiple of 16), `count` of them; box = one whole tile
inline CUtensorMap tc_make_tile_map(void* base, uint64_t rows, uint64_t cols, uint64_t count,
                                    CUtensorMapSwizzle swz) {
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const cuuint64_t dims[3] = {cols, rows, count};
  const cuuint64_t strides[2] = {cols * 2, rows * cols * 2};
  const cuuint32_t box[3] = {(cuuint32_t)cols, (cuuint32_t)rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = get_encode()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw cfie_error(CFIE_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

// Stream-K split of mtiles x ktiles (row tile, source tile) pairs over `grid`
// CTAs: segments (job 0, m, k0, k1) in CTA order, cbeg[c] = first segment of
// CTA c, mt_seg[m] = (first segment, count) of row tile m.
inline void streamk_segments(int mtiles, int ktiles, int grid_max, std::vector<int4>& segs,
                             std::vector<int>& cbeg, std::vector<int2>& mt_seg) {
  const long long W = (long long)mtiles * ktiles;
  const int grid = (int)std::min<long long>(grid_max, std::max<long long>(1, W));
  segs.clear();
  cbeg.assign(grid + 1, 0);
  mt_seg.assign(mtiles, make_int2(0, 0));
  for (int c = 0; c < grid; ++c) {
    const long long b = W * c / grid, e = W * (c + 1) / grid;
    cbeg[c] = (int)segs.size();
    for (long long t = b; t < e;) {
      const int m = (int)(t / ktiles), k0 = (int)(t % ktiles);
      const int k1 = (int)std::min<long long>(ktiles, k0 + (e - t));
      if (mt_seg[m].y == 0) mt_seg[m].x = (int)segs.size();
      mt_seg[m].y++;
      segs.push_back(make_int4(0, m, k0, k1));
      t += k1 - k0;
    }
  }
  cbeg[grid] = (int)segs.size();
}

// B operand planes [4][NP][pitch] for nr right-hand sides (complex128, [r][j]):
// B1 = [Xr | Xi], B2 = [-Xi | Xr] (rows = output columns), hi / lo bf16 split
// (of the FP32-rounded value, in FP32).  One thread per right-hand side r and
// source pair j, j + 1: x read once, packed bf16 pairs stored.
__global__ void k_prep_b_planes(int n, int pitch, int NP, int nr, const double2* __restrict__ x,
                                __nv_bfloat16* __restrict__ bt) {
  const int r = blockIdx.y;                       // < NP / 2
  const int j = 2 * (blockIdx.x * 256 + threadIdx.x);
  if (j >= pitch) return;
  const int NR = NP / 2;
  float re[2] = {0.f, 0.f}, im[2] = {0.f, 0.f};
  if (r < nr) {
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (j + u < n) {
        const double2 v = x[(size_t)r * n + j + u];
        re[u] = (float)v.x;
        im[u] = (float)v.y;
      }
  }
  const __nv_bfloat162 hr = __floats2bfloat162_rn(re[0], re[1]);
  const __nv_bfloat162 lr =
      __floats2bfloat162_rn(re[0] - __low2float(hr), re[1] - __high2float(hr));
  const __nv_bfloat162 hi = __floats2bfloat162_rn(im[0], im[1]);
  const __nv_bfloat162 li =
      __floats2bfloat162_rn(im[0] - __low2float(hi), im[1] - __high2float(hi));
  const size_t plane = (size_t)NP * pitch;
  __nv_bfloat162* b = reinterpret_cast<__nv_bfloat162*>(bt);
  const size_t e0 = ((size_t)r * pitch + j) / 2, e1 = ((size_t)(NR + r) * pitch + j) / 2;
  const size_t p2 = plane / 2;
  // row r: B1 = Xr, B2 = -Xi;  row NR + r: B1 = Xi, B2 = Xr
  b[e0] = hr;
  b[p2 + e0] = lr;
  b[2 * p2 + e0] = __hneg2(hi);
  b[3 * p2 + e0] = __hneg2(li);
  b[e1] = hi;
  b[p2 + e1] = li;
  b[2 * p2 + e1] = hr;
  b[3 * p2 + e1] = lr;
}

inline void prep_b_planes(cfie_ctx* ctx, int n, int pitch, int NP, int nr, const double2* x,
                          __nv_bfloat16* bt) {
  k_prep_b_planes<<<dim3((unsigned)((pitch / 2 + 255) / 256), NP / 2), 256, 0, ctx->stream>>>(
      n, pitch, NP, nr, x, bt);
  CFIE_CHECK_LAUNCH();
}

}  // namespace
