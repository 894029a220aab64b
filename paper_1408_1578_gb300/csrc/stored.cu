// Stored-matrix path: the sound-soft Nystrom matrix A (eq. 1 of the paper,
// entries exactly as the fused tensor-core matvec evaluates them, near band
// from FP64)
// is assembled once per operator and kept in HBM as four bf16 planes
//     A = (Ahi_re + Alo_re) + i (Ahi_im + Alo_im),   hi = bf16(a), lo = bf16(a - hi),
// 8 bytes per complex entry, i.e. the bytes of complex64 with ~16 significant
// bits per component.  Each plane is stored tile by tile: the 128 x 64 tiles
// (16 KB, row-major inside) of a 128-row block one after another along the
// sources, the blocks in row order, so that every TMA load of the contraction
// reads 16 contiguous kilobytes.  Each block matvec Y = A X (up to 32 right-hand sides per
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
// back with tcgen05.ld and write y (whole row tiles per CTA) or FP32 partial
// sums (source ranges split across CTAs, stream-K), which a reduction kernel
// adds in FP64 in a fixed order.
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
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "internal.h"
#include "pair32.cuh"
#include "tc_common.cuh"

namespace {

constexpr int BM = 128;     // rows (targets) per CTA tile = UMMA M
constexpr int BK = 64;      // sources per K tile (64 bf16 = one 128-byte swizzle row)
constexpr int STAGES = 2;
// K tiles accumulated in one tensor-memory accumulator before the epilogue adds
// it into its running sums: the tensor core's FP32 accumulation is not rounded
// to nearest and its error grows with the MMAs summed into one accumulator, so
// chunks of 256 sources keep it near 2e-6 for every n.
constexpr int SCK = 4;

// ---------------------------------------------------------------------------
// assembly and operand preparation
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// row maxima (float bits, in place) -> exponents E with max < 2^E (1e-4 margin
// for the FP32 evaluation), 0 for rows without far entries
__global__ void k_rowexp_from_max(int n, unsigned* __restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float m = __uint_as_float(r[i]);
  int e = 0;
  if (m > 0.f) frexpf(m * 1.0001f, &e);
  reinterpret_cast<int*>(r)[i] = e;
}

// planes [4][mt][kt][128][64] (mt = ceil(n / 128) row blocks, kt = pitch / 64
// source tiles): hi_re, hi_im, lo_re, lo_im; grid (ceil(pitch / 256), n); the
// rows of the last block past n are zeroed beforehand
__global__ void __launch_bounds__(256)
k_assemble(int n, int pitch, int b, int bd, const float4* __restrict__ pk,
           const float2* __restrict__ wkt, const float2* __restrict__ band,
           __nv_bfloat16* __restrict__ planes, unsigned* __restrict__ rmax) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * 256 + threadIdx.x;
  float2 a = make_float2(0.f, 0.f);
  float far_max = 0.f;
  if (j < n) {
    int d = i - j;
    if (d < 0) d += n;
    const int dd = d <= b ? d : (d >= n - b ? d - n : INT_MAX);
    if (dd != INT_MAX) {
      a = band[(size_t)i * (2 * b + 1) + dd + b];
    } else {
      // the folded entry of the fused matvec, to the accuracy the bf16 hi + lo
      // planes keep (packed coordinates and factors, Kress table / (pi h) at
      // i - j + n)
      a = entry_folded32<KIND_SOFT>(pk[i], make_float4(0.f, 0.f, 0.f, 0.f), pk[j], pk[n + j],
                                    wkt[i - j + n].x);
    }
    // largest far entry of the row (outside the double-float band of width bd):
    // the row exponent of the tensor-core residual
    if (rmax && d > bd && d < n - bd) far_max = fmaxf(fabsf(a.x), fabsf(a.y));
  }
  if (rmax) {
    for (int o = 16; o > 0; o >>= 1) far_max = fmaxf(far_max, __shfl_xor_sync(0xffffffffu, far_max, o));
    if ((threadIdx.x & 31) == 0 && far_max > 0.f) atomicMax(&rmax[i], __float_as_uint(far_max));
  }
  if (j >= pitch) return;
  __nv_bfloat16 hr, lr, hi, li;
  split_bf16(a.x, hr, lr);
  split_bf16(a.y, hi, li);
  const size_t plane = (size_t)((n + BM - 1) / BM) * BM * pitch;
  const size_t e = (((size_t)(i / BM) * (pitch / BK) + j / BK) * BM + i % BM) * BK + j % BK;
  planes[e] = hr;
  planes[plane + e] = hi;
  planes[2 * plane + e] = lr;
  planes[3 * plane + e] = li;
}

// One GEMM job: 32 right-hand sides of one stored operator.  64-byte aligned
// (it holds the two tensor maps the TMA unit reads).
struct alignas(64) gemm_job {
  CUtensorMap ta;          // A planes: 4 mt kt tiles of 128 x 64 bf16, box one tile
  CUtensorMap tb;          // B planes [4 NP rows][pitch] bf16, box NP x 64
  __nv_bfloat16* bt;       // B planes of this job
  long long xoff;          // first element of the job's right-hand sides in x / y
  int n, pitch, nr, mt0;   // size, row pitch, right-hand sides (<= 32), first global m tile
};

struct gemm_io {
  const double2* x;
  double2* y;
};

template <int NP>
struct pgemm_smem {
  __nv_bfloat16 A[STAGES][4][BM * BK];   // planes: hi_re, hi_im, lo_re, lo_im
  __nv_bfloat16 B[STAGES][4][NP * BK];   // planes: B1 hi, B1 lo, B2 hi, B2 lo
  uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2];
  uint64_t mdone;                        // completion of every MMA issued (abort path)
  uint32_t tmem_base;
  int abort;
  int issued[STAGES];                    // last issued phase parity per stage, -1 = none
};

template <int NP>
constexpr size_t pgemm_smem_bytes() {
  return sizeof(pgemm_smem<NP>) + 1024;  // + slack to align the 1024-byte swizzle atoms
}

// Persistent stream-K contraction over every job of a plan.  The (m tile,
// k tile) pairs of all jobs form one list; CTA c owns a contiguous range of it,
// cut into segments (one job, one m tile, a run of k tiles).  With io set
// (every m tile one whole segment) the epilogue writes y itself; otherwise it
// writes FP32 partial sums per segment for the reduction kernel.  Warp 0 issues the
// TMA loads, warp 1 the MMAs (double-buffered accumulators, 2 x NP TMEM
// columns), warps 2-5 drain finished accumulators to the partial-sum slot of
// their segment while the next segment accumulates.
template <int NP>
__global__ void __launch_bounds__(192, 1)
k_gemm_persistent(const gemm_job* __restrict__ jobs, const int4* __restrict__ segs,
                  const int* __restrict__ cbeg, float2* __restrict__ partial,
                  const gemm_io* __restrict__ io, int* __restrict__ err, int stall) {
  constexpr int NR = NP / 2;
  constexpr uint32_t TMEM_COLS = 2 * NP <= 32 ? 32 : (2 * NP <= 64 ? 64 : (2 * NP <= 128 ? 128 : 256));
  constexpr uint32_t STAGE_BYTES = 4u * BM * BK * 2u + 4u * NP * BK * 2u;
  extern __shared__ unsigned char raw[];
  pgemm_smem<NP>& S = *reinterpret_cast<pgemm_smem<NP>*>(
      (reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sb = cbeg[blockIdx.x], se = cbeg[blockIdx.x + 1];

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
      S.issued[s] = -1;
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.tfull[b], 1);
      mbar_init(&S.tempty[b], 4);   // one arrival per epilogue warp
    }
    mbar_init(&S.mdone, 1);
    S.abort = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&S.tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer: the matrix planes are streamed once per matvec
      // (evict first), the right-hand-side planes are reused by every row
      // tile of their job (evict last)
      const uint64_t pol_a = l2_evict_first(), pol_b = l2_evict_last();
      int it = 0;
      for (int s = sb; s < se && !*(volatile int*)&S.abort; ++s) {
        const int4 sg = segs[s];
        const gemm_job* J = jobs + sg.x;
        for (int k = sg.z; k < sg.w; ++k, ++it) {
          const int st = it % STAGES;
          if (it >= STAGES && !mbar_wait(&S.empty[st], ((it / STAGES) - 1) & 1)) {
            atomicExch(err, 1);
            S.abort = 1;
            break;
          }
          mbar_arrive_expect_tx(&S.full[st], STAGE_BYTES);
          S.issued[st] = (it / STAGES) & 1;
          // fault injection for the failure tests: the first stage's copies are
          // never issued, so the wait on its barrier runs out
          if (stall && it == 0) continue;
          const int kc = k * BK;
          const int kt = J->pitch / BK, mt = (J->n + BM - 1) / BM;
#pragma unroll
          for (int p = 0; p < 4; ++p)
            tma_load_3d_hint(S.A[st][p], &J->ta, &S.full[st], 0, 0, (p * mt + sg.y) * kt + k,
                             pol_a);
#pragma unroll
          for (int p = 0; p < 4; ++p)
            tma_load_2d_hint(S.B[st][p], &J->tb, &S.full[st], kc, p * NP, pol_b);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: one accumulator buffer per chunk of SCK source tiles
      constexpr uint32_t idesc = make_idesc(BM, NP);
      int it = 0, cc = 0;
      for (int s = sb; s < se && !*(volatile int*)&S.abort; ++s) {
        const int4 sg = segs[s];
        for (int c0 = sg.z; c0 < sg.w; c0 += SCK, ++cc) {
          const int c1 = min(sg.w, c0 + SCK);
          const int tb = cc & 1, use = cc >> 1;
          if (use >= 1 && !mbar_wait(&S.tempty[tb], (use - 1) & 1)) {
            atomicExch(err, 4);
            S.abort = 1;
          }
          if (*(volatile int*)&S.abort) break;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(tb * NP);
          for (int k = c0; k < c1; ++k, ++it) {
            const int st = it % STAGES;
            if (!mbar_wait(&S.full[st], (it / STAGES) & 1)) {
              atomicExch(err, 2);
              S.abort = 1;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(S.A[st][0]), a1 = smem_u32(S.A[st][1]);
            const uint32_t a2 = smem_u32(S.A[st][2]), a3 = smem_u32(S.A[st][3]);
            const uint32_t b0 = smem_u32(S.B[st][0]), b1 = smem_u32(S.B[st][1]);
            const uint32_t b2 = smem_u32(S.B[st][2]), b3 = smem_u32(S.B[st][3]);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t off = kk * 32;  // 16 bf16 along K inside the 128-byte swizzle row
              const uint32_t acc0 = (k > c0 || kk > 0) ? 1u : 0u;
              umma_bf16(d, smem_desc(a0 + off), smem_desc(b0 + off), idesc, acc0);  // hr * B1 hi
              umma_bf16(d, smem_desc(a0 + off), smem_desc(b1 + off), idesc, 1u);    // hr * B1 lo
              umma_bf16(d, smem_desc(a2 + off), smem_desc(b0 + off), idesc, 1u);    // lr * B1 hi
              umma_bf16(d, smem_desc(a1 + off), smem_desc(b2 + off), idesc, 1u);    // hi * B2 hi
              umma_bf16(d, smem_desc(a1 + off), smem_desc(b3 + off), idesc, 1u);    // hi * B2 lo
              umma_bf16(d, smem_desc(a3 + off), smem_desc(b2 + off), idesc, 1u);    // li * B2 hi
            }
            umma_commit(&S.empty[st]);
          }
          umma_commit(&S.tfull[tb]);  // arrives when this chunk's MMAs have completed
        }
      }
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, one row per
    // thread, running sums of the chunks of a segment in registers
    const int q = warp & 3;
    const int row = 32 * q + lane;
    int cc = 0;
    bool stop = false;
    for (int s = sb; s < se && !stop; ++s) {
      const int4 sg = segs[s];
      float run[NP];
      for (int c0 = sg.z; c0 < sg.w; c0 += SCK, ++cc) {
        const int tb = cc & 1, use = cc >> 1;
        if (*(volatile int*)&S.abort || !mbar_wait(&S.tfull[tb], use & 1)) {
          if (lane == 0) {
            atomicExch(err, 3);
            S.abort = 1;
          }
          stop = true;
          break;
        }
        __syncwarp();
        tc_fence_after();
        const bool first = c0 == sg.z;
#pragma unroll
        for (int cb = 0; cb < NP; cb += 16) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(tb * NP + cb), v);
#pragma unroll
          for (int r = 0; r < 16; ++r) run[cb + r] = first ? v[r] : run[cb + r] + v[r];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.tempty[tb]);
      }
      if (stop) break;
      if (io) {
        // every row tile is one segment (whole-tile dealings): the sums are
        // the product itself, written to y without a reduction pass
        const gemm_job* J = jobs + sg.x;
        const int i = sg.y * BM + row;
        if (i < J->n) {
          double2* y = io->y + J->xoff + i;
#pragma unroll
          for (int r = 0; r < NR; ++r)
            if (r < J->nr) y[(size_t)r * J->n] = make_double2(run[r], run[NR + r]);
        }
      } else {
        float2* dst = partial + (size_t)s * BM * NR + row;
#pragma unroll
        for (int r = 0; r < NR; ++r) dst[(size_t)r * BM] = make_float2(run[r], run[NR + r]);
      }
    }
  }
  __syncthreads();
  // after an abort, wait (bounded) for copies still in flight and for every
  // MMA the MMA thread issued (they may still read shared memory and write
  // tensor memory), then free TMEM
  if (*(volatile int*)&S.abort) {
    if (threadIdx.x == 0)
      for (int s = 0; s < STAGES; ++s)
        if (S.issued[s] >= 0) mbar_wait(&S.full[s], (uint32_t)S.issued[s]);
    if (warp == 1 && lane == 0) {
      umma_commit(&S.mdone);
      mbar_wait(&S.mdone, 0);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// B operand planes of every job: B1 = [Xr | Xi], B2 = [-Xi | Xr] (rows = output
// columns), hi / lo bf16 split; grid (NR, jobs): right-hand side r fills its
// columns r and NR + r from one read of x (the split of -Xi is the negated
// split of Xi), each CTA striding over the job's pitch
__global__ void k_prep_b_jobs(const gemm_job* __restrict__ jobs, const gemm_io* __restrict__ io,
                              int NP) {
  const gemm_job& J = jobs[blockIdx.y];
  const int r = blockIdx.x;
  const int NR = NP / 2;
  const size_t plane = (size_t)NP * J.pitch;
  for (int j = threadIdx.x; j < J.pitch; j += blockDim.x) {
    double2 xv = make_double2(0.0, 0.0);
    if (j < J.n && r < J.nr) xv = io->x[J.xoff + (long long)r * J.n + j];
    // the split of the FP32 value (x - hi is exact in FP32; FP64 arithmetic
    // here would run on the slow FP64 pipe)
    const float fr = (float)xv.x, fi = (float)xv.y;
    const __nv_bfloat16 hr = __float2bfloat16_rn(fr), hi = __float2bfloat16_rn(fi);
    const __nv_bfloat16 lr = __float2bfloat16_rn(fr - __bfloat162float(hr));
    const __nv_bfloat16 li = __float2bfloat16_rn(fi - __bfloat162float(hi));
    const size_t e = (size_t)r * J.pitch + j, f = (size_t)(NR + r) * J.pitch + j;
    J.bt[e] = hr;                      // column r: B1 = Xr, B2 = -Xi
    J.bt[plane + e] = lr;
    J.bt[2 * plane + e] = __hneg(hi);
    J.bt[3 * plane + e] = __hneg(li);
    J.bt[f] = hi;                      // column NR + r: B1 = Xi, B2 = Xr
    J.bt[plane + f] = li;
    J.bt[2 * plane + f] = hr;
    J.bt[3 * plane + f] = lr;
  }
}

// y = sum of the segment partials of each (job, m tile), fixed order, FP64;
// grid (global m tiles, NR), 128 threads (rows)
__global__ void k_reduce_jobs(const gemm_job* __restrict__ jobs, const int2* __restrict__ mt_job,
                              const int2* __restrict__ mt_seg, const float2* __restrict__ partial,
                              const gemm_io* __restrict__ io, int NR) {
  const int g = blockIdx.x, r = blockIdx.y, row = threadIdx.x;
  const int2 jm = mt_job[g];
  const gemm_job& J = jobs[jm.x];
  const int i = jm.y * BM + row;
  if (i >= J.n || r >= J.nr) return;
  const int2 sr = mt_seg[g];
  double sx = 0.0, sy = 0.0;
  for (int s = sr.x; s < sr.x + sr.y; ++s) {
    const float2 p = partial[((size_t)s * NR + r) * BM + row];
    sx += p.x;
    sy += p.y;
  }
  io->y[J.xoff + (long long)r * J.n + i] = make_double2(sx, sy);
}

// ---------------------------------------------------------------------------
// host: tensor maps, plans, graphs
// ---------------------------------------------------------------------------
// bf16 matrix of `rows` x `cols` (row pitch `pitch` elements), box box_rows x 64
CUtensorMap make_map(void* base, uint64_t rows, uint64_t cols, uint64_t pitch, uint32_t box_rows) {
  return tc_make_map(base, rows, cols, pitch, box_rows, BK, CU_TENSOR_MAP_SWIZZLE_128B);
}

unsigned nblk(size_t len, int t = 256) { return (unsigned)((len + t - 1) / t); }

constexpr int kNP = 64;            // 32 right-hand sides per job
constexpr int kNR = kNP / 2;

}  // namespace

int stored_pitch(int n) { return (n + 63) / 64 * 64; }

// Build the job list, the stream-K segment table and the CUDA graph
// (B preparation, persistent contraction, reduction) for the given operators
// and right-hand-side counts; x / y are read from the plan's io slot.
void gemm_plan_build(gemm_plan& G, cfie_ctx* ctx, const std::vector<cfie_op*>& ops,
                     const std::vector<int>& nrhs, const std::vector<long long>& xoff,
                     int dealing) {
  cudaStream_t st = ctx->stream;
  std::vector<gemm_job> jobs;
  std::vector<size_t> bt_off;
  size_t bt_total = 0;
  int mt_total = 0;
  for (size_t o = 0; o < ops.size(); ++o) {
    cfie_op* op = ops[o];
    if (op->layout != CFIE_STORED) throw cfie_error(CFIE_EINVAL, "operator is not stored");
    const int n = op->n, pitch = stored_pitch(n);
    for (int r0 = 0; r0 < nrhs[o]; r0 += kNR) {
      gemm_job J;
      std::memset(&J, 0, sizeof(J));
      J.n = n;
      J.pitch = pitch;
      J.nr = std::min(kNR, nrhs[o] - r0);
      J.xoff = xoff[o] + (long long)r0 * n;
      J.mt0 = mt_total;
      mt_total += (n + BM - 1) / BM;
      bt_off.push_back(bt_total);
      bt_total += (size_t)4 * kNP * pitch;
      jobs.push_back(J);
    }
  }
  G.bt.reserve(sizeof(__nv_bfloat16) * bt_total);
  for (size_t k = 0, o = 0; o < ops.size(); ++o) {
    cfie_op* op = ops[o];
    for (int r0 = 0; r0 < nrhs[o]; r0 += kNR, ++k) {
      gemm_job& J = jobs[k];
      J.bt = G.bt.as<__nv_bfloat16>() + bt_off[k];
      J.ta = tc_make_tile_map(op->stored.p, BM, BK,
                              4 * (uint64_t)((J.n + BM - 1) / BM) * (J.pitch / BK),
                              CU_TENSOR_MAP_SWIZZLE_128B);
      J.tb = make_map(J.bt, 4 * (uint64_t)kNP, (uint64_t)J.pitch, J.pitch, kNP);
    }
  }
  // One CTA per SM.  How the (job, row tile, K tile) work is dealt to them:
  //  GEMM_DEAL_AUTO        stream-K with few row tiles, round-robin with many
  //  GEMM_DEAL_ROUND_ROBIN whole (job, row tile) units, unit u to CTA u % grid:
  //                        the CTAs work on neighbouring units of few jobs at any
  //                        time, so the jobs' right-hand-side planes stay in L2
  //  GEMM_DEAL_GREEDY      whole units in job order, each to the CTA with the
  //                        least work so far: balanced within one unit when
  //                        sizes differ (round-robin is not), and the CTAs,
  //                        progressing evenly, still work on neighbouring units
  //  GEMM_DEAL_STREAMK     the (row tile, K tile) pairs split evenly, segments
  //                        cut at row-tile boundaries (partial sums added by the
  //                        reduction kernel)
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  long long W = 0;
  std::vector<long long> job_base(jobs.size() + 1, 0);
  for (size_t k = 0; k < jobs.size(); ++k) {
    const long long mt = (jobs[k].n + BM - 1) / BM, kt = (jobs[k].n + BK - 1) / BK;
    job_base[k + 1] = job_base[k] + mt * kt;
  }
  W = job_base.back();
  const int grid = (int)std::min<long long>(sms, std::max<long long>(1, W));
  std::vector<int4> segs;
  std::vector<int> cbeg(grid + 1, 0);
  std::vector<int2> mt_job(mt_total), mt_seg(mt_total, make_int2(0, 0));
  size_t jk = 0;
  if (dealing == GEMM_DEAL_AUTO)
    dealing = mt_total >= 4 * grid ? GEMM_DEAL_ROUND_ROBIN : GEMM_DEAL_STREAMK;
  G.dealing = dealing;
  if (dealing == GEMM_DEAL_ROUND_ROBIN || dealing == GEMM_DEAL_GREEDY) {
    std::vector<std::vector<int4>> per(grid);
    if (dealing == GEMM_DEAL_ROUND_ROBIN) {
      int u = 0;
      for (size_t k = 0; k < jobs.size(); ++k) {
        const int mt = (jobs[k].n + BM - 1) / BM, kt = (jobs[k].n + BK - 1) / BK;
        for (int m = 0; m < mt; ++m, ++u) per[u % grid].push_back(make_int4((int)k, m, 0, kt));
      }
    } else {
      std::vector<long long> load(grid, 0);
      for (size_t k = 0; k < jobs.size(); ++k) {
        const int mt = (jobs[k].n + BM - 1) / BM, kt = (jobs[k].n + BK - 1) / BK;
        for (int m = 0; m < mt; ++m) {
          const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
          per[c].push_back(make_int4((int)k, m, 0, kt));
          load[c] += kt;
        }
      }
    }
    for (int c = 0; c < grid; ++c) {
      cbeg[c] = (int)segs.size();
      for (const int4& sg : per[c]) {
        const int g = jobs[sg.x].mt0 + sg.y;
        mt_seg[g] = make_int2((int)segs.size(), 1);
        segs.push_back(sg);
      }
    }
  }
  for (int c = 0; c < grid && dealing == GEMM_DEAL_STREAMK; ++c) {
    const long long b = W * c / grid, e = W * (c + 1) / grid;
    cbeg[c] = (int)segs.size();
    long long t = b;
    while (t < e) {
      while (job_base[jk + 1] <= t) ++jk;
      const gemm_job& J = jobs[jk];
      const long long kt = (J.n + BK - 1) / BK;
      const long long local = t - job_base[jk];
      const int m = (int)(local / kt), k0 = (int)(local % kt);
      const int k1 = (int)std::min<long long>(kt, k0 + (e - t));
      const int g = J.mt0 + m;
      if (mt_seg[g].y == 0) mt_seg[g].x = (int)segs.size();
      mt_seg[g].y++;
      segs.push_back(make_int4((int)jk, m, k0, k1));
      t += k1 - k0;
    }
  }
  cbeg[grid] = (int)segs.size();
  for (size_t k = 0; k < jobs.size(); ++k) {
    const int mt = (jobs[k].n + BM - 1) / BM;
    for (int m = 0; m < mt; ++m) mt_job[jobs[k].mt0 + m] = make_int2((int)k, m);
  }
  G.grid = grid;
  G.njobs = (int)jobs.size();
  G.mt_total = mt_total;
  G.nsegs = (int)segs.size();
  int max_pitch = 0;
  for (auto& J : jobs) max_pitch = std::max(max_pitch, J.pitch);
  G.max_pitch = max_pitch;
  G.jobs.reserve(sizeof(gemm_job) * jobs.size());
  G.tables.reserve(sizeof(int4) * segs.size() + sizeof(int) * cbeg.size() +
                   2 * sizeof(int2) * mt_total + 256);
  // whole-tile dealings give one segment per m tile: y is written by the
  // contraction's epilogue, with no partial sums and no reduction launch
  const bool direct = (int)segs.size() == mt_total;
  if (!direct) G.partial.reserve(sizeof(float2) * (size_t)segs.size() * BM * kNR);
  G.io.reserve(sizeof(gemm_io));
  G.err.reserve(sizeof(int));
  char* tb = G.tables.as<char>();
  const size_t o_segs = 0;
  const size_t o_cbeg = (sizeof(int4) * segs.size() + 15) & ~size_t(15);
  const size_t o_mtj = (o_cbeg + sizeof(int) * cbeg.size() + 15) & ~size_t(15);
  const size_t o_mts = (o_mtj + sizeof(int2) * mt_total + 15) & ~size_t(15);
  CFIE_CHECK_CUDA(cudaMemcpyAsync(G.jobs.p, jobs.data(), sizeof(gemm_job) * jobs.size(),
                                  cudaMemcpyHostToDevice, st));
  CFIE_CHECK_CUDA(cudaMemcpyAsync(tb + o_segs, segs.data(), sizeof(int4) * segs.size(),
                                  cudaMemcpyHostToDevice, st));
  CFIE_CHECK_CUDA(cudaMemcpyAsync(tb + o_cbeg, cbeg.data(), sizeof(int) * cbeg.size(),
                                  cudaMemcpyHostToDevice, st));
  CFIE_CHECK_CUDA(cudaMemcpyAsync(tb + o_mtj, mt_job.data(), sizeof(int2) * mt_total,
                                  cudaMemcpyHostToDevice, st));
  CFIE_CHECK_CUDA(cudaMemcpyAsync(tb + o_mts, mt_seg.data(), sizeof(int2) * mt_total,
                                  cudaMemcpyHostToDevice, st));
  CFIE_CHECK_CUDA(cudaMemsetAsync(G.err.p, 0, sizeof(int), st));
  CFIE_CHECK_CUDA(cudaStreamSynchronize(st));

  // CFIE_FAULT_INJECT=tma_stall (failure tests only) makes the contraction's
  // bounded waits run out
  const char* fi = std::getenv("CFIE_FAULT_INJECT");
  G.stall = (fi && std::strcmp(fi, "tma_stall") == 0) ? 1 : 0;
  // capture the two or three launches once; replays read x / y from the io slot
  const size_t smem = pgemm_smem_bytes<kNP>();
  CFIE_CHECK_CUDA(cudaFuncSetAttribute(k_gemm_persistent<kNP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaStream_t cs;
  CFIE_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaError_t e1 = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e1 == cudaSuccess) {
    const gemm_job* dj = G.jobs.as<gemm_job>();
    const gemm_io* io = G.io.as<gemm_io>();
    k_prep_b_jobs<<<dim3(kNR, G.njobs), 256, 0, cs>>>(dj, io, kNP);
    k_gemm_persistent<kNP><<<grid, 192, smem, cs>>>(
        dj, reinterpret_cast<const int4*>(tb + o_segs), reinterpret_cast<const int*>(tb + o_cbeg),
        direct ? nullptr : G.partial.as<float2>(), direct ? io : nullptr, G.err.as<int>(),
        G.stall);
    if (!direct)
      k_reduce_jobs<<<dim3(mt_total, kNR), BM, 0, cs>>>(
          dj, reinterpret_cast<const int2*>(tb + o_mtj),
          reinterpret_cast<const int2*>(tb + o_mts), G.partial.as<float2>(), io, kNR);
    e1 = cudaStreamEndCapture(cs, &graph);
  }
  cudaStreamDestroy(cs);
  CFIE_CHECK_CUDA(e1);
  if (G.exec) cudaGraphExecDestroy(G.exec);
  G.exec = nullptr;
  cudaError_t e2 = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  CFIE_CHECK_CUDA(e2);
  G.launches_per_run = direct ? 2 : 3;
}

void gemm_plan_run(gemm_plan& G, cfie_ctx* ctx, const double2* x, double2* y) {
  const gemm_io io{x, y};
  // pageable source: the copy is staged before cudaMemcpyAsync returns
  CFIE_CHECK_CUDA(cudaMemcpyAsync(G.io.p, &io, sizeof(io), cudaMemcpyHostToDevice, ctx->stream));
  prof_scope ps(ctx, CFIE_K_MATVEC_TENSOR);
  CFIE_CHECK_CUDA(cudaGraphLaunch(G.exec, ctx->stream));
  g_cfie_launches += G.launches_per_run;
}

// The autotuner of the batched contraction: each dealing built and its graph
// replay timed (one warm-up, then the mean of two, CUDA events on the context
// stream, on zero vectors); the fastest is kept and remembered per batch shape
// (the sequence of (n, right-hand sides)) for the process.
namespace {
std::mutex g_tune_mu;
std::map<std::vector<long long>, int> g_tune;
}  // namespace

int gemm_plan_tune(gemm_plan& G, cfie_ctx* ctx, const std::vector<cfie_op*>& ops,
                   const std::vector<int>& nrhs, const std::vector<long long>& xoff, size_t L,
                   float* ms) {
  std::vector<long long> key;
  for (size_t k = 0; k < ops.size(); ++k) {
    key.push_back(ops[k]->n);
    key.push_back(nrhs[k]);
  }
  ms[0] = ms[1] = ms[2] = 0.f;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      gemm_plan_build(G, ctx, ops, nrhs, xoff, it->second);
      return it->second;
    }
  }
  cudaStream_t st = ctx->stream;
  dbuf xy;
  xy.reserve(sizeof(double2) * 2 * L);
  CFIE_CHECK_CUDA(cudaMemsetAsync(xy.p, 0, sizeof(double2) * 2 * L, st));
  const double2* x = xy.as<double2>();
  double2* y = xy.as<double2>() + L;
  cudaEvent_t e0, e1;
  CFIE_CHECK_CUDA(cudaEventCreate(&e0));
  CFIE_CHECK_CUDA(cudaEventCreate(&e1));
  ctx->prof_suspend++;
  int best = GEMM_DEAL_ROUND_ROBIN;
  float best_ms = 0.f;
  try {
    for (int d = GEMM_DEAL_ROUND_ROBIN; d <= GEMM_DEAL_STREAMK; ++d) {
      gemm_plan_build(G, ctx, ops, nrhs, xoff, d);
      gemm_plan_run(G, ctx, x, y);
      CFIE_CHECK_CUDA(cudaEventRecord(e0, st));
      gemm_plan_run(G, ctx, x, y);
      gemm_plan_run(G, ctx, x, y);
      CFIE_CHECK_CUDA(cudaEventRecord(e1, st));
      CFIE_CHECK_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      CFIE_CHECK_CUDA(cudaEventElapsedTime(&t, e0, e1));
      ms[d] = 0.5f * t;
      if (gemm_plan_take_error(G, ctx))
        throw cfie_error(CFIE_ETIMEOUT, "tensor-core kernel gave up a bounded wait");
      if (d == GEMM_DEAL_ROUND_ROBIN || ms[d] < best_ms) {
        best = d;
        best_ms = ms[d];
      }
    }
  } catch (...) {
    ctx->prof_suspend--;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  ctx->prof_suspend--;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (G.dealing != best) gemm_plan_build(G, ctx, ops, nrhs, xoff, best);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (g_tune.size() >= 64) g_tune.clear();
  g_tune[key] = best;
  return best;
}

int gemm_plan_take_error(gemm_plan& G, cfie_ctx* ctx) {
  if (!G.err.p) return 0;
  int e = 0;
  CFIE_CHECK_CUDA(
      cudaMemcpyAsync(&e, G.err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CFIE_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  if (e) CFIE_CHECK_CUDA(cudaMemsetAsync(G.err.p, 0, sizeof(int), ctx->stream));
  return e;
}

void gemm_plan_release(gemm_plan& G) {
  if (G.exec) cudaGraphExecDestroy(G.exec);
  G.exec = nullptr;
}

void stored_prepare(cfie_op* op) {
  if (op->bc != CFIE_SOUND_SOFT)
    throw cfie_error(CFIE_EINVAL, "the stored layout supports the sound-soft operator");
  const int n = op->n;
  const int pitch = stored_pitch(n);
  const size_t plane = (size_t)((n + BM - 1) / BM) * BM * pitch;   // whole row blocks
  op->stored.reserve(sizeof(__nv_bfloat16) * 4 * plane);
  CFIE_CHECK_CUDA(cudaMemsetAsync(op->stored.p, 0, sizeof(__nv_bfloat16) * 4 * plane,
                                  op->ctx->stream));
  float* base = op->geo32.as<float>();
  const dim3 grid(nblk(pitch), n);
  // the row maxima of the far entries come with the assembly (sound soft:
  // the tensor-core residual's row exponents), not from a separate pass
  unsigned* rmax = nullptr;
  if (op->df_b > 0) {
    op->df_rowexp.reserve(sizeof(int) * (size_t)n);
    rmax = reinterpret_cast<unsigned*>(op->df_rowexp.as<int>());
    CFIE_CHECK_CUDA(cudaMemsetAsync(rmax, 0, sizeof(unsigned) * n, op->ctx->stream));
  }
  k_assemble<<<grid, 256, 0, op->ctx->stream>>>(
      n, pitch, op->band_b, op->df_b, reinterpret_cast<const float4*>(base + geo32_pack_offset(n)),
      reinterpret_cast<const float2*>(base + geo32_wk_offset(n)), op->band.as<float2>(),
      op->stored.as<__nv_bfloat16>(), rmax);
  CFIE_CHECK_LAUNCH();
  if (rmax) {
    k_rowexp_from_max<<<nblk(n), 256, 0, op->ctx->stream>>>(n, rmax);
    CFIE_CHECK_LAUNCH();
  }
  CFIE_CHECK_CUDA(cudaStreamSynchronize(op->ctx->stream));
}

void matvec_stored(cfie_op* op, const double2* x, double2* y, int nrhs) {
  if (op->plan_nrhs != nrhs) {
    gemm_plan_build(op->plan, op->ctx, {op}, {nrhs}, {0}, GEMM_DEAL_AUTO);
    op->plan_nrhs = nrhs;
  }
  gemm_plan_run(op->plan, op->ctx, x, y);
}

int stored_take_error(cfie_op* op) { return gemm_plan_take_error(op->plan, op->ctx); }
