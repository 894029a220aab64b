// Matrix-free FP32 matvec with the source summation on the tensor cores.
//
// Same entries as the FP32 fused kernel (sound-soft operator of eq. 1: FP32
// pair evaluation with two-float phase and Hankel asymptotics, FP64-evaluated
// near band), but instead of the register-blocked FP32 contraction the entries
// of each 128 x 32 tile are written, split as bf16 hi + lo, straight into
// shared memory in the tensor cores' 64-byte-swizzled K-major layout, and one
// thread issues tcgen05.mma against the right-hand-side block (bf16 hi / lo
// planes brought in by TMA):
//
//     [Yr | Yi] += Ar [Xr | Xi] + Ai [-Xi | Xr],  each product hi*hi + hi*lo + lo*hi,
//
// FP32 accumulation in tensor memory.  Work is split stream-K: the
// (128-row tile, 32-source tile) pairs form one list and each CTA (one per SM)
// takes a contiguous range, cut into segments that end at row-tile boundaries.
// Warp roles (22 warps): 0-15 evaluate pair entries into the stage ring, 16
// issues the TMA loads of the right-hand sides, of each tile's source geometry
// and of its Kress window, 17 issues the MMAs (double-buffered accumulators),
// 18-21 drain finished accumulators into per-segment partial sums, which a
// second kernel adds in a fixed order.  All mbarrier waits are bounded (error
// flag, drain, TMEM freed on every path).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <string>

#include "internal.h"
#include "pair32.cuh"
#include "tc_common.cuh"

namespace {

constexpr int TBM = 128;     // targets per tile (UMMA M)
constexpr int TBK = 32;      // sources per tile (32 bf16 = one 64-byte swizzle row)
constexpr int TSTAGES = 3;
// Source tiles accumulated in one tensor-memory accumulator before the epilogue
// warps add it into their running sums.  The tensor core's FP32 accumulation
// does not round to nearest: its error grows with the number of MMAs summed
// into one accumulator (~2e-8 relative per MMA), so chunks of 256 sources keep
// that bias near 2e-6 whatever n is, while the running sums (FP32 adds, rounded
// to nearest) and the FP64 segment reduction add only unbiased rounding.
constexpr int CK = 8;
constexpr int WKW = TBM + TBK + 2;   // Kress window of a tile (+ alignment slack)
constexpr int NPROD = 16;    // producer warps
constexpr int WTMA = NPROD, WMMA = NPROD + 1;   // then the epilogue warps
constexpr int TNT = (NPROD + 6) * 32;
constexpr int QI = 2;        // rows whose entries a producer lane evaluates together

struct tc_params {
  int n, b, ktiles;
  const float2* wext;    // Kress table / (pi h) at i - j + n, paired with the next source's
  const float4* pk;      // packed coordinates, source factors, target factors (n each)
  const float2* band;    // near entries of the evaluated kind (soft A, or S, or D')
};

// bf16 hi / lo split of two entries of one row (adjacent sources k, k + 1)
// into the four A planes: one packed 32-bit word per plane at byte offset o
__device__ __forceinline__ void store_split2(unsigned char* a0, unsigned char* a1,
                                             unsigned char* a2, unsigned char* a3, uint32_t o,
                                             float2 e0, float2 e1) {
  const __nv_bfloat162 hr = __floats2bfloat162_rn(e0.x, e1.x);
  const __nv_bfloat162 hi = __floats2bfloat162_rn(e0.y, e1.y);
  const __nv_bfloat162 lr =
      __floats2bfloat162_rn(e0.x - __low2float(hr), e1.x - __high2float(hr));
  const __nv_bfloat162 li =
      __floats2bfloat162_rn(e0.y - __low2float(hi), e1.y - __high2float(hi));
  *reinterpret_cast<__nv_bfloat162*>(a0 + o) = hr;
  *reinterpret_cast<__nv_bfloat162*>(a1 + o) = hi;
  *reinterpret_cast<__nv_bfloat162*>(a2 + o) = lr;
  *reinterpret_cast<__nv_bfloat162*>(a3 + o) = li;
}

template <int NP>
struct tc_smem {
  __nv_bfloat16 A[TSTAGES][4][TBM * TBK];   // hi_re, hi_im, lo_re, lo_im
  __nv_bfloat16 B[TSTAGES][4][NP * TBK];    // B1 hi, B1 lo, B2 hi, B2 lo
  float4 tgt[TBM];                          // targets (x hi, x lo, y hi, y lo)
  float4 tgn[TBM];                          // target factors (D' only)
  float4 src[TSTAGES][2][TBK];              // sources: coordinates, factors
  float2 wk[TSTAGES][WKW];                  // Kress weight pairs / (pi h) of a plain tile
  uint64_t full[TSTAGES], empty[TSTAGES], sfull[TSTAGES], tfull[2], tempty[2];
  uint64_t mdone;                           // completion of every MMA issued (abort path)
  uint32_t tmem_base;
  int abort;
  int issued[TSTAGES], sissued[TSTAGES];
  int wofs[TSTAGES];                        // plain tile: window entry of (row 0, source 0); else -1
};

template <int NP>
constexpr size_t tc_smem_bytes() {
  return sizeof(tc_smem<NP>) + 1024;
}

// byte offset of element (row r, k) in a 64-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t sw64(int r, int k) {
  return (uint32_t)(r * 64 + ((((k >> 3) ^ (r >> 1)) & 3) << 4) + (k & 7) * 2);
}

template <int NP, int KIND>
__global__ void __launch_bounds__(TNT, 1)
k_fused_tc(tc_params P, const __grid_constant__ CUtensorMap tmB, const int4* __restrict__ segs,
           const int* __restrict__ cbeg, float2* __restrict__ partial, int* __restrict__ err) {
  constexpr int NR = NP / 2;
  // two accumulator buffers, then the epilogue's running sums (NP columns each)
  constexpr uint32_t TMEM_COLS = 3 * NP <= 256 ? 256 : 512;
  constexpr uint32_t RUN = 2 * NP;
  constexpr uint32_t B_BYTES = 4u * NP * TBK * 2u;
  extern __shared__ unsigned char raw[];
  tc_smem<NP>& S = *reinterpret_cast<tc_smem<NP>*>((reinterpret_cast<uintptr_t>(raw) + 1023) &
                                                    ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sb = cbeg[blockIdx.x], se = cbeg[blockIdx.x + 1];
  const int n = P.n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      mbar_init(&S.full[s], NPROD + 1);        // one arrival per producer warp + the TMA thread
      mbar_init(&S.empty[s], 1);
      mbar_init(&S.sfull[s], 1);
      S.issued[s] = -1;
      S.sissued[s] = -1;
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.tfull[b], 1);
      mbar_init(&S.tempty[b], 4);
    }
    mbar_init(&S.mdone, 1);
    S.abort = 0;
    fence_mbar_init();
  }
  if (warp == WMMA) {
    tmem_alloc(&S.tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;

  if (warp < NPROD) {
    // ---- pair-entry producers.  Warp w owns rows w + NPROD q (q < TBM / NPROD);
    // each step of its loop covers two of them: lanes 0-15 the first, lanes
    // 16-31 the second, lane l the two adjacent sources 2 (l % 16), +1, so
    // that the bf16 pairs go to shared memory as packed 32-bit words.
    const int half = lane >> 4, jp = 2 * (lane & 15);
    // byte offset of the lane's two sources in its first row of a step; the
    // rows of step q lie 2 NPROD q rows further on, a multiple of the 8-row
    // period of the 64-byte swizzle, hence 2 NPROD q 64 bytes further
    static_assert((2 * NPROD) % 8 == 0, "row step must keep the swizzle phase");
    const uint32_t sbase = sw64(warp + NPROD * half, jp);
    int it = 0;
    for (int s = sb; s < se; ++s) {
      const int4 sg = segs[s];
      const int m0 = sg.y * TBM;
      // stage the target geometry of this warp's own rows: no other warp
      // reads them, so a warp-level barrier is enough
      __syncwarp();
      if (lane < TBM / NPROD) {
        const int r = warp + NPROD * lane;
        const int i = m0 + r;
        const bool ok = i < n;
        S.tgt[r] = ok ? P.pk[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (KIND == KIND_DP) S.tgn[r] = ok ? P.pk[2 * n + i] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncwarp();
      for (int k = sg.z; k < sg.w; ++k, ++it) {
        const int st = it % TSTAGES;
        const int j0 = k * TBK;
        const int j = j0 + jp;                       // first of the lane's two sources
        // exits are warp-uniform: the warp arrives on the stage barrier as one
        if (__any_sync(0xffffffffu, *(volatile int*)&S.abort)) break;
        // this tile's source geometry and Kress window, brought in by the TMA
        // warp once the MMAs of the stage's previous tile were done (so the A
        // planes of the stage are free as well)
        if (!__all_sync(0xffffffffu, mbar_wait(&S.sfull[st], (it / TSTAGES) & 1))) {
          if (lane == 0) {
            atomicExch(err, 15);
            S.abort = 1;
          }
          break;
        }
        const float4 sc[2] = {S.src[st][0][jp], S.src[st][0][jp + 1]};
        const float4 sn[2] = {S.src[st][1][jp], S.src[st][1][jp + 1]};
        unsigned char* a0 = reinterpret_cast<unsigned char*>(S.A[st][0]);
        unsigned char* a1 = reinterpret_cast<unsigned char*>(S.A[st][1]);
        unsigned char* a2 = reinterpret_cast<unsigned char*>(S.A[st][2]);
        unsigned char* a3 = reinterpret_cast<unsigned char*>(S.A[st][3]);
        // Plain tiles (all but ~1%, flagged by the TMA warp) skip the per-pair
        // range and band tests and take the Kress weights from the staged
        // window of the unwrapped table (entry i - j + n)
        const int wofs = S.wofs[st];
        constexpr int QS = TBM / NPROD / 2;          // loop steps (two rows each)
        if (wofs >= 0) {
          const float2* wq = S.wk[st] + wofs + warp + NPROD * half - jp;
          float2 wv[QS];
#pragma unroll
          for (int q = 0; q < QS; ++q) wv[q] = wq[2 * NPROD * q];
          // QI rows at a time: the phases (special-function ops) of their
          // 2 QI entries first, then the series and assembly, so that the
          // independent chains interleave
#pragma unroll
          for (int q0 = 0; q0 < QS; q0 += QI) {
            pair_phase f[QI][2];
            float4 tn[QI];
#pragma unroll
            for (int r = 0; r < QI; ++r) {
              const int il = warp + NPROD * (2 * (q0 + r) + half);
              const float4 tg = S.tgt[il];
              tn[r] = KIND == KIND_DP ? S.tgn[il] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int u = 0; u < 2; ++u)
                f[r][u] = pair_phase32_tc(tg.x, tg.y, tg.z, tg.w, sc[u].x, sc[u].y, sc[u].z,
                                          sc[u].w);
            }
#pragma unroll
            for (int r = 0; r < QI; ++r) {
              const int q = q0 + r;
              float2 e[2];
#pragma unroll
              for (int u = 0; u < 2; ++u)
                e[u] = entry_finish32<KIND>(f[r][u], tn[r], sn[u], u ? wv[q].y : wv[q].x);
              store_split2(a0, a1, a2, a3, sbase + (uint32_t)(2 * NPROD * 64 * q), e[0], e[1]);
            }
          }
        } else {
#pragma unroll 1
          for (int q = 0; q < QS; ++q) {
            const int il = warp + NPROD * (2 * q + half);
            const int i = m0 + il;
            const float4 tg = S.tgt[il];
            const float4 tn = KIND == KIND_DP ? S.tgn[il] : make_float4(0.f, 0.f, 0.f, 0.f);
            float2 e[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int jj = j + u;
              float2 a = make_float2(0.f, 0.f);
              if (i < n && jj < n) {
                int d = i - jj;
                if (d < 0) d += n;
                const int dd = d <= P.b ? d : (d >= n - P.b ? d - n : INT_MAX);
                if (dd != INT_MAX)
                  a = P.band[(size_t)i * (2 * P.b + 1) + dd + P.b];
                else
                  a = entry_folded32<KIND>(tg, tn, sc[u], sn[u], P.wext[i - jj + n].x);
              }
              e[u] = a;
            }
            store_split2(a0, a1, a2, a3, sbase + (uint32_t)(2 * NPROD * 64 * q), e[0], e[1]);
          }
        }
        // generic-proxy writes become visible to the tensor core's async proxy;
        // the warp's writes are ordered before its one arrival by __syncwarp
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.full[st]);
      }
      if (__any_sync(0xffffffffu, *(volatile int*)&S.abort)) break;
    }
  } else if (warp == WTMA) {
    if (lane == 0) {
      // ---- TMA producer of the right-hand-side planes
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      int it = 0;
      for (int s = sb; s < se && !*(volatile int*)&S.abort; ++s) {
        const int4 sg = segs[s];
        for (int k = sg.z; k < sg.w; ++k, ++it) {
          const int st = it % TSTAGES;
          if (it >= TSTAGES && !mbar_wait(&S.empty[st], ((it / TSTAGES) - 1) & 1)) {
            atomicExch(err, 12);
            S.abort = 1;
            break;
          }
          mbar_arrive_expect_tx(&S.full[st], B_BYTES);
          S.issued[st] = (it / TSTAGES) & 1;
#pragma unroll
          for (int p = 0; p < 4; ++p) tma_load_2d(S.B[st][p], &tmB, &S.full[st], k * TBK, p * NP);
          // Source coordinates and factors of the tile.  A tile is plain when
          // it holds full rows and sources and no pair of the near band: d =
          // i - j spans [dlo, dhi] there, and the band is |d - t n| <= b for
          // t = -1, 0, 1; a plain tile also gets the window of the Kress table
          // (entries dlo + n ... dhi + n) from the 16-byte boundary below it.
          // Window bytes: WKW float2 = 1296, a multiple of 16.
          const int m0 = sg.y * TBM, j0 = k * TBK;
          const int dlo = m0 - j0 - (TBK - 1), dhi = m0 + TBM - 1 - j0;
          bool near = false;
#pragma unroll
          for (int t = -1; t <= 1; ++t) near |= (dhi >= t * n - P.b) && (dlo <= t * n + P.b);
          const bool plain = !near && m0 + TBM <= n && j0 + TBK <= n;
          S.wofs[st] = plain ? m0 - j0 + n - ((dlo + n) & ~1) : -1;
          mbar_arrive_expect_tx(&S.sfull[st], 2u * TBK * 16u + (plain ? WKW * 8u : 0u));
          S.sissued[st] = (it / TSTAGES) & 1;
          bulk_load(S.src[st][0], P.pk + j0, TBK * 16u, &S.sfull[st]);
          bulk_load(S.src[st][1], P.pk + n + j0, TBK * 16u, &S.sfull[st]);
          if (plain) bulk_load(S.wk[st], P.wext + ((dlo + n) & ~1), WKW * 8u, &S.sfull[st]);
        }
      }
    }
  } else if (warp == WMMA) {
    if (lane == 0) {
      // ---- MMA issuer: one accumulator buffer per chunk of CK source tiles
      constexpr uint32_t idesc = make_idesc(TBM, NP);
      int it = 0, cc = 0;
      for (int s = sb; s < se && !*(volatile int*)&S.abort; ++s) {
        const int4 sg = segs[s];
        for (int c0 = sg.z; c0 < sg.w; c0 += CK, ++cc) {
          const int c1 = min(sg.w, c0 + CK);
          const int tb = cc & 1, use = cc >> 1;
          if (use >= 1 && !mbar_wait(&S.tempty[tb], (use - 1) & 1)) {
            atomicExch(err, 14);
            S.abort = 1;
          }
          if (*(volatile int*)&S.abort) break;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(tb * NP);
          for (int k = c0; k < c1; ++k, ++it) {
            const int st = it % TSTAGES;
            if (!mbar_wait(&S.full[st], (it / TSTAGES) & 1)) {
              atomicExch(err, 13);
              S.abort = 1;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(S.A[st][0]), a1 = smem_u32(S.A[st][1]);
            const uint32_t a2 = smem_u32(S.A[st][2]), a3 = smem_u32(S.A[st][3]);
            const uint32_t b0 = smem_u32(S.B[st][0]), b1 = smem_u32(S.B[st][1]);
            const uint32_t b2 = smem_u32(S.B[st][2]), b3 = smem_u32(S.B[st][3]);
#pragma unroll
            for (int kk = 0; kk < TBK / 16; ++kk) {
              const uint32_t off = kk * 32;
              const uint32_t acc0 = (k > c0 || kk > 0) ? 1u : 0u;
              umma_bf16(d, smem_desc_sw64(a0 + off), smem_desc_sw64(b0 + off), idesc, acc0);
              umma_bf16(d, smem_desc_sw64(a0 + off), smem_desc_sw64(b1 + off), idesc, 1u);
              umma_bf16(d, smem_desc_sw64(a2 + off), smem_desc_sw64(b0 + off), idesc, 1u);
              umma_bf16(d, smem_desc_sw64(a1 + off), smem_desc_sw64(b2 + off), idesc, 1u);
              umma_bf16(d, smem_desc_sw64(a1 + off), smem_desc_sw64(b3 + off), idesc, 1u);
              umma_bf16(d, smem_desc_sw64(a3 + off), smem_desc_sw64(b2 + off), idesc, 1u);
            }
            umma_commit(&S.empty[st]);
          }
          umma_commit(&S.tfull[tb]);
        }
      }
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, one row per
    // thread, and keeps the segment's running sums in the same lanes of the
    // last NP tensor-memory columns (FP32 adds, rounded to nearest)
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const uint32_t lanes = tmem + ((uint32_t)(32 * q) << 16);
    int cc = 0;
    bool stop = false;
    for (int s = sb; s < se && !stop; ++s) {
      const int4 sg = segs[s];
      for (int c0 = sg.z; c0 < sg.w; c0 += CK, ++cc) {
        const int tb = cc & 1, use = cc >> 1;
        if (*(volatile int*)&S.abort || !mbar_wait(&S.tfull[tb], use & 1)) {
          if (lane == 0) {
            atomicExch(err, 15);
            S.abort = 1;
          }
          stop = true;
          break;
        }
        __syncwarp();
        tc_fence_after();
        const uint32_t base = lanes + (uint32_t)(tb * NP);
        const bool first = c0 == sg.z;
#pragma unroll 2
        for (int cb = 0; cb < NP; cb += 16) {
          float v[16];
          tmem_ld16(base + (uint32_t)cb, v);
          if (!first) {
            float r[16];
            tmem_ld16(lanes + RUN + (uint32_t)cb, r);
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] += r[k];
          }
          tmem_st16(lanes + RUN + (uint32_t)cb, v);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.tempty[tb]);
      }
      if (stop) break;
      float2* dst = partial + (size_t)s * TBM * NR + row;
#pragma unroll 1
      for (int cb = 0; cb < NR; cb += 16) {
        float re[16], im[16];
        tmem_ld16(lanes + RUN + (uint32_t)cb, re);
        tmem_ld16(lanes + RUN + (uint32_t)(NR + cb), im);
#pragma unroll
        for (int k = 0; k < 16; ++k) dst[(size_t)(cb + k) * TBM] = make_float2(re[k], im[k]);
      }
    }
  }
  __syncthreads();
  // after an abort, wait (bounded) for copies in flight and for every MMA
  // issued, then free TMEM
  if (*(volatile int*)&S.abort) {
    if (threadIdx.x == 0)
      for (int s = 0; s < TSTAGES; ++s) {
        if (S.issued[s] >= 0) mbar_wait(&S.full[s], (uint32_t)S.issued[s]);
        if (S.sissued[s] >= 0) mbar_wait(&S.sfull[s], (uint32_t)S.sissued[s]);
      }
    if (warp == WMMA && lane == 0) {
      umma_commit(&S.mdone);
      mbar_wait(&S.mdone, 0);
    }
  }
  __syncthreads();
  if (warp == WMMA) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// y[r][i] = sum of the (one to a few) segment partials of row tile i / 128, in
// a fixed order; FP32 adds (the partials are FP32 sums of bf16 products: FP64
// adds would buy nothing here and run at 1/64 of the FP32 rate)
__global__ void k_reduce_tc(int n, int nr, int NR, const int2* __restrict__ mt_seg,
                            const float2* __restrict__ partial, double2* __restrict__ y) {
  const int m = blockIdx.x, r = blockIdx.y, row = threadIdx.x;
  const int i = m * TBM + row;
  if (i >= n || r >= nr) return;
  const int2 sr = mt_seg[m];
  float sx = 0.f, sy = 0.f;
  for (int s = sr.x; s < sr.x + sr.y; ++s) {
    const float2 p = partial[((size_t)s * NR + r) * TBM + row];
    sx += p.x;
    sy += p.y;
  }
  y[(size_t)r * n + i] = make_double2(sx, sy);
}

unsigned nb(size_t len, int t = 256) { return (unsigned)((len + t - 1) / t); }

template <int NP, int KIND>
void run_fused(cfie_op* op, const double2* x, double2* y, int r0, int nr) {
  constexpr int NR = NP / 2;
  tc_plan& T = op->tc[NP == 64 ? 0 : 1];
  const int n = op->n;
  cudaStream_t st = op->ctx->stream;
  const int pitch = (n + 63) / 64 * 64;
  if (!T.built) {
    const int mtiles = (n + TBM - 1) / TBM, ktiles = (n + TBK - 1) / TBK;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, op->ctx->device);
    std::vector<int4> segs;
    std::vector<int> cbeg;
    std::vector<int2> mt_seg;
    streamk_segments(mtiles, ktiles, sms, segs, cbeg, mt_seg);
    T.grid = (int)cbeg.size() - 1;
    T.nsegs = (int)segs.size();
    T.mtiles = mtiles;
    T.tables.reserve(sizeof(int4) * segs.size() + sizeof(int) * cbeg.size() +
                     sizeof(int2) * mt_seg.size() + 64);
    char* tb = T.tables.as<char>();
    T.o_cbeg = (sizeof(int4) * segs.size() + 15) & ~size_t(15);
    T.o_mts = (T.o_cbeg + sizeof(int) * cbeg.size() + 15) & ~size_t(15);
    CFIE_CHECK_CUDA(cudaMemcpyAsync(tb, segs.data(), sizeof(int4) * segs.size(),
                                    cudaMemcpyHostToDevice, st));
    CFIE_CHECK_CUDA(cudaMemcpyAsync(tb + T.o_cbeg, cbeg.data(), sizeof(int) * cbeg.size(),
                                    cudaMemcpyHostToDevice, st));
    CFIE_CHECK_CUDA(cudaMemcpyAsync(tb + T.o_mts, mt_seg.data(), sizeof(int2) * mt_seg.size(),
                                    cudaMemcpyHostToDevice, st));
    T.bt.reserve(sizeof(__nv_bfloat16) * 4 * (size_t)NP * pitch);
    T.partial.reserve(sizeof(float2) * (size_t)T.nsegs * TBM * NR);
    T.err.reserve(sizeof(int));
    CFIE_CHECK_CUDA(cudaMemsetAsync(T.err.p, 0, sizeof(int), st));
    const CUtensorMap mb = tc_make_map(T.bt.p, 4 * (uint64_t)NP, (uint64_t)pitch, pitch, NP,
                                       TBK, CU_TENSOR_MAP_SWIZZLE_64B);
    std::memcpy(T.tmB, &mb, sizeof(mb));
    CFIE_CHECK_CUDA(cudaStreamSynchronize(st));
    T.built = true;
  }
  prep_b_planes(op->ctx, n, pitch, NP, nr, x + (size_t)r0 * n, T.bt.as<__nv_bfloat16>());
  tc_params P{};
  P.n = n;
  P.b = op->band_b;
  P.ktiles = (n + TBK - 1) / TBK;
  float* base = op->geo32.as<float>();
  P.wext = reinterpret_cast<const float2*>(base + geo32_wk_offset(n));
  P.pk = reinterpret_cast<const float4*>(base + geo32_pack_offset(n));
  // the FP32 band holds the soft entries, or S then D' for the hard operator
  P.band = op->band.as<float2>() +
           (KIND == KIND_DP ? (size_t)n * (2 * (size_t)op->band_b + 1) : (size_t)0);
  const size_t smem = tc_smem_bytes<NP>();
  CFIE_CHECK_CUDA(cudaFuncSetAttribute(k_fused_tc<NP, KIND>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  char* tb = T.tables.as<char>();
  {
    prof_scope ps(op->ctx, CFIE_K_MATVEC_FP32);
    k_fused_tc<NP, KIND><<<T.grid, TNT, smem, st>>>(P, *reinterpret_cast<const CUtensorMap*>(T.tmB),
                                             reinterpret_cast<const int4*>(tb),
                                             reinterpret_cast<const int*>(tb + T.o_cbeg),
                                             T.partial.as<float2>(), T.err.as<int>());
    CFIE_CHECK_LAUNCH();
  }
  k_reduce_tc<<<dim3(T.mtiles, nr), TBM, 0, st>>>(n, nr, NR,
                                                 reinterpret_cast<const int2*>(tb + T.o_mts),
                                                 T.partial.as<float2>(), y + (size_t)r0 * n);
  CFIE_CHECK_LAUNCH();
}

template <int KIND>
void run_blocks(cfie_op* op, const double2* x, double2* y, int nrhs) {
  for (int r0 = 0; r0 < nrhs; r0 += 64) {
    const int nr = std::min(64, nrhs - r0);
    if (nr > 32)
      run_fused<128, KIND>(op, x, y, r0, nr);
    else
      run_fused<64, KIND>(op, x, y, r0, nr);
  }
}

// hard operator inputs of the S sums: [u, n1 x, n2 x] (u = (1/|z'|) d/dt x)
__global__ void k_hard_inputs(int n, size_t tot, const double2* __restrict__ x,
                              const float2* __restrict__ u32, geom_dev g,
                              double2* __restrict__ v) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= tot) return;
  const int i = (int)(e % n);
  const double inv = 1.0 / g.sp[i];
  const double2 xv = x[e];
  const float2 uv = u32[e];
  v[e] = make_double2(uv.x, uv.y);
  v[tot + e] = make_double2(g.nx[i] * inv * xv.x, g.nx[i] * inv * xv.y);
  v[2 * tot + e] = make_double2(g.ny[i] * inv * xv.x, g.ny[i] * inv * xv.y);
}

// y = x/2 - D' x - i (omega^2 / eta) (n1 S(n1 x) + n2 S(n2 x)), t = S u (FP32)
__global__ void k_hard_combine(int n, size_t tot, double omega, double eta, geom_dev g,
                               const double2* __restrict__ x, const double2* __restrict__ ys,
                               const double2* __restrict__ yd, float2* __restrict__ t32,
                               double2* __restrict__ y) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= tot) return;
  const int i = (int)(e % n);
  const double inv = 1.0 / g.sp[i];
  const double n1 = g.nx[i] * inv, n2 = g.ny[i] * inv;
  const double2 s1 = ys[tot + e], s2 = ys[2 * tot + e];
  const double2 m = make_double2(n1 * s1.x + n2 * s2.x, n1 * s1.y + n2 * s2.y);
  const double k = omega * omega / eta;
  const double2 xv = x[e], d = yd[e];
  y[e] = make_double2(0.5 * xv.x - d.x + k * m.y, 0.5 * xv.y - d.y - k * m.x);
  t32[e] = make_float2((float)ys[e].x, (float)ys[e].y);
}

}  // namespace

void matvec_fp32_tc(cfie_op* op, const double2* x, double2* y, int nrhs) {
  if (op->bc == CFIE_SOUND_SOFT) {
    run_blocks<KIND_SOFT>(op, x, y, nrhs);
    return;
  }
  // sound hard (eq. 2 with Maue's identity): S applied to [u, n1 x, n2 x] and
  // D' to x, each with the tensor-core sums, then the spectral derivative
  const int n = op->n;
  const size_t tot = (size_t)n * nrhs;
  cudaStream_t st = op->ctx->stream;
  op->xin32.reserve(sizeof(float2) * tot * 3);
  float2* x32 = op->xin32.as<float2>();
  float2* u32 = x32 + tot;
  float2* t32 = x32 + 2 * tot;
  op->tcv.reserve(sizeof(double2) * tot * 4);
  double2* v = op->tcv.as<double2>();        // [u, n1 x, n2 x], then S of them
  op->tcs.reserve(sizeof(double2) * tot * 4);
  double2* ys = op->tcs.as<double2>();       // S [u, n1 x, n2 x], then D' x
  k_to32_fp32(op, x, x32, tot);
  spectral32_apply(op, x32, u32, nrhs);
  k_hard_inputs<<<nb(tot), 256, 0, st>>>(n, tot, x, u32, op->g, v);
  CFIE_CHECK_LAUNCH();
  run_blocks<KIND_S>(op, v, ys, 3 * nrhs);
  run_blocks<KIND_DP>(op, x, ys + 3 * tot, nrhs);
  k_hard_combine<<<nb(tot), 256, 0, st>>>(n, tot, op->omega, op->eta, op->g, x, ys, ys + 3 * tot,
                                          t32, y);
  CFIE_CHECK_LAUNCH();
  spectral32_accumulate(op, t32, y, nrhs);
}

int tc_take_error(cfie_op* op) {
  int e = 0;
  for (auto& T : op->tc) {
    if (!T.err.p) continue;
    int v = 0;
    CFIE_CHECK_CUDA(cudaMemcpyAsync(&v, T.err.p, sizeof(int), cudaMemcpyDeviceToHost,
                                    op->ctx->stream));
    CFIE_CHECK_CUDA(cudaStreamSynchronize(op->ctx->stream));
    if (v) {
      e = v;
      CFIE_CHECK_CUDA(cudaMemsetAsync(T.err.p, 0, sizeof(int), op->ctx->stream));
    }
  }
  return e;
}
