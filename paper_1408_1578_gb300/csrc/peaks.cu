// Issue-rate probes of the arithmetic pipes the kernels are bound by: FP32
// FMA, the MUFU (special function) unit and FP64 FMA.  Each thread runs
// eight independent dependency chains for a fixed number of iterations; the
// chain results are stored so that nothing is removed as dead code.  The grid
// is 8 CTAs of 256 threads per SM (full occupancy of the issue slots).
#include <algorithm>

#include "internal.h"

namespace {

constexpr int PT = 256;

__global__ void __launch_bounds__(PT) k_fma32(int iters, float a, float b, float* out) {
  float x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * PT + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PT) k_mufu(int iters, float* out) {
  float x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = 1.0f + (float)(threadIdx.x + c) * 1e-3f;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = rsqrtf(x[c]);   // fixed point 1, stays finite
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * PT + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PT) k_fma64(int iters, double a, double b, float* out) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[blockIdx.x * PT + threadIdx.x] = (float)s;
}

}  // namespace

void measure_peaks(cfie_ctx* ctx, cfie_peaks* out) {
  {
    int sms = 0, dev = 0;
    CFIE_CHECK_CUDA(cudaGetDevice(&dev));
    CFIE_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * 8;
    dbuf sink;
    sink.reserve(sizeof(float) * grid * PT);
    float* o = sink.as<float>();
    cudaStream_t st = ctx->stream;
    cudaEvent_t e0, e1;
    CFIE_CHECK_CUDA(cudaEventCreate(&e0));
    CFIE_CHECK_CUDA(cudaEventCreate(&e1));
    auto timed = [&](auto launch) {
      launch();   // warm-up
      CFIE_CHECK_CUDA(cudaEventRecord(e0, st));
      for (int r = 0; r < 3; ++r) launch();
      CFIE_CHECK_CUDA(cudaEventRecord(e1, st));
      CFIE_CHECK_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      CFIE_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      return ms / 3.0 / 1e3;
    };
    const double lanes = (double)grid * PT * 8;
    const int it32 = 1 << 16, itmu = 1 << 13, it64 = 1 << 11;
    const double t32 = timed([&] {
      k_fma32<<<grid, PT, 0, st>>>(it32, 0.999f, 1e-4f, o);
      CFIE_CHECK_LAUNCH();
    });
    const double tmu = timed([&] {
      k_mufu<<<grid, PT, 0, st>>>(itmu, o);
      CFIE_CHECK_LAUNCH();
    });
    const double t64 = timed([&] {
      k_fma64<<<grid, PT, 0, st>>>(it64, 0.999, 1e-4, o);
      CFIE_CHECK_LAUNCH();
    });
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out->sms = sms;
    out->fp32_fma_per_s = lanes * it32 / t32;
    out->mufu_per_s = lanes * itmu / tmu;
    out->fp64_fma_per_s = lanes * it64 / t64;
  }
}
