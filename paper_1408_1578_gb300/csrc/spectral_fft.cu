// Spectral tangential derivative of the sound-hard operator (Maue's identity,
// Section 1) by FFT: for each density column,
//
//     d/dt x = IDFT( i m' DFT(x) ),  m' = m for m < n/2, m - n for m > n/2,
//                                    0 at the Nyquist mode m = n/2,
//
// then divided by |z'| (d/ds).  This is the same operator as the circulant
// c_d = (-1)^d cot(pi d / n) / 2, at O(n log n) instead of O(n^2) per column.
// A DFT of any length n goes through Bluestein's chirp-z identity
//
//     X_m = conj(b_m) sum_j (x_j conj(b_j)) b_(m-j),   b_k = exp(i pi k^2 / n),
//
// a linear convolution computed with power-of-two FFTs of length N >= 2n - 1
// (Stockham radix-2 passes, out of place, twiddles exp(-2 pi i q / N)); the
// inverse DFT is conj(DFT(conj(D))) / n.  The FFT of the wrapped chirp is
// precomputed per operator.  FP64 for the true residuals, FP32 for the inner
// matvecs (same code, element type a template parameter).
#include <algorithm>

#include "internal.h"

namespace {

template <typename T> struct cx;
template <> struct cx<double2> {
  using S = double;
  static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};
template <> struct cx<float2> {
  using S = float;
  static __device__ __forceinline__ float2 make(double a, double b) {
    return make_float2((float)a, (float)b);
  }
};

template <typename T>
__device__ __forceinline__ T cmul(T a, T b) {
  return cx<T>::make(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ T cmulc(T a, T b) {   // a * conj(b)
  return cx<T>::make(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// twiddles exp(-2 pi i q / N), q < N / 2 (FP64 and FP32 copies)
__global__ void k_twiddles(int N, double2* __restrict__ tw, float2* __restrict__ tw32) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N / 2) return;
  double s, c;
  sincospi(-2.0 * q / N, &s, &c);
  tw[q] = make_double2(c, s);
  tw32[q] = make_float2((float)c, (float)s);
}

// chirp b_k = exp(i pi (k^2 mod 2n) / n), k < n (the square reduced exactly in
// integers before the sine and cosine)
__global__ void k_chirp(int n, double2* __restrict__ b, float2* __restrict__ b32) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const long long q = ((long long)k * k) % (2LL * n);
  double s, c;
  sincospi((double)q / n, &s, &c);
  b[k] = make_double2(c, s);
  b32[k] = make_float2((float)c, (float)s);
}

// its wrapped copy B[k] = b_k (k < n), B[N - k] = b_k (0 < k < n), zero elsewhere
__global__ void k_chirp_wrap(int n, int N, const double2* __restrict__ b, double2* __restrict__ B) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double2 v = make_double2(0.0, 0.0);
  if (k < n) v = b[k];
  else if (k > N - n) v = b[N - k];
  B[k] = v;
}

// one Stockham radix-2 pass over `cols` columns of length N (half-size m)
template <typename T>
__global__ void k_fft_pass(int N, int m, int cols, const T* __restrict__ in, T* __restrict__ out,
                           const T* __restrict__ tw, int inverse) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= N / 2 || c >= cols) return;
  const int j = i / m, k = i - j * m;
  T w = tw[(size_t)k * (N / (2 * m))];
  if (inverse) w.y = -w.y;
  const T* a = in + (size_t)c * N;
  T* o = out + (size_t)c * N;
  const T u = a[j * m + k], v = cmul(w, a[j * m + k + N / 2]);
  o[2 * j * m + k] = cx<T>::make(u.x + v.x, u.y + v.y);
  o[2 * j * m + k + m] = cx<T>::make(u.x - v.x, u.y - v.y);
}

// a[c][j] = x[c][j] conj(b_j) for j < n, 0 up to N
template <typename T, typename X>
__global__ void k_bs_pre(int n, int N, int cols, const X* __restrict__ x, const T* __restrict__ b,
                         T* __restrict__ a) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (j >= N) return;
  T v = cx<T>::make(0.0, 0.0);
  if (j < n) {
    const X xv = x[(size_t)c * n + j];
    v = cmulc(cx<T>::make(xv.x, xv.y), b[j]);
  }
  a[(size_t)c * N + j] = v;
}

// a *= Bf (pointwise, every column)
template <typename T>
__global__ void k_bs_mul(int N, int cols, T* __restrict__ a, const T* __restrict__ bf) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (k >= N) return;
  a[(size_t)c * N + k] = cmul(a[(size_t)c * N + k], bf[k]);
}

// X_m = conj(b_m) conv_m / N; D_m = i m' X_m; a2_m = conj(D_m) conj(b_m), 0 up to N
template <typename T>
__global__ void k_bs_mid(int n, int N, int cols, const T* __restrict__ conv,
                         const T* __restrict__ b, T* __restrict__ a2) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (m >= N) return;
  using S = typename cx<T>::S;
  T v = cx<T>::make(0.0, 0.0);
  if (m < n) {
    const T X = cmulc(conv[(size_t)c * N + m], b[m]);
    const S mm = (S)(2 * m < n ? m : (2 * m == n ? 0 : m - n)) / (S)N;
    const T D = cx<T>::make(-mm * X.y, mm * X.x);      // i m' X / N
    v = cmulc(cx<T>::make(D.x, -D.y), b[m]);          // conj(D) conj(b)
  }
  a2[(size_t)c * N + m] = v;
}

// out_j = base_j + (scale / |z'_j|) (1 / n) conj(conj(b_j) conv2_j / N)
template <typename T, typename O>
__global__ void k_bs_out(int n, int N, int cols, const T* __restrict__ conv2,
                         const T* __restrict__ b, const double* __restrict__ sp, double2 scale,
                         const O* __restrict__ base, O* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (j >= n) return;
  const T w = cmulc(conv2[(size_t)c * N + j], b[j]);
  const double f = 1.0 / ((double)n * (double)N * sp[j]);
  const double dx = (double)w.x * f, dy = -(double)w.y * f;     // conj
  double ox = scale.x * dx - scale.y * dy, oy = scale.x * dy + scale.y * dx;
  if (base) {
    const O bv = base[(size_t)c * n + j];
    ox += (double)bv.x;
    oy += (double)bv.y;
  }
  O r;
  r.x = ox;
  r.y = oy;
  out[(size_t)c * n + j] = r;
}

// The whole derivative of one column in one CTA when both length-N work
// buffers fit in shared memory: chirp premultiply, FFT, times Bf, inverse FFT,
// derivative, FFT, times Bf, inverse FFT, output, with barriers between passes.
template <typename T>
__device__ __forceinline__ void smem_fft(int N, int L, T* a, T* b, const T* __restrict__ tw,
                                         int inverse, T*& res) {
  int m = 1;
  for (int p = 0; p < L; ++p, m *= 2) {
    for (int i = threadIdx.x; i < N / 2; i += blockDim.x) {
      const int j = i / m, k = i - j * m;
      T w = tw[(size_t)k * (N / (2 * m))];
      if (inverse) w.y = -w.y;
      const T u = a[j * m + k], v = cmul(w, a[j * m + k + N / 2]);
      b[2 * j * m + k] = cx<T>::make(u.x + v.x, u.y + v.y);
      b[2 * j * m + k + m] = cx<T>::make(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
    T* t = a;
    a = b;
    b = t;
  }
  res = a;
}

template <typename T, typename X, typename O>
__global__ void __launch_bounds__(512)
k_spectral_smem(int n, int N, int L, const X* __restrict__ in, const T* __restrict__ ch,
                const T* __restrict__ bf, const T* __restrict__ tw, const double* __restrict__ sp,
                double2 scale, const O* __restrict__ base, O* __restrict__ out) {
  using S = typename cx<T>::S;
  extern __shared__ __align__(16) unsigned char raw[];
  T* a = reinterpret_cast<T*>(raw);
  T* b = a + N;
  const int c = blockIdx.x;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    T v = cx<T>::make(0.0, 0.0);
    if (j < n) {
      const X xv = in[(size_t)c * n + j];
      v = cmulc(cx<T>::make(xv.x, xv.y), ch[j]);
    }
    a[j] = v;
  }
  __syncthreads();
  T* r;
  smem_fft(N, L, a, b, tw, 0, r);
  for (int k = threadIdx.x; k < N; k += blockDim.x) r[k] = cmul(r[k], bf[k]);
  __syncthreads();
  T* o = r == a ? b : a;
  smem_fft(N, L, r, o, tw, 1, r);
  o = r == a ? b : a;
  for (int m = threadIdx.x; m < N; m += blockDim.x) {
    T v = cx<T>::make(0.0, 0.0);
    if (m < n) {
      const T Xm = cmulc(r[m], ch[m]);
      const S mm = (S)(2 * m < n ? m : (2 * m == n ? 0 : m - n)) / (S)N;
      const T D = cx<T>::make(-mm * Xm.y, mm * Xm.x);
      v = cmulc(cx<T>::make(D.x, -D.y), ch[m]);
    }
    o[m] = v;
  }
  __syncthreads();
  smem_fft(N, L, o, r, tw, 0, r);
  for (int k = threadIdx.x; k < N; k += blockDim.x) r[k] = cmul(r[k], bf[k]);
  __syncthreads();
  o = r == a ? b : a;
  smem_fft(N, L, r, o, tw, 1, r);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const T w = cmulc(r[j], ch[j]);
    const double f = 1.0 / ((double)n * (double)N * sp[j]);
    const double dx = (double)w.x * f, dy = -(double)w.y * f;
    double ox = scale.x * dx - scale.y * dy, oy = scale.x * dy + scale.y * dx;
    if (base) {
      const O bv = base[(size_t)c * n + j];
      ox += (double)bv.x;
      oy += (double)bv.y;
    }
    O q;
    q.x = ox;
    q.y = oy;
    out[(size_t)c * n + j] = q;
  }
}

unsigned nb(size_t len, int t = 256) { return (unsigned)((len + t - 1) / t); }

// FFT of `cols` columns of length N between the two work buffers; returns the
// buffer holding the result
template <typename T>
T* fft(cudaStream_t st, int N, int L, int cols, T* a, T* b, const T* tw, int inverse) {
  int m = 1;
  for (int p = 0; p < L; ++p, m *= 2) {
    k_fft_pass<T><<<dim3(nb(N / 2), cols), 256, 0, st>>>(N, m, cols, a, b, tw, inverse);
    CFIE_CHECK_LAUNCH();
    std::swap(a, b);
  }
  return a;
}

template <typename T>
const T* tw_of(const fft_plan& F);
template <> const double2* tw_of<double2>(const fft_plan& F) { return F.tw.as<double2>(); }
template <> const float2* tw_of<float2>(const fft_plan& F) { return F.tw32.as<float2>(); }
template <typename T>
const T* chirp_of(const fft_plan& F);
template <> const double2* chirp_of<double2>(const fft_plan& F) { return F.chirp.as<double2>(); }
template <> const float2* chirp_of<float2>(const fft_plan& F) { return F.chirp32.as<float2>(); }
template <typename T>
const T* bf_of(const fft_plan& F);
template <> const double2* bf_of<double2>(const fft_plan& F) { return F.bf.as<double2>(); }
template <> const float2* bf_of<float2>(const fft_plan& F) { return F.bf32.as<float2>(); }

__global__ void k_to_f32(size_t len, const double2* __restrict__ a, float2* __restrict__ b) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < len) b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// out = base + scale (1/|z'|) d/dt in, columns of length n, element type T for
// the transforms
template <typename T, typename X, typename O>
void spectral_fft(cfie_op* op, const X* in, O* out, const O* base, double2 scale, int cols) {
  fft_plan& F = op->fft;
  const int n = op->n, N = F.N, L = F.L;
  cudaStream_t st = op->ctx->stream;
  const size_t smem = 2 * sizeof(T) * (size_t)N;
  constexpr size_t kSmemMax = (size_t)128 * 1024;
  if (smem <= kSmemMax) {
    // one CTA per column, everything in shared memory.  The attribute is the
    // bound of this branch, not this launch's size: it is per kernel and
    // process-wide, and operators of other sizes launch the same kernel from
    // other host threads (server slots)
    prof_scope ps(op->ctx, CFIE_K_SPECTRAL);
    CFIE_CHECK_CUDA(cudaFuncSetAttribute(k_spectral_smem<T, X, O>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemMax));
    k_spectral_smem<T, X, O><<<cols, 512, smem, st>>>(n, N, L, in, chirp_of<T>(F), bf_of<T>(F),
                                                     tw_of<T>(F), op->g.sp, scale, base, out);
    CFIE_CHECK_LAUNCH();
    return;
  }
  dbuf& w = sizeof(T) == 16 ? F.work : F.work32;
  w.reserve(sizeof(T) * 2 * (size_t)N * cols);
  T* a = w.as<T>();
  T* b = a + (size_t)N * cols;
  const T* tw = tw_of<T>(F);
  const T* ch = chirp_of<T>(F);
  const T* bf = bf_of<T>(F);
  const dim3 gN(nb(N), cols), gn(nb(n), cols);
  prof_scope ps(op->ctx, CFIE_K_SPECTRAL);
  k_bs_pre<T, X><<<gN, 256, 0, st>>>(n, N, cols, in, ch, a);
  CFIE_CHECK_LAUNCH();
  T* r = fft<T>(st, N, L, cols, a, b, tw, 0);
  k_bs_mul<T><<<gN, 256, 0, st>>>(N, cols, r, bf);
  CFIE_CHECK_LAUNCH();
  T* o = r == a ? b : a;
  r = fft<T>(st, N, L, cols, r, o, tw, 1);
  o = r == a ? b : a;
  k_bs_mid<T><<<gN, 256, 0, st>>>(n, N, cols, r, ch, o);
  CFIE_CHECK_LAUNCH();
  r = fft<T>(st, N, L, cols, o, r, tw, 0);
  k_bs_mul<T><<<gN, 256, 0, st>>>(N, cols, r, bf);
  CFIE_CHECK_LAUNCH();
  o = r == a ? b : a;
  r = fft<T>(st, N, L, cols, r, o, tw, 1);
  k_bs_out<T, O><<<gn, 256, 0, st>>>(n, N, cols, r, ch, op->g.sp, scale, base, out);
  CFIE_CHECK_LAUNCH();
}

}  // namespace

void fft_prepare(cfie_op* op) {
  fft_plan& F = op->fft;
  const int n = op->n;
  int N = 1, L = 0;
  while (N < 2 * n - 1) {
    N *= 2;
    ++L;
  }
  F.N = N;
  F.L = L;
  cudaStream_t st = op->ctx->stream;
  F.tw.reserve(sizeof(double2) * (N / 2));
  F.tw32.reserve(sizeof(float2) * (N / 2));
  F.chirp.reserve(sizeof(double2) * n);
  F.chirp32.reserve(sizeof(float2) * n);
  F.bf.reserve(sizeof(double2) * N);
  F.bf32.reserve(sizeof(float2) * N);
  k_twiddles<<<nb(N / 2), 256, 0, st>>>(N, F.tw.as<double2>(), F.tw32.as<float2>());
  CFIE_CHECK_LAUNCH();
  k_chirp<<<nb(n), 256, 0, st>>>(n, F.chirp.as<double2>(), F.chirp32.as<float2>());
  CFIE_CHECK_LAUNCH();
  // Bf = FFT of the wrapped chirp (FP64), then its FP32 copy
  dbuf tmp;
  tmp.reserve(sizeof(double2) * 2 * (size_t)N);
  double2* a = tmp.as<double2>();
  k_chirp_wrap<<<nb(N), 256, 0, st>>>(n, N, F.chirp.as<double2>(), a);
  CFIE_CHECK_LAUNCH();
  double2* r = fft<double2>(st, N, L, 1, a, a + N, F.tw.as<double2>(), 0);
  CFIE_CHECK_CUDA(cudaMemcpyAsync(F.bf.p, r, sizeof(double2) * N, cudaMemcpyDeviceToDevice, st));
  k_to_f32<<<nb(N), 256, 0, st>>>(N, F.bf.as<double2>(), F.bf32.as<float2>());
  CFIE_CHECK_LAUNCH();
}

void spectral_fft64(cfie_op* op, const double2* in, double2* out, const double2* base,
                    double2 scale, int nrhs) {
  spectral_fft<double2, double2, double2>(op, in, out, base, scale, nrhs);
}

void spectral_fft32_apply(cfie_op* op, const float2* in, float2* out, int nrhs) {
  spectral_fft<float2, float2, float2>(op, in, out, nullptr, make_double2(1.0, 0.0), nrhs);
}

void spectral_fft32_accumulate(cfie_op* op, const float2* in, double2* y, double2 scale,
                               int nrhs) {
  spectral_fft<float2, float2, double2>(op, in, y, y, scale, nrhs);
}
