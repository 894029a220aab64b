// Block GMRES over the right-hand sides of one operator: one Krylov space
//     span{R, A R, A^2 R, ...}
// shared by the s columns of the residual block R, the variant of the Arnoldi
// step Section 3 leaves open (the paper runs one GMRES per incident wave).  The
// plane waves of many directions share most of their Krylov space at high
// frequency, so a block step (one block matvec, the same cost as one step of s
// independent GMRES) gains far more than one dimension per right-hand side.
//
// Block Arnoldi step k (basis V = [V_0 .. V_k], column-major n x p):
//     W = A V_k
//     block classical Gram-Schmidt twice:  H = V^H W,  W -= V H   (two passes)
//     W = V_{k+1} R_k                       (rank-revealing Cholesky QR, twice)
// with the block column [H; R_k] appended to the block Hessenberg matrix, whose
// QR (Householder, updated column by column on the host) gives every column's
// least-squares residual ||E_1 B - Hbar Y|| as the convergence test.  The
// Gram-Schmidt products and the Gram matrices are GEMMs over the n rows on the
// GPU (basis in FP64, or FP32 for the inner solves of the refined precisions,
// with FP64 sums across row chunks); the s x s Cholesky factorisations and the
// least squares, O(s^3) per step, run in FP64 on the host.  Rank deficiency
// (repeated directions, converged columns, a zero right-hand side) is handled by
// the pivoted Cholesky: directions whose Gram diagonal falls below a relative
// threshold are dropped from the next block (deflation), so blocks may shrink.
//
// The refined precisions run the block solve as the inner solve of the
// mixed-precision refinement: r = f - A x with the FP64-accurate matvec, an inner
// block GMRES on A_fast d = r to a per-column tolerance, x += d.
#include <algorithm>
#include <cmath>
#include <complex>
#include <thread>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace {

using cplx = std::complex<double>;

template <typename T> struct bt;
template <> struct bt<double2> {
  using S = double;
  static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};
template <> struct bt<float2> {
  using S = float;
  static __device__ __forceinline__ float2 make(double a, double b) {
    return make_float2((float)a, (float)b);
  }
};

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// Both products use 64 x 64 output tiles, 4 x 4 per thread (16 outputs from
// 4 + 4 shared-memory loads per step of the reduction).
constexpr int BT = 64;       // output tile edge
constexpr int BR = 16;       // reduction rows staged per step
constexpr int IPC = 1024;    // rows per chunk of the inner products (FP64 sums across chunks)

// part[chunk][a][b] = sum over the chunk's rows of conj(X[i, a]) Y[i, b]
// (a < pa, b < pb; X, Y column-major with leading dimension n)
template <typename T>
__global__ void __launch_bounds__(256)
k_bip(int n, int pa, int pb, const T* __restrict__ X, const T* __restrict__ Y,
      double2* __restrict__ part) {
  using S = typename bt<T>::S;
  __shared__ T xs[BR][BT + 1], ys[BR][BT + 1];
  const int a0 = blockIdx.x * BT, b0 = blockIdx.y * BT;
  const int r0 = blockIdx.z * IPC, r1 = min(n, r0 + IPC);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  S are[4][4], aim[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) are[i][j] = aim[i][j] = 0;
  for (int i0 = r0; i0 < r1; i0 += BR) {
    for (int e = threadIdx.x; e < BR * BT; e += 256) {
      const int rr = e % BR, c = e / BR;
      const int i = i0 + rr;
      xs[rr][c] = (i < r1 && a0 + c < pa) ? X[(size_t)(a0 + c) * n + i] : bt<T>::make(0.0, 0.0);
      ys[rr][c] = (i < r1 && b0 + c < pb) ? Y[(size_t)(b0 + c) * n + i] : bt<T>::make(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < BR; ++rr) {
      T u[4], v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        u[q] = xs[rr][ty + 16 * q];
        v[q] = ys[rr][tx + 16 * q];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          are[i][j] = fma(u[i].x, v[j].x, fma(u[i].y, v[j].y, are[i][j]));
          aim[i][j] = fma(u[i].x, v[j].y, fma(-u[i].y, v[j].x, aim[i][j]));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
      if (a < pa && b < pb)
        part[((size_t)blockIdx.z * pa + a) * pb + b] =
            make_double2((double)are[i][j], (double)aim[i][j]);
    }
}

// C[a][b] = sum over chunks of part (fixed order)
__global__ void k_bip_reduce(int chunks, int pa, int pb, const double2* __restrict__ part,
                             double2* __restrict__ C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= pa * pb) return;
  double sr = 0.0, si = 0.0;
  for (int c = 0; c < chunks; ++c) {
    const double2 v = part[(size_t)c * pa * pb + e];
    sr += v.x;
    si += v.y;
  }
  C[e] = make_double2(sr, si);
}

// Y[i, b] = beta Y[i, b] + alpha sum_a X[i, a] M[a][b]  (i < n, b < pb, a < pa;
// M row-major pa x pb in FP64); Y is a different buffer from X
template <typename T>
__global__ void __launch_bounds__(256)
k_bupd(int n, int pa, int pb, const T* __restrict__ X, const double2* __restrict__ M,
       T* __restrict__ Y, double alpha, double beta) {
  using S = typename bt<T>::S;
  __shared__ T xs[BR][BT + 1];   // [a][row]
  __shared__ T ms[BR][BT + 1];   // [a][column]
  const int i0 = blockIdx.x * BT, b0 = blockIdx.y * BT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  S are[4][4], aim[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) are[i][j] = aim[i][j] = 0;
  for (int k0 = 0; k0 < pa; k0 += BR) {
    for (int e = threadIdx.x; e < BR * BT; e += 256) {
      const int r = e % BT, k = e / BT;
      const int i = i0 + r, a = k0 + k;
      xs[k][r] = (i < n && a < pa) ? X[(size_t)a * n + i] : bt<T>::make(0.0, 0.0);
      const int c = e % BT, kk = e / BT;
      const int aa = k0 + kk, bb = b0 + c;
      const double2 v = (aa < pa && bb < pb) ? M[(size_t)aa * pb + bb] : make_double2(0.0, 0.0);
      ms[kk][c] = bt<T>::make(v.x, v.y);
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < BR; ++k) {
      T x[4], m[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        x[q] = xs[k][ty + 16 * q];
        m[q] = ms[k][tx + 16 * q];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          are[i][j] = fma(x[i].x, m[j].x, fma(-x[i].y, m[j].y, are[i][j]));
          aim[i][j] = fma(x[i].x, m[j].y, fma(x[i].y, m[j].x, aim[i][j]));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int row = i0 + ty + 16 * i;
    if (row >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int b = b0 + tx + 16 * j;
      if (b >= pb) continue;
      const size_t o = (size_t)b * n + row;
      double yr = alpha * (double)are[i][j], yi = alpha * (double)aim[i][j];
      if (beta != 0.0) {
        const T y = Y[o];
        yr += beta * (double)y.x;
        yi += beta * (double)y.y;
      }
      Y[o] = bt<T>::make(yr, yi);
    }
  }
}

// per-column squared 2-norms in FP64 (one CTA per column)
__global__ void k_colnorm2(int n, const double2* __restrict__ x, double* __restrict__ out) {
  __shared__ double red[32];
  const double2* v = x + (size_t)blockIdx.x * n;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i].x * v[i].x + v[i].y * v[i].y;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

__global__ void k_bsub(size_t len, const double2* __restrict__ f, const double2* __restrict__ ax,
                       double2* __restrict__ r) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < len) r[e] = make_double2(f[e].x - ax[e].x, f[e].y - ax[e].y);
}
__global__ void k_badd(size_t len, const double2* __restrict__ d, double2* __restrict__ x) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < len) x[e] = make_double2(x[e].x + d[e].x, x[e].y + d[e].y);
}
template <typename A, typename B>
__global__ void k_bconv(size_t len, const A* __restrict__ x, B* __restrict__ y) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < len) y[e] = bt<B>::make((double)x[e].x, (double)x[e].y);
}

unsigned nbl(size_t len, int t = 256) { return (unsigned)((len + t - 1) / t); }

// ---------------------------------------------------------------------------
// host: small dense linear algebra in FP64
// ---------------------------------------------------------------------------
// Cholesky with diagonal pivoting of the Hermitian positive semi-definite
// c x c matrix G (row-major): G[P, P] ~ R^H R with R (r x c, upper trapezoidal
// in pivoted order); stops at the first pivot below thresh * (largest
// diagonal).  Returns r; perm[j] is the column of G at pivoted position j.
int chol_pivoted(std::vector<cplx> G, int c, double thresh, std::vector<cplx>& R,
                 std::vector<int>& perm) {
  perm.resize(c);
  for (int j = 0; j < c; ++j) perm[j] = j;
  double dmax = 0.0;
  for (int j = 0; j < c; ++j) dmax = std::max(dmax, G[(size_t)j * c + j].real());
  R.assign((size_t)c * c, cplx(0.0));
  if (!(dmax > 0.0)) return 0;
  int r = 0;
  for (int j = 0; j < c; ++j) {
    int p = j;
    double best = G[(size_t)j * c + j].real();
    for (int q = j + 1; q < c; ++q)
      if (G[(size_t)q * c + q].real() > best) best = G[(size_t)q * c + q].real(), p = q;
    if (!(best > thresh * dmax)) break;
    if (p != j) {   // symmetric swap of rows / columns j and p, and of R's columns
      for (int q = 0; q < c; ++q) std::swap(G[(size_t)j * c + q], G[(size_t)p * c + q]);
      for (int q = 0; q < c; ++q) std::swap(G[(size_t)q * c + j], G[(size_t)q * c + p]);
      for (int q = 0; q < j; ++q) std::swap(R[(size_t)q * c + j], R[(size_t)q * c + p]);
      std::swap(perm[j], perm[p]);
    }
    const double d = std::sqrt(best);
    R[(size_t)j * c + j] = d;
    for (int q = j + 1; q < c; ++q) R[(size_t)j * c + q] = G[(size_t)j * c + q] / d;
    // Schur complement of the remaining block: the upper triangle, then its
    // mirror (the block stays Hermitian)
    for (int a = j + 1; a < c; ++a) {
      const cplx ra = std::conj(R[(size_t)j * c + a]);
      cplx* ga = &G[(size_t)a * c];
      const cplx* rj = &R[(size_t)j * c];
      for (int b = a; b < c; ++b) ga[b] -= ra * rj[b];
      for (int b = a + 1; b < c; ++b) G[(size_t)b * c + a] = std::conj(ga[b]);
    }
    ++r;
  }
  return r;
}

// Cholesky G = S^H S of a Hermitian positive definite r x r matrix (S upper
// triangular, row-major); false if a pivot is not positive
bool chol_plain(const std::vector<cplx>& G, int r, std::vector<cplx>& S) {
  S.assign((size_t)r * r, cplx(0.0));
  for (int j = 0; j < r; ++j) {
    double d = G[(size_t)j * r + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(S[(size_t)k * r + j]);
    if (!(d > 0.0)) return false;
    const double dd = std::sqrt(d);
    S[(size_t)j * r + j] = dd;
    for (int q = j + 1; q < r; ++q) {
      cplx v = G[(size_t)j * r + q];
      for (int k = 0; k < j; ++k) v -= std::conj(S[(size_t)k * r + j]) * S[(size_t)k * r + q];
      S[(size_t)j * r + q] = v / dd;
    }
  }
  return true;
}

// inverse of the r x r upper triangular leading block of R (row-major, c
// columns), as an r x r row-major matrix
std::vector<cplx> upper_inverse(const std::vector<cplx>& R, int c, int r) {
  std::vector<cplx> X((size_t)r * r, cplx(0.0));
  for (int j = 0; j < r; ++j) {
    X[(size_t)j * r + j] = 1.0 / R[(size_t)j * c + j];
    for (int i = j - 1; i >= 0; --i) {
      cplx s = 0.0;
      for (int k = i + 1; k <= j; ++k) s += R[(size_t)i * c + k] * X[(size_t)k * r + j];
      X[(size_t)i * r + j] = -s / R[(size_t)i * c + i];
    }
  }
  return X;
}

// f(i) for i < count on up to 8 host threads (sequentially when the work is
// small: `work` is the number of complex multiply-adds it takes)
template <typename F>
void parallel_for(int count, double work, F f) {
  int nt = (int)std::min<unsigned>(8u, std::max(1u, std::thread::hardware_concurrency()));
  nt = std::min(nt, count);
  if (nt <= 1 || work < 2e5) {
    for (int i = 0; i < count; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([=, &f] {
      for (int i = t; i < count; i += nt) f(i);
    });
  for (auto& x : th) x.join();
}

// Least squares of the block Hessenberg system, QR by Householder reflections
// added column by column: min over Y of ||G - Hbar Y|| per right-hand-side
// column, with G = [B; 0].
struct block_ls {
  int s = 0;                          // right-hand-side columns
  int rows = 0, cols = 0;             // current size of Hbar
  std::vector<std::vector<cplx>> Rc;  // columns of the triangular factor (length cols_j + 1)
  std::vector<std::vector<cplx>> hv;  // reflectors: vector over rows [start, start + len)
  std::vector<int> hstart;
  std::vector<double> htau;
  std::vector<std::vector<cplx>> G;   // transformed right-hand sides, per column of B

  void start(const std::vector<cplx>& B, int r0, int s_) {   // B: r0 x s_, row-major
    s = s_;
    rows = r0;
    cols = 0;
    Rc.clear();
    hv.clear();
    hstart.clear();
    htau.clear();
    G.assign(s, std::vector<cplx>());
    for (int b = 0; b < s; ++b) {
      G[b].assign(r0, cplx(0.0));
      for (int i = 0; i < r0; ++i) G[b][i] = B[(size_t)i * s + b];
    }
  }
  static void reflect(const std::vector<cplx>& v, int st, double tau, std::vector<cplx>& x) {
    cplx d = 0.0;
    for (size_t q = 0; q < v.size(); ++q) d += std::conj(v[q]) * x[st + q];
    d *= tau;
    for (size_t q = 0; q < v.size(); ++q) x[st + q] -= v[q] * d;
  }
  // new rows (zero in every earlier column), then one column of length rows
  void grow(int new_rows) {
    rows = new_rows;
    for (auto& g : G) g.resize(rows, cplx(0.0));
  }
  // a block of columns (each of length rows): the earlier reflectors applied
  // to all of them in parallel, then column by column the block's own ones and
  // a new reflector, which are applied to the right-hand sides in parallel
  void add_block(std::vector<std::vector<cplx>>& B) {
    const size_t nprev = hv.size();
    const int nb = (int)B.size();
    double len = 0.0;
    for (size_t j = 0; j < nprev; ++j) len += (double)hv[j].size();
    parallel_for(nb, len * nb, [&](int c) {
      for (size_t j = 0; j < nprev; ++j) reflect(hv[j], hstart[j], htau[j], B[c]);
    });
    for (int c = 0; c < nb; ++c) {
      for (size_t j = nprev; j < hv.size(); ++j) reflect(hv[j], hstart[j], htau[j], B[c]);
      new_reflector(B[c]);
    }
    double blen = 0.0;
    for (size_t j = nprev; j < hv.size(); ++j) blen += (double)hv[j].size();
    parallel_for(s, blen * s, [&](int b) {
      for (size_t j = nprev; j < hv.size(); ++j) reflect(hv[j], hstart[j], htau[j], G[b]);
    });
  }
  // the reflector that zeroes column `cols` below its diagonal (earlier
  // reflectors already applied); the right-hand sides are left to the caller
  void new_reflector(const std::vector<cplx>& col) {
    const int j = cols;
    double nrm2 = 0.0;
    for (int q = j; q < rows; ++q) nrm2 += std::norm(col[q]);
    const double nrm = std::sqrt(nrm2);
    std::vector<cplx> v(rows - j);
    for (int q = j; q < rows; ++q) v[q - j] = col[q];
    const cplx x0 = col[j];
    const cplx ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cplx(1.0);
    const cplx alpha = -ph * nrm;
    v[0] -= alpha;
    double vn2 = 0.0;
    for (const cplx& c : v) vn2 += std::norm(c);
    const double tau = vn2 > 0 ? 2.0 / vn2 : 0.0;
    std::vector<cplx> rc(j + 1);
    for (int q = 0; q < j; ++q) rc[q] = col[q];
    rc[j] = vn2 > 0 ? alpha : x0;
    Rc.push_back(rc);
    hv.push_back(v);
    hstart.push_back(j);
    htau.push_back(tau);
    ++cols;
  }
  double residual(int b) const {
    double t = 0.0;
    for (int q = cols; q < rows; ++q) t += std::norm(G[b][q]);
    return std::sqrt(t);
  }
  // Y (cols x s, row-major) from the triangular system, by columns of R (each
  // stored contiguously): y_i = g_i / R_ii, then g_q -= R_qi y_i for q < i
  std::vector<cplx> solve() const {
    std::vector<cplx> Y((size_t)cols * s, cplx(0.0));
    parallel_for(s, 0.5 * (double)cols * cols * s, [&](int b) {
      std::vector<cplx> y(G[b].begin(), G[b].begin() + cols);
      for (int i = cols - 1; i >= 0; --i) {
        const std::vector<cplx>& ri = Rc[i];
        const cplx yi = y[i] / ri[i];
        y[i] = yi;
        for (int q = 0; q < i; ++q) y[q] -= ri[q] * yi;
      }
      for (int i = 0; i < cols; ++i) Y[(size_t)i * s + b] = y[i];
    });
    return Y;
  }
};

// ---------------------------------------------------------------------------
// host: the block solve
// ---------------------------------------------------------------------------
template <typename T>
struct bg_ws {
  int n = 0, s = 0, cap = 0;     // rows, right-hand sides, basis columns
  T* V = nullptr;                // basis, n x cap
  T* W = nullptr;                // n x s
  T* Q = nullptr;                // n x s (orthonormalisation output)
  double2* vin = nullptr;        // matvec input / output (n x s each)
  double2* vout = nullptr;
  double2* part = nullptr;       // inner-product partials
  double2* small = nullptr;      // cap x s FP64 matrices (Y, Z, Gram)
  double2 *H1 = nullptr, *H2 = nullptr;   // the two Gram-Schmidt coefficient blocks
  double* nrm = nullptr;
  int chunks = 0;
};

struct bg_ctx {
  cfie_op* op;
  cudaStream_t st;
  bool refined;
  std::function<void(const double2*, double2*, int)> mv;   // y = A_x x for c columns
  std::function<void(const double2*, double2*, int)> prec; // right preconditioner (may be empty)
};

// Hd (device, pa x pb row-major FP64) = X^H Y; asynchronous
template <typename T>
void ip_dev(const bg_ctx& C, const bg_ws<T>& w, const T* X, int pa, const T* Y, int pb,
            double2* Hd) {
  prof_scope ps(C.op->ctx, CFIE_K_ARNOLDI);
  const dim3 grid((unsigned)((pa + BT - 1) / BT), (unsigned)((pb + BT - 1) / BT),
                  (unsigned)w.chunks);
  k_bip<T><<<grid, 256, 0, C.st>>>(w.n, pa, pb, X, Y, w.part);
  CFIE_CHECK_LAUNCH();
  k_bip_reduce<<<nbl((size_t)pa * pb), 256, 0, C.st>>>(w.chunks, pa, pb, w.part, Hd);
  CFIE_CHECK_LAUNCH();
}

// Y = beta Y + alpha X Md (Md device, pa x pb row-major FP64); asynchronous
template <typename T>
void upd_dev(const bg_ctx& C, const bg_ws<T>& w, const T* X, int pa, const double2* Md, int pb,
             T* Y, double alpha, double beta) {
  prof_scope ps(C.op->ctx, CFIE_K_ARNOLDI);
  const dim3 grid((unsigned)((w.n + BT - 1) / BT), (unsigned)((pb + BT - 1) / BT));
  k_bupd<T><<<grid, 256, 0, C.st>>>(w.n, pa, pb, X, Md, Y, alpha, beta);
  CFIE_CHECK_LAUNCH();
}

// the same with the result (or the matrix) on the host; synchronous
template <typename T>
void inner_products(const bg_ctx& C, const bg_ws<T>& w, const T* X, int pa, const T* Y, int pb,
                    std::vector<cplx>& out) {
  ip_dev(C, w, X, pa, Y, pb, w.small);
  out.resize((size_t)pa * pb);
  CFIE_CHECK_CUDA(cudaMemcpyAsync(out.data(), w.small, sizeof(double2) * pa * pb,
                                  cudaMemcpyDeviceToHost, C.st));
  CFIE_CHECK_CUDA(cudaStreamSynchronize(C.st));
}

template <typename T>
void update(const bg_ctx& C, const bg_ws<T>& w, const T* X, int pa, const std::vector<cplx>& M,
            int pb, T* Y, double alpha, double beta) {
  CFIE_CHECK_CUDA(cudaMemcpyAsync(w.small, M.data(), sizeof(double2) * pa * pb,
                                  cudaMemcpyHostToDevice, C.st));
  upd_dev(C, w, X, pa, w.small, pb, Y, alpha, beta);
  CFIE_CHECK_CUDA(cudaStreamSynchronize(C.st));   // M dies on return
}

// The factors of one block QR: W P = Q1 R (pivoted Cholesky QR), Q1 = Q2 S
// (the second pass); R_out = S R P^T follows from them (qr_rout).
struct qr_parts {
  int r = 0, c = 0;
  std::vector<cplx> R, S;
  std::vector<int> perm;
};

// W (c columns) = Q R_out, R_out r x c row-major, from the factors
std::vector<cplx> qr_rout(const qr_parts& f) {
  const int r = f.r, c = f.c;
  std::vector<cplx> RP((size_t)r * c, cplx(0.0));
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < c; ++j) RP[(size_t)i * c + f.perm[j]] = f.R[(size_t)i * c + j];
  std::vector<cplx> Rout((size_t)r * c, cplx(0.0));
  for (int i = 0; i < r; ++i)
    for (int k = i; k < r; ++k) {
      const cplx a = f.S[(size_t)i * r + k];
      for (int j = 0; j < c; ++j) Rout[(size_t)i * c + j] += a * RP[(size_t)k * c + j];
    }
  return Rout;
}

// W (c columns) = Q R_out with Q written to `dst` (r orthonormal columns);
// returns r (0: W is numerically zero) and the factors of R_out.
template <typename T>
int block_qr(const bg_ctx& C, bg_ws<T>& w, T* Wc, int c, T* dst, double thresh, qr_parts& f) {
  std::vector<cplx> G, R;
  std::vector<int> perm;
  inner_products(C, w, Wc, c, Wc, c, G);
  const int r = chol_pivoted(G, c, thresh, R, perm);
  f.r = r;
  f.c = c;
  if (r == 0) return 0;
  // Z = P[:, :r] R11^-1: column j of Z is R11^-1's column j placed on the pivoted rows
  const std::vector<cplx> R11i = upper_inverse(R, c, r);
  std::vector<cplx> Z((size_t)c * r, cplx(0.0));
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) Z[(size_t)perm[i] * r + j] = R11i[(size_t)i * r + j];
  update(C, w, Wc, c, Z, r, w.Q, 1.0, 0.0);
  // second pass on Q (well conditioned: a plain Cholesky)
  inner_products(C, w, w.Q, r, w.Q, r, G);
  std::vector<cplx> S;   // Q = Q2 S
  if (!chol_plain(G, r, S)) throw cfie_error(CFIE_ECUDA, "block GMRES: orthonormalisation lost rank");
  const std::vector<cplx> Si = upper_inverse(S, r, r);
  update(C, w, w.Q, r, Si, r, dst, 1.0, 0.0);
  // W P = Q R  ->  W = Q (R P^T), then Q = Q2 S: W = Q2 (S R P^T)
  f.R = std::move(R);
  f.S = std::move(S);
  f.perm = std::move(perm);
  return r;
}

// One cycle: basis from the residual block r (n x s, FP64), x_upd += V Y (or
// P V Y).  tol[b]: absolute targets of the least-squares residuals.  Returns
// the block steps taken; *met is set when every column met its target.
template <typename T>
int cycle(const bg_ctx& C, bg_ws<T>& w, const double2* r, const std::vector<double>& tol,
          int max_blocks, double thresh, double2* x_upd, bool* met, cfie_solve_stats& stats) {
  const int n = w.n, s = w.s;
  *met = false;
  // first block: QR of the residual
  k_bconv<double2, T><<<nbl((size_t)n * s), 256, 0, C.st>>>((size_t)n * s, r, w.W);
  CFIE_CHECK_LAUNCH();
  qr_parts f0;
  const int r0 = block_qr(C, w, w.W, s, w.V, thresh, f0);
  if (r0 == 0) {
    *met = true;
    return 0;
  }
  const std::vector<cplx> B = qr_rout(f0);
  block_ls ls;
  ls.start(B, r0, s);
  std::vector<int> bsz{r0};   // block sizes
  int p = r0, steps = 0;
  stats.cycles++;
  // W = A (P) V_k for the newest block, queued on the stream without waiting
  auto queue_matvec = [&](int pk, int sk) {
    const T* Vk = w.V + (size_t)(pk - sk) * n;
    k_bconv<T, double2><<<nbl((size_t)n * sk), 256, 0, C.st>>>((size_t)n * sk, Vk, w.vin);
    CFIE_CHECK_LAUNCH();
    if (C.prec) {
      C.prec(w.vin, w.vout, sk);
      C.mv(w.vout, w.vin, sk);
      k_bconv<double2, T><<<nbl((size_t)n * sk), 256, 0, C.st>>>((size_t)n * sk, w.vin, w.W);
    } else {
      C.mv(w.vin, w.vout, sk);
      k_bconv<double2, T><<<nbl((size_t)n * sk), 256, 0, C.st>>>((size_t)n * sk, w.vout, w.W);
    }
    CFIE_CHECK_LAUNCH();
  };
  queue_matvec(p, r0);
  while (true) {
    const int sk = bsz.back();
    // the matvec of block k is queued (first block above, later ones ahead of
    // the previous step's least-squares update)
    if (C.refined)
      stats.inner_matvecs++;
    else
      stats.fp64_matvecs++;
    // block CGS2 against V[:, :p], the coefficients staying on the device
    ip_dev(C, w, w.V, p, w.W, sk, w.H1);
    upd_dev(C, w, w.V, p, w.H1, sk, w.W, -1.0, 1.0);
    ip_dev(C, w, w.V, p, w.W, sk, w.H2);
    upd_dev(C, w, w.V, p, w.H2, sk, w.W, -1.0, 1.0);
    std::vector<cplx> H1((size_t)p * sk), H2((size_t)p * sk);
    CFIE_CHECK_CUDA(cudaMemcpyAsync(H1.data(), w.H1, sizeof(double2) * p * sk,
                                    cudaMemcpyDeviceToHost, C.st));
    CFIE_CHECK_CUDA(cudaMemcpyAsync(H2.data(), w.H2, sizeof(double2) * p * sk,
                                    cudaMemcpyDeviceToHost, C.st));
    stats.arnoldi_elems += 4LL * (long long)n * p * sk;
    const bool room = p + s <= w.cap;
    qr_parts fk;
    int rn = 0;
    if (room) rn = block_qr(C, w, w.W, sk, w.V + (size_t)p * n, thresh, fk);
    // the next block's matvec goes to the GPU before the host forms R_k and
    // updates the least squares, so the two overlap; if this step ends the
    // cycle, its result is simply not read (the stream orders every later use
    // of W)
    if (rn > 0 && steps + 1 < max_blocks) queue_matvec(p + rn, rn);
    const std::vector<cplx> Rk = rn > 0 ? qr_rout(fk) : std::vector<cplx>();
    // block column [H; R_k] into the least squares
    ls.grow(p + rn);
    std::vector<std::vector<cplx>> blk(sk, std::vector<cplx>(p + rn, cplx(0.0)));
    for (int j = 0; j < sk; ++j) {
      for (int i = 0; i < p; ++i) blk[j][i] = H1[(size_t)i * sk + j] + H2[(size_t)i * sk + j];
      for (int i = 0; i < rn; ++i) blk[j][p + i] = Rk[(size_t)i * sk + j];
    }
    ls.add_block(blk);
    ++steps;
    stats.arnoldi_steps++;
    bool all = true;
    for (int b = 0; b < s; ++b) all = all && ls.residual(b) <= tol[b];
    if (all) *met = true;
    if (all || rn == 0 || steps >= max_blocks || !room) {
      // x_upd += V[:, :cols] Y (cols = columns with Hbar entries)
      const std::vector<cplx> Y = ls.solve();
      const int cols = ls.cols;
      if (C.prec) {
        update(C, w, w.V, cols, Y, s, w.W, 1.0, 0.0);
        k_bconv<T, double2><<<nbl((size_t)n * s), 256, 0, C.st>>>((size_t)n * s, w.W, w.vin);
        CFIE_CHECK_LAUNCH();
        C.prec(w.vin, w.vout, s);
        k_badd<<<nbl((size_t)n * s), 256, 0, C.st>>>((size_t)n * s, w.vout, x_upd);
        CFIE_CHECK_LAUNCH();
      } else {
        update(C, w, w.V, cols, Y, s, w.W, 1.0, 0.0);
        k_bconv<T, double2><<<nbl((size_t)n * s), 256, 0, C.st>>>((size_t)n * s, w.W, w.vin);
        CFIE_CHECK_LAUNCH();
        k_badd<<<nbl((size_t)n * s), 256, 0, C.st>>>((size_t)n * s, w.vin, x_upd);
        CFIE_CHECK_LAUNCH();
      }
      return steps;
    }
    bsz.push_back(rn);
    p += rn;
  }
}

void col_norms(const bg_ctx& C, int n, int s, const double2* v, double* dnrm,
               std::vector<double>& out) {
  k_colnorm2<<<s, 256, 0, C.st>>>(n, v, dnrm);
  CFIE_CHECK_LAUNCH();
  out.resize(s);
  CFIE_CHECK_CUDA(cudaMemcpyAsync(out.data(), dnrm, sizeof(double) * s, cudaMemcpyDeviceToHost, C.st));
  CFIE_CHECK_CUDA(cudaStreamSynchronize(C.st));
  for (double& v2 : out) v2 = std::sqrt(v2);
}

template <typename T>
void solve_impl(cfie_op* op, const double2* f, double2* x, int s, double rtol, int restart,
                int maxit, int* iters, double* relres, cfie_status* status, bool refined,
                dbuf& wsb) {
  const int n = op->n;
  cudaStream_t st = op->ctx->stream;
  bg_ctx C{op, st, refined, nullptr, nullptr};
  if (refined)
    C.mv = [op](const double2* a, double2* b, int c) { apply_inner(op, a, b, c); };
  else
    C.mv = [op](const double2* a, double2* b, int c) { matvec_fp64(op, a, b, c); };
  if (op->dirprec) {
    cfie_dirprec* P = op->dirprec;
    C.prec = [P](const double2* a, double2* b, int c) { dirprec_apply(P, a, b, c); };
  }
  auto fp64_mv = [op](const double2* a, double2* b, int c) { matvec_residual(op, a, b, c); };
  const int blocks = restart > 0 ? restart : maxit;
  bg_ws<T> w;
  w.n = n;
  w.s = s;
  w.cap = std::max(s, std::min(blocks + 1, 512) * s);
  w.chunks = (n + IPC - 1) / IPC;
  const size_t nv = (size_t)n * s;
  const size_t bytes = sizeof(T) * ((size_t)n * w.cap + 2 * nv) + sizeof(double2) * (2 * nv) +
                       sizeof(double2) * ((size_t)w.chunks * w.cap * s + 3 * (size_t)w.cap * s) +
                       sizeof(double) * s + 10 * 256;
  wsb.reserve(bytes);
  char* b = wsb.as<char>();
  size_t o = 0;
  auto take = [&](size_t by) {
    void* at = b + o;
    o += (by + 255) & ~size_t(255);
    return at;
  };
  w.V = static_cast<T*>(take(sizeof(T) * (size_t)n * w.cap));
  w.W = static_cast<T*>(take(sizeof(T) * nv));
  w.Q = static_cast<T*>(take(sizeof(T) * nv));
  w.vin = static_cast<double2*>(take(sizeof(double2) * nv));
  w.vout = static_cast<double2*>(take(sizeof(double2) * nv));
  w.part = static_cast<double2*>(take(sizeof(double2) * (size_t)w.chunks * w.cap * s));
  w.small = static_cast<double2*>(take(sizeof(double2) * (size_t)w.cap * s));
  w.H1 = static_cast<double2*>(take(sizeof(double2) * (size_t)w.cap * s));
  w.H2 = static_cast<double2*>(take(sizeof(double2) * (size_t)w.cap * s));
  w.nrm = static_cast<double*>(take(sizeof(double) * s));
  // outer vectors: residual r, correction d (refined), A x
  op->K.r.reserve(sizeof(double2) * nv);
  op->K.d.reserve(sizeof(double2) * nv);
  op->K.w.reserve(sizeof(double2) * nv);
  double2* r = op->K.r.as<double2>();
  double2* d = op->K.d.as<double2>();
  double2* ax = op->K.w.as<double2>();
  cfie_solve_stats& stats = op->stats;
  stats = cfie_solve_stats{};
  stats.basis_fp32 = std::is_same<T, float2>::value ? 1 : 0;
  // pivots of the Gram matrix below this fraction of its largest diagonal are
  // dropped: Cholesky QR resolves singular values down to about sqrt(eps) of
  // the largest in FP64 Gram arithmetic (and to the FP32 data's own precision
  // with an FP32 basis), and the second pass then restores orthogonality
  const double thresh = std::is_same<T, float2>::value ? 1e-10 : 1e-14;

  std::vector<double> fn, rn, xn;
  col_norms(C, n, s, f, w.nrm, fn);
  col_norms(C, n, s, x, w.nrm, xn);
  bool xz = true;
  for (double v : xn) xz = xz && v == 0.0;
  auto true_residual = [&]() {
    stats.fp64_matvecs++;
    fp64_mv(x, ax, s);
    k_bsub<<<nbl(nv), 256, 0, st>>>(nv, f, ax, r);
    CFIE_CHECK_LAUNCH();
    col_norms(C, n, s, r, w.nrm, rn);
  };
  if (xz) {
    CFIE_CHECK_CUDA(cudaMemcpyAsync(r, f, sizeof(double2) * nv, cudaMemcpyDeviceToDevice, st));
    rn = fn;
  } else {
    true_residual();
  }
  int steps = 0;
  auto converged = [&]() {
    for (int q = 0; q < s; ++q)
      if (rn[q] > rtol * (fn[q] > 0 ? fn[q] : 1.0) && fn[q] > 0) return false;
    return true;
  };
  for (int outer = 0; outer < 64 && !converged() && steps < maxit; ++outer) {
    std::vector<double> tol(s);
    if (refined) {
      stats.refinements++;
      for (int q = 0; q < s; ++q) {
        double tau = rn[q] > 0 ? 0.3 * rtol * fn[q] / rn[q] : 1.0;
        tau = std::min(0.5, std::max(1e-4, tau));
        tol[q] = tau * rn[q];
      }
      CFIE_CHECK_CUDA(cudaMemsetAsync(d, 0, sizeof(double2) * nv, st));
      // inner cycles on A_fast d = r, restarted from the inner residual
      op->K.rin.reserve(sizeof(double2) * nv);
      double2* rin = op->K.rin.as<double2>();
      CFIE_CHECK_CUDA(cudaMemcpyAsync(rin, r, sizeof(double2) * nv, cudaMemcpyDeviceToDevice, st));
      for (int cyc = 0; cyc < 64 && steps < maxit; ++cyc) {
        bool met = false;
        steps += cycle(C, w, rin, tol, std::min(blocks, maxit - steps), thresh, d, &met, stats);
        if (met) break;
        stats.inner_matvecs++;
        C.mv(d, ax, s);   // inner residual r - A_fast d (unpreconditioned d)
        k_bsub<<<nbl(nv), 256, 0, st>>>(nv, r, ax, rin);
        CFIE_CHECK_LAUNCH();
        std::vector<double> irn;
        col_norms(C, n, s, rin, w.nrm, irn);
        bool all = true;
        for (int q = 0; q < s; ++q) all = all && irn[q] <= tol[q];
        if (all) break;
      }
      k_badd<<<nbl(nv), 256, 0, st>>>(nv, d, x);
      CFIE_CHECK_LAUNCH();
    } else {
      for (int q = 0; q < s; ++q) tol[q] = rtol * fn[q];
      bool met = false;
      steps += cycle(C, w, r, tol, std::min(blocks, maxit - steps), thresh, x, &met, stats);
    }
    true_residual();
  }
  *status = CFIE_OK;
  for (int q = 0; q < s; ++q) {
    const double rel = fn[q] > 0 ? rn[q] / fn[q] : 0.0;
    if (relres) relres[q] = rel;
    if (iters) iters[q] = steps;
    if (!(rel <= rtol)) *status = CFIE_ENOCONV;
  }
}

}  // namespace

void block_gmres_solve(cfie_op* op, const double2* f, double2* x, int nrhs, double rtol,
                       int restart, int maxit, int* iters, double* relres, cfie_status* status,
                       dbuf& ws) {
  const bool refined = op->prec != CFIE_FP64;
  if (refined && op->basis32)
    solve_impl<float2>(op, f, x, nrhs, rtol, restart, maxit, iters, relres, status, true, ws);
  else
    solve_impl<double2>(op, f, x, nrhs, rtol, restart, maxit, iters, relres, status, refined, ws);
}
