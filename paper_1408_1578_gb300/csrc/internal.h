// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cfie.h"

#define CFIE_PI 3.14159265358979323846
#define CFIE_EULER 0.57721566490153286061

// ----------------------------------------------------------------------------
// error plumbing
// ----------------------------------------------------------------------------
struct cfie_error : public std::exception {
  cfie_status code;
  std::string msg;
  cfie_error(cfie_status c, std::string m) : code(c), msg(std::move(m)) {}
  const char* what() const noexcept override { return msg.c_str(); }
};

#define CFIE_CHECK_CUDA(call)                                                          \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      throw cfie_error(e_ == cudaErrorMemoryAllocation ? CFIE_ENOMEM : CFIE_ECUDA,     \
                       std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

#include <atomic>
extern std::atomic<long long> g_cfie_launches;  // kernel launches issued by the library
#define CFIE_CHECK_LAUNCH()                 \
  do {                                      \
    ++g_cfie_launches;                      \
    CFIE_CHECK_CUDA(cudaGetLastError());    \
  } while (0)

#define CFIE_REQUIRE(cond, msg)                                  \
  do {                                                           \
    if (!(cond)) throw cfie_error(CFIE_EINVAL, (msg));           \
  } while (0)

// ----------------------------------------------------------------------------
// device buffer owned by the library
// ----------------------------------------------------------------------------
// Stream on which the calling thread's library work is ordered.  Device
// buffers are allocated and freed on it through the device's stream-ordered
// memory pool: a buffer freed after its last use on that stream is reused at
// once by later work, without the device-wide synchronisation and address
// mapping of cudaMalloc / cudaFree.  Entry points set it to the context
// stream (stream_scope); 0 (the legacy default stream) outside them.
inline cudaStream_t& alloc_stream() {
  static thread_local cudaStream_t s = nullptr;
  return s;
}
struct stream_scope {
  cudaStream_t prev;
  explicit stream_scope(cudaStream_t s) : prev(alloc_stream()) { alloc_stream() = s; }
  ~stream_scope() { alloc_stream() = prev; }
  stream_scope(const stream_scope&) = delete;
  stream_scope& operator=(const stream_scope&) = delete;
};

struct dbuf {
  void* p = nullptr;
  size_t bytes = 0;
  dbuf() = default;
  dbuf(const dbuf&) = delete;
  dbuf& operator=(const dbuf&) = delete;
  ~dbuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, alloc_stream());
    p = nullptr;
    bytes = 0;
  }
  // grow to at least `need` bytes (contents not kept)
  void reserve(size_t need) {
    if (need <= bytes) return;
    release();
    CFIE_CHECK_CUDA(cudaMallocAsync(&p, need, alloc_stream()));
    bytes = need;
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

// ----------------------------------------------------------------------------
// handles
// ----------------------------------------------------------------------------
struct cfie_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  // per-launch event timing
  bool profiling = false;
  int prof_suspend = 0;   // > 0: per-launch scopes are off (an outer scope times the work)
  bool tune_batches = true;   // time the contraction's work dealings per batch shape
  struct pending { int cls; cudaEvent_t a, b; };
  std::vector<pending> inflight;
  std::vector<cudaEvent_t> pool;
  double ms[CFIE_K_COUNT] = {0};
  long long launches[CFIE_K_COUNT] = {0};
};

enum geom_kind { G_CIRCLE = 0, G_ELLIPSE = 1, G_STAR = 2, G_KITE = 3, G_SAMPLES = 4 };

struct cfie_geom {
  cfie_ctx* ctx = nullptr;
  int kind = G_CIRCLE;
  double p0 = 1.0, p1 = 1.0;              // circle radius / ellipse a, b
  std::vector<double> a, b;               // star coefficients
  int n_samples = 0;
  std::vector<double> z, dz, ddz;         // caller samples (2n each)
};

// A set of independent GMRES problems laid out as segments of one vector.
struct pset_dev {
  const size_t* off;   // [P] segment offsets
  const int* len;      // [P] segment lengths
  const int* nch;      // [P] 2048-element chunks per segment
  const int* chb;      // [P] first chunk slot of the segment
  const int2* items;   // [Q] (problem, chunk) work list
};
struct pset {
  int P = 0, Q = 0;
  size_t L = 0;
  std::vector<int> len;   // host copy of the segment lengths
  pset_dev dev{};
  dbuf buf;
};

// Krylov workspace (basis, Hessenberg, Givens data, residual vectors)
struct krylov_ws {
  dbuf V, H, w, r, d, rin, small;
  dbuf pz, pz2;             // right preconditioning: P v for the matvec, P (V y) for the update
  dbuf V32, w32, vin;       // FP32 basis of the inner solves (refined precisions)
  double* host = nullptr;   // pinned mirror of per-problem norms
  int host_cap = 0;
  // during an Arnoldi step's matvec: which problems still take part (empty
  // outside one: all); a batch skips the operators none of whose problems do
  std::vector<int> live;
};

#include <functional>
// matvecs of one solve: y = A x on the whole super vector
struct solve_fns {
  std::function<void(const double2*, double2*)> inner;   // the fast (FP32 / tensor) matvec
  std::function<void(const double2*, double2*)> fp64;    // the FP64 matvec (true residuals)
  // right preconditioner y = P x (empty: none): GMRES runs on A P and x += P (V y)
  std::function<void(const double2*, double2*)> prec;
  bool basis32 = true;   // refined precisions: inner Krylov basis in FP32
};

// Device-side geometry of an operator (structure of arrays, FP64 masters).
struct geom_dev {
  double* x;      // z1
  double* y;      // z2
  double* nx;     // nu~_1 = z2'      (unnormalised outward normal, |nu~| = |z'|)
  double* ny;     // nu~_2 = -z1'
  double* sp;     // |z'|
  double* kap;    // L2(t,t) = (z2' z1'' - z1' z2'') / (4 pi |z'|^2)
};

// Plan of the stored-matrix contraction over a list of jobs (stored.cu).
enum { GEMM_DEAL_AUTO = -1, GEMM_DEAL_ROUND_ROBIN = 0, GEMM_DEAL_GREEDY = 1, GEMM_DEAL_STREAMK = 2 };
struct gemm_plan {
  int grid = 0, njobs = 0, mt_total = 0, nsegs = 0, max_pitch = 0, launches_per_run = 0;
  int dealing = GEMM_DEAL_AUTO;   // how the work was dealt to the CTAs
  int stall = 0;   // fault injection for the failure tests (CFIE_FAULT_INJECT=tma_stall)
  dbuf jobs, tables, partial, bt, io, err;
  cudaGraphExec_t exec = nullptr;
};

// Stream-K plan of the fused matrix-free tensor-core matvec (matvec_tc.cu).
struct tc_plan {
  bool built = false;
  int grid = 0, nsegs = 0, mtiles = 0;
  size_t o_cbeg = 0, o_mts = 0;
  dbuf tables, bt, partial, err;
  alignas(64) unsigned char tmB[128];   // CUtensorMap of the B planes
};

// Plan of the tensor-core residual for one right-hand-side block width
// (matvec_df.cu): stream-K segments, density slice planes and their tensor
// map, per-segment double-float sums, column exponents, band part, error flag.
struct rtc_plan {
  bool built = false;
  int grid = 0, nsegs = 0, mtiles = 0, pitch = 0;
  size_t o_cbeg = 0, o_mts = 0;
  dbuf tables, bt, acc, fx, yb, err;
  alignas(64) unsigned char tmB[128];
};

// Bluestein / radix-2 FFT tables of an operator's spectral derivative
// (spectral_fft.cu): power-of-two length N >= 2 n - 1, twiddles, chirp, FFT of
// the wrapped chirp (FP64 and FP32), work buffers.
struct fft_plan {
  int N = 0, L = 0;
  dbuf tw, tw32, chirp, chirp32, bf, bf32, work, work32;
};

struct cfie_op {
  cfie_ctx* ctx = nullptr;
  int n = 0;
  double omega = 0, eta = 0, h = 0;
  cfie_bc bc = CFIE_SOUND_SOFT;
  cfie_precision prec = CFIE_FP64;
  cfie_layout layout = CFIE_MATRIX_FREE;

  dbuf geo;          // 6 n doubles (geom_dev)
  geom_dev g{};
  dbuf wtab;         // n doubles: w_d = R_d - h ln(4 sin^2(pi d / n)), w_0 = R_0
  dbuf ctab;         // n doubles: spectral derivative circulant c_d = (-1)^d cot(pi d / n) / 2
  dbuf diag;         // complex diagonal entries: soft A_ii; hard (S_ii, D'_ii)
  double R0 = 0;

  // scratch for the matrix-free FP64 matvec (split-source partial sums)
  dbuf partial;
  dbuf tmp1, tmp2;   // hard path: u = d/ds x, t = S u

  // FP32 path (created for CFIE_FP32_REFINED)
  dbuf geo32;        // hi/lo coordinates + FP32 normals / speeds
  dbuf band;         // near-field band entries (complex64), n x (2 b + 1) per operator
  int band_b = -1;
  dbuf xin32, xin32b; // FP32 staging of the input (and hard-path helpers)
  dbuf tcv, tcs;      // sound-hard tensor-core path: S inputs, S and D' outputs
  fft_plan fft;       // sound hard: FFT spectral derivative

  // FP64-accurate residual matvec in double-float arithmetic (sound-soft)
  dbuf df_geo, df_band, df_part, df_x;
  int df_b = -1;
  dbuf df_rowexp;    // sound soft: row exponents of the far entries (tensor-core residual)
  rtc_plan rtc[3];   // tensor-core residual plans for 16, 32, 64 right-hand sides per pass
  int res_variant = 0;   // residual: 0 automatic, 1 CUDA-core Dot2, 2 tensor cores

  // FP32 matvec variant: 0 = autotuned, 1 = FP32-pipe contraction, 2 = tensor cores
  int variant = 0, tuned_nrhs = -1, tuned_choice = 1;
  int basis32 = 1;   // inner Krylov basis in FP32 for the refined precisions
  tc_plan tc[2];   // 32- and 64-right-hand-side plans

  // stored path (CFIE_STORED): bf16 hi/lo planes of A and the contraction plan
  dbuf stored;
  gemm_plan plan;
  int plan_nrhs = -1;

  // GMRES workspace and problem set (one problem per right-hand side)
  krylov_ws K;
  pset ps;
  int ps_nrhs = -1;

  cfie_solve_stats stats{};
  cfie_dirprec* dirprec = nullptr;   // right preconditioner of cfie_gmres_solve (not owned)
  int block_gmres = 0;               // cfie_gmres_solve as one block GMRES over the columns
  dbuf bgws;                         // its workspace (basis, blocks, partial sums)
};

// Directional preconditioner of Section 2 built for one sound-soft operator
// (dirprec.cu): segments, level matrices and the W~ solve tables on the device.
struct cfie_dirprec {
  cfie_ctx* ctx = nullptr;
  int n = 0, q = 0, p = 0, m = 0, Ktot = 0, nS = 0, nRest = 0, nnz = 0;
  double omega = 0, eta = 0, L = 0;
  std::vector<int> first, level, count, koff;
  std::vector<double> e;          // m x m e_ij (complex128 interleaved, zero diagonal)
  // level matrices (complex64, row-major), per-segment GEMM descriptors and
  // work items, W~ solve tables, the inverse of W~'s coupled block
  dbuf mats, descs, items, wsolve, Z;
  int item_off[5] = {0}, item_cnt[5] = {0};
  dbuf work;                      // work vectors, grown with the number of right-hand sides
};

// A batch of operators solved in lockstep (one problem per right-hand side of
// every operator; vectors are the operators' blocks concatenated).
struct cfie_batch {
  cfie_ctx* ctx = nullptr;
  std::vector<cfie_op*> ops;
  std::vector<int> nrhs;
  std::vector<long long> off;
  std::vector<int> pfirst;   // index of each operator's first problem
  size_t L = 0;
  bool all_stored = false;
  int basis32 = 1;
  float tune_ms[3] = {0.f, 0.f, 0.f};   // contraction time per dealing when tuned
  cfie_precision prec = CFIE_FP64;
  gemm_plan plan;
  krylov_ws K;
  pset ps;
  cfie_solve_stats stats{};
  // streams on which the operators' residual matvecs run concurrently
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> aux_ev;
};

// ----------------------------------------------------------------------------
// profiling helpers (capi.cu)
// ----------------------------------------------------------------------------
void prof_begin(cfie_ctx* c, int cls, cudaEvent_t* a);
void prof_end(cfie_ctx* c, int cls, cudaEvent_t a);
void prof_harvest(cfie_ctx* c, bool wait);

struct prof_scope {
  cfie_ctx* c;
  int cls;
  cudaEvent_t a = nullptr;
  prof_scope(cfie_ctx* c_, int cls_) : c(c_), cls(cls_) { prof_begin(c, cls, &a); }
  ~prof_scope() { prof_end(c, cls, a); }
};

// ----------------------------------------------------------------------------
// kernels' host entry points
// ----------------------------------------------------------------------------
// geometry.cu
void geometry_sample(cfie_op* op, const cfie_geom* geom);
void kress_tables(cfie_op* op);
void rhs_plane_waves(cfie_op* op, int nrhs, const double* theta_host, double2* f);
// matvec_fp64.cu
void matvec_fp64(cfie_op* op, const double2* x, double2* y, int nrhs);
void spectral_apply(cfie_op* op, const double2* in, double2* out, const double2* base,
                    double2 scale, int nrhs);
// spectral_fft.cu: the same derivative by FFT (tables built by fft_prepare)
void fft_prepare(cfie_op* op);
void spectral_fft64(cfie_op* op, const double2* in, double2* out, const double2* base,
                    double2 scale, int nrhs);
void spectral_fft32_apply(cfie_op* op, const float2* in, float2* out, int nrhs);
void spectral_fft32_accumulate(cfie_op* op, const float2* in, double2* y, double2 scale,
                               int nrhs);
// sound-hard combination of the four FP64-layout partial sums (S u, S n1 x,
// S n2 x, D' x): t = S u, y = x / 2 - D' x - i (omega^2 / eta) (n1 S n1 x + n2 S n2 x)
void reduce_hard_fp64(cfie_op* op, const double2* part, int splits, const double2* x,
                      double2* t, double2* y, int nrhs);
void matvec_fp64_static(cfie_op* op, const double2* x, double2* y, int nrhs);
size_t static_scratch_capacity();
// matvec_fp32.cu
void fp32_prepare(cfie_op* op);
void fp32_band(cfie_op* op);   // after df_prepare
// FP32 helpers shared with the tensor-core kernels: x32 = x, u32 = (1/|z'|) d/dt x32,
// y += (1/(i eta)) (1/|z'|) d/dt t32
void k_to32_fp32(cfie_op* op, const double2* x, float2* x32, size_t tot);
void spectral32_apply(cfie_op* op, const float2* x32, float2* u32, int nrhs);
void spectral32_accumulate(cfie_op* op, const float2* t32, double2* y, int nrhs);
void matvec_fp32(cfie_op* op, const double2* x, double2* y, int nrhs);
// stored.cu
void gemm_plan_build(gemm_plan& G, cfie_ctx* ctx, const std::vector<cfie_op*>& ops,
                     const std::vector<int>& nrhs, const std::vector<long long>& xoff,
                     int dealing);
// the dealing of a batch's contraction picked by timing each once (cached per
// batch shape for the process); ms[3] receives the candidates' times (0 when cached)
int gemm_plan_tune(gemm_plan& G, cfie_ctx* ctx, const std::vector<cfie_op*>& ops,
                   const std::vector<int>& nrhs, const std::vector<long long>& xoff,
                   size_t L, float* ms);
void gemm_plan_run(gemm_plan& G, cfie_ctx* ctx, const double2* x, double2* y);
int gemm_plan_take_error(gemm_plan& G, cfie_ctx* ctx);
void gemm_plan_release(gemm_plan& G);
void stored_prepare(cfie_op* op);
void matvec_stored(cfie_op* op, const double2* x, double2* y, int nrhs);
int stored_take_error(cfie_op* op);
// matvec_df.cu
void df_prepare(cfie_op* op);
bool df_available(const cfie_op* op);
void matvec_df(cfie_op* op, const double2* x, double2* y, int nrhs);
// residual matvec of refined solves: double-float when available, else FP64
void matvec_residual(cfie_op* op, const double2* x, double2* y, int nrhs);
// matvec_tc.cu
void matvec_fp32_tc(cfie_op* op, const double2* x, double2* y, int nrhs);
int tc_take_error(cfie_op* op);
int df_take_error(cfie_op* op);
// arnoldi.cu
void pset_build(pset& ps, const std::vector<size_t>& off, const std::vector<int>& len,
                cudaStream_t st);
void pset_uniform(pset& ps, int n, int nrhs, cudaStream_t st);
void measure_peaks(cfie_ctx* ctx, cfie_peaks* out);
void field_eval(cfie_op* op, const double2* q, int nrhs, int npts, const double2* pts,
                double2* u);
void gmres_set(cudaStream_t st, cfie_ctx* ctx, krylov_ws& K, const pset& ps,
               const solve_fns& fns, bool refined, const double2* f, double2* x, double rtol,
               int restart, int maxit, int* iters, double* relres, cfie_status* status,
               cfie_solve_stats& stats);
void krylov_release(krylov_ws& K);
// dispatch (capi.cu)
void apply_inner(cfie_op* op, const double2* x, double2* y, int nrhs);
// dirprec.cu: the directional preconditioner of Section 2
void dirprec_build(cfie_dirprec* P, cfie_op* op, cfie_curve kind, const double* params,
                   int nparams, int q, int p, int m_leaf, int t_keep);
void dirprec_apply(cfie_dirprec* P, const double2* x, double2* y, int nrhs);
int dirprec_n(const cfie_dirprec* P);
int dirprec_segments(const cfie_dirprec* P, double* e);
// block_gmres.cu: block GMRES over the nrhs columns of one operator
void block_gmres_solve(cfie_op* op, const double2* f, double2* x, int nrhs, double rtol,
                       int restart, int maxit, int* iters, double* relres, cfie_status* status,
                       dbuf& ws);
