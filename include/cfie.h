/*
 * cfie.h -- C ABI of the GB300 combined-field integral equation (CFIE) library.
 *
 * The library discretises and solves the 2-D exterior Helmholtz scattering
 * problems of Section 1 of Ying, "Directional preconditioner for high frequency
 * obstacle scattering":
 *
 *   sound soft  (eq. 1):  (1/2 I + D - i eta S) q = -u_I
 *   sound hard  (eq. 2):  (1/2 I - D' + N/(i eta)) q = -du_I/dn
 *
 * with G(x, y) = (i/4) H0^(1)(omega |x - y|) and the operators S, D, D', N of
 * Section 1, discretised by the Nystrom method (Section 1) with Kress's
 * logarithmic-split trapezoidal rule on n equispaced parameter nodes
 * t_j = 2 pi j / n, N by Maue's identity N = d/ds S d/ds + omega^2 (n.S n).
 * Eq. 2's sign is used for the sound-hard operator.  Krylov solves use GMRES
 * with restart, as in Section 3.
 *
 * Call sequence: cfie_ctx_create -> cfie_geometry_* -> cfie_discretise ->
 * cfie_rhs_plane_waves -> cfie_apply / cfie_gmres_solve -> *_destroy.
 * Host-only helpers that need no context or GPU: cfie_arclength_samples (the
 * node set of Section 2, for cfie_geometry_samples) and the setup pieces of the
 * directional preconditioner of Section 2 (cfie_dirprec_plan,
 * cfie_dirprec_level, cfie_dirprec_threshold, cfie_dirprec_w_pattern).  The
 * preconditioner itself: cfie_dirprec_create -> cfie_op_set_preconditioner /
 * cfie_dirprec_apply -> cfie_dirprec_destroy.  Many operators at once:
 * cfie_discretise_many (set-up overlapped) and cfie_batch_* (lockstep solves,
 * one persistent tensor-core launch per matvec for stored operators); one
 * Krylov space over all directions: cfie_op_set_block_gmres; a stream of
 * requests: cfie_server_* (batched slots, admission by HBM footprint).
 *
 * Conventions for every entry point:
 *  - All compute runs on the context's CUDA device and stream; calls that take
 *    device buffers are asynchronous on that stream unless stated otherwise.
 *  - Complex vectors are interleaved complex128 (re, im doubles), "column-major
 *    n x nrhs": right-hand side k occupies elements [k*n, (k+1)*n).  Device
 *    buffers belong to the caller, must be 16-byte aligned and hold n*nrhs
 *    complex128 values; they must not overlap unless stated.
 *  - Handles (cfie_ctx, cfie_geom, cfie_op) and the device memory behind them
 *    belong to the library and are freed by the matching *_destroy call.  A
 *    geometry must outlive the operators made from it only until
 *    cfie_discretise returns (operators copy what they need).
 *  - Every call returns a cfie_status and never aborts or exits.  On error the
 *    context keeps a message readable with cfie_last_error; outputs are left
 *    unspecified unless stated.
 *  - A context is not thread-safe: use one context per host thread.
 *  - Library device memory comes from the device's stream-ordered pool
 *    (cudaMallocAsync / cudaFreeAsync on the context stream); cfie_ctx_create
 *    raises the pool's release threshold so that buffers freed when operators
 *    are destroyed are reused by the next ones instead of returned to the
 *    driver.
 */
#ifndef CFIE_H
#define CFIE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CFIE_OK = 0,
  CFIE_EINVAL = 1,    /* invalid argument (sizes, null pointers, non-finite values) */
  CFIE_ENOMEM = 2,    /* device or host allocation failed */
  CFIE_ECUDA = 3,     /* a CUDA call failed; see cfie_last_error */
  CFIE_ENOCONV = 4,   /* GMRES hit maxit before rtol; x holds the last iterate */
  CFIE_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
  CFIE_EBUSY = 6      /* the server has no free slot for the request */
} cfie_status;

typedef enum { CFIE_SOUND_SOFT = 0, CFIE_SOUND_HARD = 1 } cfie_bc;

/* Precision of the operator application used inside GMRES.
 *  CFIE_FP64          FP64 kernel evaluation and FP64 sums everywhere.
 *  CFIE_FP32_REFINED  FP32 on-the-fly kernel evaluation (two-float phase, FP64
 *                     near band) for the inner matvecs, with iterative
 *                     refinement on the outer residual.  The inner Krylov
 *                     basis, its inner products and updates are FP32 by
 *                     default (cfie_op_set_inner_basis(op, 0): FP64); the
 *                     Hessenberg matrix, Givens rotations, least-squares solve
 *                     and solution update are FP64; the true residuals are
 *                     FP64-accurate (double-float arithmetic, a few 1e-12
 *                     relative: cfie_apply_residual).
 *  CFIE_TENSOR_REFINED stored complex matrix contracted on the tensor cores
 *                     (split-complex, FP32 accumulation) for the inner matvecs;
 *                     Krylov basis and residuals as for CFIE_FP32_REFINED. */
typedef enum { CFIE_FP64 = 0, CFIE_FP32_REFINED = 1, CFIE_TENSOR_REFINED = 2 } cfie_precision;

typedef enum { CFIE_MATRIX_FREE = 0, CFIE_STORED = 1 } cfie_layout;

typedef struct cfie_ctx cfie_ctx;
typedef struct cfie_geom cfie_geom;
typedef struct cfie_op cfie_op;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (may be NULL for the legacy default stream); the caller keeps ownership of
 * it and it must outlive the context.  Writes the handle to *out. */
cfie_status cfie_ctx_create(int device, void* cuda_stream, cfie_ctx** out);
/* Free a context (NULL is ignored).  Destroy its geometries, operators and
 * batches first; the caller's stream is left alone. */
void cfie_ctx_destroy(cfie_ctx* ctx);

/* Message of the last failing call on this context ("" if none).  The string
 * belongs to the context and stays valid until its next call. */
const char* cfie_last_error(const cfie_ctx* ctx);

/* --- Geometry: counter-clockwise 2 pi-periodic curves z(t) (Section 1 asks for
 * a smooth boundary; Section 2 samples it at equispaced points). ------------ */

/* Circle of the given radius about the origin.  radius > 0. */
cfie_status cfie_geometry_circle(cfie_ctx* ctx, double radius, cfie_geom** out);
/* Ellipse (a cos t, b sin t), a, b > 0 (the obstacle of Tables 1 and 3). */
cfie_status cfie_geometry_ellipse(cfie_ctx* ctx, double a, double b, cfie_geom** out);
/* Star z(t) = r(t) (cos t, sin t), r(t) = 1 + sum_{k=1..K} a[k-1] cos kt + b[k-1] sin kt.
 * a, b: host arrays of K doubles (copied); 1 <= K <= 64; r must stay positive. */
cfie_status cfie_geometry_fourier_star(cfie_ctx* ctx, int K, const double* a,
                                       const double* b, cfie_geom** out);
/* Kite z(t) = (cos t + 0.65 cos 2t - 0.65, 1.5 sin t). */
cfie_status cfie_geometry_kite(cfie_ctx* ctx, cfie_geom** out);
/* Caller-sampled curve: host arrays of n points (x, y interleaved, 2n doubles
 * each) holding z, z', z'' at t_j = 2 pi j / n.  Copied.  Only discretisations
 * with exactly this n are allowed. */
cfie_status cfie_geometry_samples(cfie_ctx* ctx, int n, const double* z, const double* dz,
                                  const double* ddz, cfie_geom** out);
/* Free a geometry (NULL is ignored).  Operators discretised from it keep their
 * own device copy of the nodes and stay valid. */
void cfie_geom_destroy(cfie_geom* geom);

/* Curves of the cfie_geometry_* constructors, by name, for host-side helpers. */
typedef enum {
  CFIE_CURVE_CIRCLE = 0,
  CFIE_CURVE_ELLIPSE = 1,
  CFIE_CURVE_STAR = 2,
  CFIE_CURVE_KITE = 3
} cfie_curve;

/* Samples of a curve at n points equispaced in arclength, the node set of
 * Section 2 (segments of 2^l p equispaced points, 2^l wavelengths long).  The
 * curve is the one the matching cfie_geometry_* call builds, with params
 * (host, nparams doubles, copied): circle {radius}; ellipse {a, b}; star
 * {a_1..a_K, b_1..b_K}, nparams = 2K, 1 <= K <= 64; kite none (params may be
 * NULL).  Outputs (host arrays of 2n doubles, x and y interleaved: the layout
 * cfie_geometry_samples takes): z, dz/dsigma and d2z/dsigma2 at
 * sigma_j = 2 pi j / n, where sigma = 2 pi s / L is the arclength s from the
 * curve's point at t = 0, rescaled to [0, 2 pi) (constant speed L / (2 pi));
 * *perimeter receives L unless perimeter is NULL.  n even, 8 <= n <= 2^20.
 * CFIE_EINVAL for invalid arguments or a curve whose speed vanishes (a star
 * whose r reaches 0).  Host only: needs no context and no GPU; the arclength
 * is accurate to a few units in the last place of L. */
cfie_status cfie_arclength_samples(cfie_curve kind, const double* params, int nparams, int n,
                                   double* z, double* dz, double* ddz, double* perimeter);

/* Structure of the directional preconditioner (Section 2.1) for the curve
 * sampled at n = 4^q p points equispaced in arclength (cfie_arclength_samples
 * with the same curve and n; p points per wavelength 2 pi / omega).
 *  - Segments, in order along the curve from its point at t = 0: 2^q pieces of
 *    2^q p points, each halved until it is almost planar (2^l <= 2^q / sqrt(c),
 *    c the largest |curvature| at its nodes) or a non-planar leaf
 *    (2^l <= m_leaf).  Segment i holds the 2^level[i] p nodes from first[i].
 *  - For i != j, with c_i the curve point halfway (in arclength) between the
 *    segment's first and last node, t_i the unit tangent there and
 *    a_ij = (c_i - c_j) / |c_i - c_j|: k^i_ij = [omega a_ij . t_i]_i and
 *    k^j_ij = [-omega a_ij . t_j]_j, the nearest of the 2^(l+1) + 1 equispaced
 *    wave numbers of [-omega, omega] of each segment's level (ties away from
 *    zero), as indices 0 .. 2^(l+1): kpair[2 (i m + j)] = k^i_ij,
 *    kpair[2 (i m + j) + 1] = k^j_ij; zero for i == j.
 * *m receives the number of segments.  With first, level and kpair all NULL
 * nothing else is written (the sizing call); otherwise each holds capacity,
 * capacity and 2 capacity^2 ints (host) and capacity >= *m, else CFIE_EINVAL.
 * params as for cfie_arclength_samples; 1 <= q <= 9, p >= 1, n even and
 * 8 <= n <= 2^20, omega > 0, m_leaf >= 1.  Host only: no context, no GPU. */
cfie_status cfie_dirprec_plan(cfie_curve kind, const double* params, int nparams, int q, int p,
                              double omega, int m_leaf, int capacity, int* m, int* first,
                              int* level, int* kpair);

/* Sparsity pattern of W~ = E + antidiag(T) (Section 2.2) from a plan of m
 * segments (level, kpair as cfie_dirprec_plan writes them).  Segment i owns the
 * K_i = 2^(level[i]+1) + 1 frequency unknowns from koff[i]; on success koff
 * (host, m + 1 ints) and *nnz = m (m - 1) + sum K_i are written.  With row and col
 * (host, capacity ints each, capacity >= *nnz) the positions follow: first
 * E's entry of every ordered pair i != j, i major, at
 * (koff[i] + k^i_ij, koff[j] + k^j_ij); then the anti-diagonal of every T block,
 * (koff[i] + r, koff[i] + K_i - 1 - r), r = 0 .. K_i - 1.  row and col both
 * NULL: sizes only.  CFIE_EINVAL for out-of-range levels or indices, or too
 * small a capacity, checked before any output is written (outputs untouched).
 * Host only. */
cfie_status cfie_dirprec_w_pattern(int m, const int* level, const int* kpair, int capacity,
                                   int* koff, int* nnz, int* row, int* col);

/* Level blocks of the directional preconditioner (Section 2.2, sound soft) for
 * the segments of level l (c = 2^l p nodes) of an n-node arclength
 * discretisation of a curve of perimeter L:
 *  B: c x c, the operator 1/2 I - i eta S restricted to a straight segment of c
 *     nodes with spacing L / n (Kress-Nystrom entries on a line, where the
 *     double-layer kernel vanishes);
 *  Binv: B^-1;  U: c x K, K = 2^(l+1) + 1, U(x, m) = exp(i k_m (x - (c-1)/2) L / n)
 *     with k_m = -omega + 2 omega m / (K - 1);  T: K x K, (U^t B^-1 U)^-1.
 * Each output (host, complex128 interleaved, row-major) may be NULL to skip it.
 * n even, 8 <= n <= 2^20, c <= min(n / 2, 1024), omega, eta, L > 0.
 * CFIE_EINVAL for invalid arguments or a singular block.  Host only. */
cfie_status cfie_dirprec_level(int n, int p, int level, double omega, double eta, double L,
                               double* B, double* Binv, double* U, double* T);

/* T~ of Section 2.2: the `keep` entries of the K x K block T (host,
 * complex128 interleaved, row-major) largest in modulus, copied to Tt, every
 * other entry zero; entries within a relative 2^-30 of the smallest modulus
 * kept count as tied with it and are kept too (T is symmetric: equal entries
 * differ only by rounding).  keep >= K^2 copies T.  1 <= K <= 4097, keep >= 0.  Host only. */
cfie_status cfie_dirprec_threshold(int K, const double* T, int keep, double* Tt);

/* --- Directional preconditioner (Section 2) on the GPU ------------------- */

typedef struct cfie_dirprec cfie_dirprec;

/* Build the directional preconditioner of Section 2 for a sound-soft operator
 * (eq. 1) whose nodes are the curve's n = 4^q p points equispaced in arclength
 * (cfie_arclength_samples with the same kind and params, then
 * cfie_geometry_samples and cfie_discretise with that n; p points per
 * wavelength 2 pi / omega).  Steps, following Sections 2.1 and 2.2:
 *  - segments and wave-number pairs as cfie_dirprec_plan (m_leaf the leaf
 *    length in wavelengths);
 *  - per level, B_l^-1, U_l, T_l as cfie_dirprec_level and T~_l as
 *    cfie_dirprec_threshold keeping t_keep K entries (K = 2^(l+1) + 1);
 *  - E on the GPU: e_ij = the mean over x in P_i, y in P_j of
 *    M(x, y) / (U_i(x, k^i_ij) U_j(y, k^j_ij)), the least-squares constant of
 *    the rank-1 form M_ij ~ U_i e_ij U_j^t on the block's nodes (the quantity
 *    eq. entry approximates from Chebyshev samples), from the operator's FP64
 *    entries;
 *  - W~ = E + antidiag(T) solved exactly through its sparsity: the unknowns
 *    that couple form a block inverted densely on the GPU (FP64 Gauss-Jordan
 *    with row pivoting, about half of W~'s dimension).
 * Device memory: the level matrices and W~'s coupled block (complex64,
 * 134 MB at q = 6).  Synchronous.  CFIE_EINVAL for a sound-hard operator,
 * n != 4^q p, nodes that are not the curve's arclength samples, invalid
 * q (1..9), p, m_leaf or t_keep (>= 1), or a singular block. */
cfie_status cfie_dirprec_create(cfie_op* op, cfie_curve kind, const double* params, int nparams,
                                int q, int p, int m_leaf, int t_keep, cfie_dirprec** out);
/* y = P x, eq. (eapp): b = B^-1 x, p0 = -U^t b, t = T~ p0, r = W~^-1 t,
 * p = T~ r - t, y = b - B^-1 U p, for nrhs right-hand sides in complex64
 * arithmetic (device, n x nrhs complex128 in and out, not overlapping;
 * 1 <= nrhs <= 1024).  Asynchronous on the context stream. */
cfie_status cfie_dirprec_apply(cfie_dirprec* P, const void* x_dev, void* y_dev, int nrhs);
/* Number of segments m to *m and, unless e is NULL, the m x m coefficients
 * e_ij (host, complex128 interleaved, row i major, zero diagonal). */
cfie_status cfie_dirprec_coefficients(const cfie_dirprec* P, int* m, double* e);
/* Use P as the right preconditioner of cfie_gmres_solve on op (GMRES on A P y = f,
 * x = P y; for the refined precisions the inner solves are preconditioned).
 * NULL detaches.  P must have been built for op's context and size, and must
 * outlive the solves that use it.  CFIE_EINVAL otherwise. */
cfie_status cfie_op_set_preconditioner(cfie_op* op, cfie_dirprec* P);
/* Free a preconditioner (NULL is ignored) after the context stream's queued
 * work; detach it from its operators first. */
void cfie_dirprec_destroy(cfie_dirprec* P);

/* --- Discretisation ------------------------------------------------------ */

/* Sample the curve at n nodes on the device, build the Kress weight table and
 * everything the chosen precision and layout need (near-field band, stored
 * matrix).  n even, 8 <= n <= 1<<20; omega > 0; eta > 0 (eta = omega is the
 * usual choice, Section 1 asks for eta = O(omega)).  Synchronous. */
cfie_status cfie_discretise(cfie_geom* geom, int n, double omega, double eta, cfie_bc bc,
                            cfie_precision precision, cfie_layout layout, cfie_op** out);
/* cfie_discretise for count operators at once: geoms[k] (all of one context),
 * n[k], omega[k], eta[k] (host arrays of count entries) and one boundary
 * condition, precision and layout; out[k] receives operator k (host array of
 * count handles).  The set-up runs on up to eight worker threads, each with
 * its own CUDA stream, so that the set-up kernels of different operators
 * (sampling, Kress tables, near bands, assembly) overlap on the GPU; the
 * operators then belong to the geometries' context as if made one by one,
 * with the same entries.  Synchronous.  On failure no operator is kept (every
 * out[k] NULL), the status is the first failing one's and its message is the
 * context's.  Not part of the paper (a set-up convenience for batches). */
cfie_status cfie_discretise_many(int count, cfie_geom* const* geoms, const int* n,
                                 const double* omega, const double* eta, cfie_bc bc,
                                 cfie_precision precision, cfie_layout layout, cfie_op** out);
/* Free an operator and its device buffers (NULL is ignored) after the work
 * queued on the context stream has finished.  Batches holding it must be
 * destroyed first. */
void cfie_op_destroy(cfie_op* op);

/* Number of nodes of an operator. */
int cfie_op_n(const cfie_op* op);

/* Right-hand sides for plane waves u_I = exp(i omega d.x), d = (cos theta_k,
 * sin theta_k): soft -u_I(z_j), hard -du_I/dn(z_j) (Section 1; Section 3 uses
 * one wave towards +x).  theta: host array of nrhs angles.  f_dev: device
 * output, n*nrhs complex128. */
cfie_status cfie_rhs_plane_waves(cfie_op* op, int nrhs, const double* theta, void* f_dev);

/* y = A x for nrhs right-hand sides, with A the operator's CFIE matrix applied
 * in the operator's precision (FP64 for CFIE_FP64, the FP32 / tensor inner
 * matvec otherwise).  x_dev, y_dev: device, n*nrhs complex128, must not
 * overlap.  1 <= nrhs <= 1024. */
cfie_status cfie_apply(cfie_op* op, const void* x_dev, void* y_dev, int nrhs);

/* Choose how a CFIE_FP32_REFINED operator sums over sources: 0 = autotune
 * (default: the first block matvec for a given (boundary condition, n, nrhs)
 * times both variants once on the context stream and the process keeps the
 * faster), 1 = register-blocked FP32 sums on the CUDA cores (any operator),
 * 2 = tensor cores (entries split bf16 hi + lo, tcgen05 contraction; for the
 * sound-hard operator S is applied to the three vectors of Maue's identity and
 * D' to the density, each a pass of the same kernel).  Variant 1 evaluates the
 * FP32 entries to full FP32 accuracy, variant 2 to the accuracy its bf16
 * hi + lo operands keep (two-term Hankel series, a few 1e-6 relative next to
 * the near band); both stay far inside the 1e-4 of a raw FP32 matvec. */
cfie_status cfie_op_set_variant(cfie_op* op, int variant);

/* y = A x in FP64 whatever the operator's precision (the matvec used for true
 * residuals). */
cfie_status cfie_apply_fp64(cfie_op* op, const void* x_dev, void* y_dev, int nrhs);

/* y = A x in FP64, like cfie_apply_fp64, but without allocating any device
 * memory: for callers that cannot call cudaMalloc, such as a serving process
 * that has handed all free HBM to its own pool at start-up, or code that must
 * not hit the implicit device synchronisation of cudaMalloc / cudaFree in a
 * latency-critical loop.  The paper has no counterpart; it is a deployment
 * variant of the FP64 matvec.
 *
 * Scratch (split-source partial sums; for the sound-hard operator also the two
 * derivative vectors) lives in one file-scope device array of 32 MiB that every
 * GPU loading the library holds until the process exits.  Needs
 * (soft) 16 * n * nrhs bytes, (hard) 96 * n * nrhs bytes at the least;
 * larger requests return CFIE_EINVAL with a message.  The first call on a
 * device looks the array's device address up (cudaGetSymbolAddress) with that
 * device current, and so does the first call after the device's context was
 * replaced (cudaDeviceReset); make such a call before any stream capture.  Calls
 * share the array: calls that overlap on the GPU (other streams, other host
 * threads) race.  Every scratch element a call reads was written by the same
 * call, so nothing needs clearing between calls.  Arguments as cfie_apply. */
cfie_status cfie_apply_fp64_static(cfie_op* op, const void* x_dev, void* y_dev, int nrhs);

/* y = A x with the FP64-accurate matvec the refined precisions use for their
 * true residuals: for CFIE_FP32_REFINED / CFIE_TENSOR_REFINED operators of
 * either boundary condition the same entries as cfie_apply_fp64 evaluated in
 * double-float arithmetic on the FP32 pipe (hi + lo pairs, error-free products
 * and sums; for the sound-hard operator S and D' so, the spectral derivatives
 * in FP64; a few 1e-12 relative), otherwise the FP64 matvec (also when the
 * near band of the double-float form would exceed 4 GB).  Arguments as
 * cfie_apply. */
cfie_status cfie_apply_residual(cfie_op* op, const void* x_dev, void* y_dev, int nrhs);

/* Solve A x = f for nrhs independent right-hand sides by restarted GMRES
 * (Section 3: relative tolerance and restart; zero initial guess there).
 *  f_dev   device, n*nrhs complex128 (read only)
 *  x_dev   device, n*nrhs complex128: initial guess in, solution out
 *  rtol    target for the true relative residual ||f - A x|| / ||f|| (FP64)
 *  restart Krylov dimension per cycle, 1..512; 0 = unrestarted (maxit)
 *  maxit   cap on Arnoldi steps per right-hand side (inner steps for the
 *          refined precisions)
 *  iters_out  host, nrhs ints (may be NULL): Arnoldi steps per right-hand side
 *  relres_out host, nrhs doubles (may be NULL): true relative residual
 *             recomputed from the returned x with the FP64-accurate matvec
 *             (cfie_apply_fp64 for CFIE_FP64, cfie_apply_residual otherwise)
 * Returns CFIE_ENOCONV (x holds the last iterate) if some right-hand side
 * missed rtol.  Synchronous. */
cfie_status cfie_gmres_solve(cfie_op* op, const void* f_dev, void* x_dev, int nrhs, double rtol,
                             int restart, int maxit, int* iters_out, double* relres_out);

/* How the refined precisions compute true residuals (cfie_apply_residual and
 * inside cfie_gmres_solve), all to a few 1e-12 relative: variant 1 evaluates the
 * entries in double-float (FP32 pairs) and sums with compensated Dot2 on the
 * CUDA cores; variant 2 evaluates the far entries in double-float (for the
 * sound-hard operator S and D' in separate passes), splits entries and
 * densities into six 8-bit slices on per-row / per-column power-of-two grids
 * and sums the slice products on the tensor cores, exactly in FP32 for the
 * three leading levels, with the near band on the CUDA cores; 0 (default)
 * picks 2 with 8 or more right-hand sides, else 1.  CFIE_EINVAL for the FP64
 * precision or another value. */
cfie_status cfie_op_set_residual_variant(cfie_op* op, int variant);

/* Precision of the Krylov basis of the inner solves of the refined precisions
 * (CFIE_FP32_REFINED, CFIE_TENSOR_REFINED): fp32 = 1 (default) keeps the inner
 * basis, its inner products and updates in FP32 (the inner operator is only
 * FP32-accurate, and GB300's FP64 rate is a small fraction of its FP32 rate);
 * fp32 = 0 keeps them in FP64.  The Hessenberg matrix, Givens rotations,
 * least-squares solve, solution update, true residuals and the whole FP64
 * precision stay FP64 either way.  CFIE_EINVAL for a null op or another value. */
cfie_status cfie_op_set_inner_basis(cfie_op* op, int fp32);

/* Solve the nrhs right-hand sides of cfie_gmres_solve as one block problem
 * (on = 1): block GMRES with one Krylov space span{R, A R, A^2 R, ...} shared
 * by all columns of the residual block R, instead of one GMRES per column
 * (on = 0, the default; Section 3 runs one GMRES per incident wave).  Each
 * block step is one block matvec; the basis is orthogonalised by block
 * classical Gram-Schmidt applied twice and a rank-revealing Cholesky QR
 * applied twice (directions whose Gram diagonal falls below a relative
 * 1e-14 (FP64) or 1e-10 (FP32 inner basis) are dropped: repeated or
 * converged columns shrink the next block), and the block Hessenberg least
 * squares is solved by Householder QR updated column by column (FP64, host).
 * For the refined precisions the block solve is the inner solve of the
 * refinement, with the inner basis in FP32 or FP64 (cfie_op_set_inner_basis).
 * In cfie_gmres_solve, restart then counts block steps per cycle (0:
 * unrestarted, up to 512), maxit caps the block steps, and iters_out reports
 * the block steps for every column.  A right preconditioner set on op applies
 * as in the per-column solve.  CFIE_EINVAL for a null op or another value. */
cfie_status cfie_op_set_block_gmres(cfie_op* op, int on);

/* Scattered field at off-surface points from a boundary density (Section 1:
 * u is evaluated through a boundary integral once q is known).  With the
 * operator's curve, omega, eta and boundary condition,
 *     sound soft:  u(x) = (D q)(x) - i eta (S q)(x)
 *     sound hard:  u(x) = -(S q)(x) + (D q)(x) / (i eta)
 * (the representations whose boundary limits are eq. 1 and eq. 2), by the
 * plain trapezoidal rule in FP64 whatever the operator's precision.  q_dev:
 * n x nrhs complex128, column-major (density k contiguous); pts_dev: npts
 * points as (x, y) double pairs, device memory; u_dev: npts x nrhs complex128,
 * column-major.  Points must lie off the curve; the rule is spectrally
 * accurate a few node spacings (2 pi / n in the parameter) away from it and
 * loses accuracy closer in.  Pointers 16-byte aligned; u must not overlap q or
 * pts.  Asynchronous on the context stream. */
cfie_status cfie_field_eval(cfie_op* op, const void* q_dev, int nrhs, int npts,
                            const void* pts_dev, void* u_dev);

/* Counters of the last cfie_gmres_solve on this operator. */
typedef struct {
  int cycles;            /* GMRES cycles (restarts + 1) summed over refinement steps */
  int refinements;       /* outer refinement steps (0 for CFIE_FP64) */
  int inner_matvecs;     /* block matvecs in the operator's precision */
  int fp64_matvecs;      /* block FP64 matvecs (true residuals) */
  int arnoldi_steps;     /* Arnoldi steps (max over right-hand sides) */
  int matvec_variant;    /* kernel of the last inner matvec: 0 FP64 pair kernel,
                            1 FP32 pair kernel with CUDA-core source sums, 2 FP32
                            pair kernel with tensor-core source sums, 3 stored
                            matrix on the tensor cores */
  int basis_fp32;        /* 1 if the inner solves kept their Krylov basis in FP32 */
  int residual_variant;  /* kernel of the last true residual: 0 FP64 pair kernel,
                            1 double-float Dot2, 2 sliced tensor-core sums */
  long long arnoldi_elems; /* basis elements read by one orthogonalisation pass,
                              summed over the Arnoldi steps (CGS2 makes four
                              passes: two inner products, two updates) */
} cfie_solve_stats;
/* Statistics of the operator's last cfie_gmres_solve, copied to *out (host).
 * CFIE_EINVAL for a null operator or output. */
cfie_status cfie_op_last_stats(const cfie_op* op, cfie_solve_stats* out);

/* --- Batches: many operators solved in lockstep ------------------------- */

typedef struct cfie_batch cfie_batch;

/* Group `count` operators of one context, all of the same precision, with
 * nrhs[k] right-hand sides for operator k.  Batch vectors are the operators'
 * column-major n_k x nrhs[k] blocks concatenated in order (see
 * cfie_batch_length).  When every operator uses CFIE_STORED, one block matvec of
 * the whole batch is one CUDA-graph replay: the B-operand preparation of
 * every operator, then a persistent tensor-core contraction over all
 * (operator, row tile, source tile) triples (one CTA per SM) that writes y
 * itself when its work dealing gives whole row tiles, or partial sums that a
 * third kernel adds when it splits row tiles (stream-K).  Otherwise the operators' matvecs run on up to
 * eight auxiliary streams forked from and joined back into the context stream;
 * inside a lockstep solve an operator all of whose right-hand sides have
 * converged is skipped.  The operators must outlive the batch.  Synchronous. */
cfie_status cfie_batch_create(cfie_ctx* ctx, int count, cfie_op* const* ops, const int* nrhs,
                              cfie_batch** out);
/* Number of complex128 elements of a batch vector (sum of n_k * nrhs[k]). */
long long cfie_batch_length(const cfie_batch* batch);
/* y = A x for every operator of the batch in the operators' precision. */
cfie_status cfie_batch_apply(cfie_batch* batch, const void* x_dev, void* y_dev);
/* GMRES on every right-hand side of every operator at once (each one an
 * independent problem; arguments as cfie_gmres_solve, iters_out / relres_out
 * hold one entry per right-hand side in batch order). */
cfie_status cfie_batch_gmres_solve(cfie_batch* batch, const void* f_dev, void* x_dev, double rtol,
                                   int restart, int maxit, int* iters_out, double* relres_out);
/* As cfie_op_last_stats, for the batch's last lockstep solve. */
cfie_status cfie_batch_last_stats(const cfie_batch* batch, cfie_solve_stats* out);
/* As cfie_op_set_inner_basis, for the lockstep solves of a batch. */
cfie_status cfie_batch_set_inner_basis(cfie_batch* batch, int fp32);
/* How the batch's persistent contraction deals its work to the CTAs (one per
 * SM), picked by cfie_batch_create when every operator is stored: each
 * candidate's graph replay is timed once (CUDA events, mean of two replays
 * after one warm-up) and the fastest kept; the choice is remembered for the
 * process per batch shape (the operators' n and right-hand-side counts).
 *  0  whole (operator, 128-row tile) units dealt round-robin
 *  1  whole units in operator order, each to the CTA with the least work so
 *     far (balanced within one unit; the CTAs stay on neighbouring units)
 *  2  stream-K: the (row tile, 64-source tile) pairs split evenly
 * *dealing receives the choice (-1 when the batch is not all stored); ms
 * (host, 3 floats, may be NULL) the candidates' replay times in milliseconds,
 * zeros when the choice came from the process's memory.  CFIE_EINVAL for a
 * null batch or dealing. */
cfie_status cfie_batch_tuning(const cfie_batch* batch, int* dealing, float* ms);
/* Rebuild the batch's contraction plan with the given dealing (0, 1 or 2, as
 * cfie_batch_tuning lists them) instead of the tuned one.  Synchronous.
 * CFIE_EINVAL for another value or a batch that is not all stored. */
cfie_status cfie_batch_set_dealing(cfie_batch* batch, int dealing);
/* Free a batch (NULL is ignored) after its queued work has finished; its
 * operators stay valid. */
void cfie_batch_destroy(cfie_batch* batch);


/* --- Kernel timing (CUDA events on the context stream) ------------------- */

/* Kernel classes timed when profiling is on. */
typedef enum {
  CFIE_K_MATVEC_FP64 = 0,   /* FP64 pair-evaluation matvec kernel */
  CFIE_K_MATVEC_FP32 = 1,   /* FP32 fused matrix-free matvec kernel */
  CFIE_K_MATVEC_TENSOR = 2, /* stored-matrix tensor-core contraction */
  CFIE_K_ARNOLDI = 3,       /* orthogonalisation kernels of one Arnoldi step */
  CFIE_K_SPECTRAL = 4,      /* spectral tangential derivative */
  CFIE_K_COUNT = 5
} cfie_kernel_class;

/* Turn per-launch event timing on (1) or off (0) and reset the totals. */
cfie_status cfie_ctx_set_profiling(cfie_ctx* ctx, int on);
/* Total milliseconds and launch count per kernel class since the last reset.
 * ms, launches: host arrays of CFIE_K_COUNT entries.  Synchronises the stream. */
cfie_status cfie_ctx_kernel_times(cfie_ctx* ctx, double* ms, long long* launches);

/* --- Serving: continuous batching of independent solves ------------------- */

typedef struct cfie_server cfie_server;

/* One solve request: a star obstacle r(t) = 1 + sum_k a_k cos kt + b_k sin kt
 * (host arrays of K doubles, copied), n nodes, omega, eta, boundary condition,
 * nrhs plane waves at the host angles theta (copied), residual target rtol,
 * GMRES restart / maxit, and the precision: CFIE_FP32_REFINED (matrix free)
 * or CFIE_TENSOR_REFINED (sound-soft only: the matrix stored, 8 n^2 bytes, and
 * contracted on the tensor cores; a batch of such requests runs one
 * persistent contraction launch per matvec), the served mixed-precision
 * forms, or CFIE_FP64, the plain form. */
typedef struct {
  int bc;            /* cfie_bc */
  int precision;     /* cfie_precision */
  int K;
  const double* a;
  const double* b;
  int n;
  double omega, eta;
  int nrhs;
  const double* theta;
  double rtol;
  int restart, maxit;
} cfie_request;

typedef struct {
  int done, started;
  cfie_status status;   /* of the solve (CFIE_ENOCONV: missed rtol) */
  int iters_max;        /* Arnoldi steps, max over right-hand sides */
  double relres_max;    /* true FP64 relative residual, max over right-hand sides */
  double queued_s, service_s, latency_s;   /* submit -> start, start -> done, submit -> done */
} cfie_result;

typedef struct {
  long long completed, solves, queued, running, peak_running;
  long long budget_bytes, in_use_bytes, peak_in_use_bytes;
} cfie_server_counters;

/* Start a server on `device` with `slots` concurrent solves (each slot a host
 * thread with its own context and CUDA stream) and an HBM budget for the
 * estimated footprints of the admitted requests (Krylov basis, vectors,
 * operator tables, near band, scratch).  Requests are admitted first-fit from
 * the queue whenever a slot is free and the footprint fits; one that exceeds
 * the budget on its own runs when the GPU is otherwise idle. */
cfie_status cfie_server_create(int device, size_t hbm_budget_bytes, int slots, cfie_server** out);
/* Let a slot take up to max_requests queued requests at once (default 1): when
 * a slot becomes free it takes the first request that fits the budget, then
 * the further queued requests (in queue order) with the same precision, rtol,
 * restart and maxit and an n within a factor of two of the first one's that
 * fit alongside it, and solves them together as one cfie_batch (one lockstep
 * GMRES over all their right-hand sides: one set of Arnoldi launches and one
 * host synchronisation per step for the group; stored operators share one
 * persistent contraction launch per matvec, matrix-free ones still iterating
 * have their matvecs issued on up to eight concurrent streams).  Each request
 * keeps its own result, iteration counts, residuals and solution; the times
 * of a group's requests share its start and end.  Affects requests taken after the call.  CFIE_EINVAL for a
 * null server or max_requests outside [1, 256].  Not part of the paper (a
 * serving option). */
cfie_status cfie_server_set_batching(cfie_server* server, int max_requests);
/* Solve each request with at least min_rhs right-hand sides (min_rhs >= 1;
 * 0, the default, turns this off) and at least min_n nodes alone with block
 * GMRES over its directions (cfie_op_set_block_gmres; restart and maxit count
 * block steps), never in a lockstep batch.  Block GMRES takes about half the
 * steps on large obstacles but pays host work per step, which small ones do
 * not earn back.  Affects requests taken after the call.  CFIE_EINVAL for a
 * null server, min_rhs outside [0, 1024] or a negative min_n.  Not part of the
 * paper (a serving option; block GMRES is the block variant of its GMRES). */
cfie_status cfie_server_set_block_gmres(cfie_server* server, int min_rhs, int min_n);
/* Queue a request (arguments copied; never blocks).  *ticket identifies it. */
cfie_status cfie_server_submit(cfie_server* server, const cfie_request* req, long long* ticket);
/* State of a request; when done and x_host is not NULL, copies the solution
 * (n * nrhs complex128, column-major) to x_host. */
cfie_status cfie_server_poll(cfie_server* server, long long ticket, cfie_result* out,
                             void* x_host);
/* Wait until the queue is empty and no slot is busy (CFIE_ETIMEOUT otherwise). */
cfie_status cfie_server_wait_all(cfie_server* server, double timeout_s);
/* Forget a finished request and free its host solution. */
cfie_status cfie_server_release(cfie_server* server, long long ticket);
/* Counters of the server so far, copied to *out (host).  CFIE_EINVAL for a
 * null server or output. */
cfie_status cfie_server_stats(cfie_server* server, cfie_server_counters* out);
/* Message of the server's last failing call ("" if none); valid until its next
 * call.  Per-request failures: cfie_server_request_error. */
const char* cfie_server_last_error(cfie_server* server);
/* The error message of a finished request whose status is not CFIE_OK (empty
 * otherwise, or while it runs), copied NUL-terminated into buf (host, len
 * bytes, truncated to fit).  CFIE_EINVAL for an unknown ticket, a null
 * server or buffer, or len 0. */
cfie_status cfie_server_request_error(cfie_server* server, long long ticket, char* buf,
                                      size_t len);
/* Stop the slots (running solves finish first) and free everything. */
void cfie_server_destroy(cfie_server* server);

/* Kernel launches issued by the library in this process so far (all
 * contexts).  Never fails. */
long long cfie_launch_count(void);

/* --- Pipe issue rates (the denominators of the arithmetic rooflines) ----- */

/* Measured on the context's device with CUDA events: FP32 FMAs, MUFU
 * reciprocal square roots and FP64 FMAs per second, each from eight
 * independent dependency chains per thread on 8 CTAs of 256 threads per SM.
 * Not part of the paper's method: it measures the hardware the kernels run
 * on.  Synchronous; takes well under a second. */
typedef struct {
  int sms;
  double fp32_fma_per_s;
  double mufu_per_s;
  double fp64_fma_per_s;
} cfie_peaks;
cfie_status cfie_measure_peaks(cfie_ctx* ctx, cfie_peaks* out);

#ifdef __cplusplus
}
#endif
#endif /* CFIE_H */
