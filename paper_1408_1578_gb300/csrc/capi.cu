// C ABI of the CFIE library: argument checks, handle management, dispatch to
// the kernels and per-launch event timing.  Declarations and argument
// conventions are in include/cfie.h.
#include <cmath>
#include <cstring>
#include <new>

#include "internal.h"

long long g_cfie_launches = 0;

namespace {

template <class F>
cfie_status guarded(cfie_ctx* ctx, F&& f) {
  try {
    f();
    if (ctx) ctx->err.clear();
    return CFIE_OK;
  } catch (const cfie_error& e) {
    if (ctx) ctx->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->err = "host allocation failed";
    return CFIE_ENOMEM;
  } catch (...) {
    if (ctx) ctx->err = "unexpected exception";
    return CFIE_ECUDA;
  }
}

void set_device(cfie_ctx* c) { CFIE_CHECK_CUDA(cudaSetDevice(c->device)); }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

void check_vec(const void* p, const char* name) {
  if (!p) throw cfie_error(CFIE_EINVAL, std::string(name) + " is NULL");
  if (!aligned16(p)) throw cfie_error(CFIE_EINVAL, std::string(name) + " is not 16-byte aligned");
}

cfie_geom* new_geom(cfie_ctx* ctx, int kind) {
  cfie_geom* g = new cfie_geom();
  g->ctx = ctx;
  g->kind = kind;
  return g;
}

}  // namespace

// ---------------------------------------------------------------------------
// profiling
// ---------------------------------------------------------------------------
void prof_begin(cfie_ctx* c, int cls, cudaEvent_t* a) {
  *a = nullptr;
  if (!c->profiling) return;
  if (c->pool.empty()) {
    cudaEvent_t e;
    CFIE_CHECK_CUDA(cudaEventCreate(&e));
    c->pool.push_back(e);
  }
  *a = c->pool.back();
  c->pool.pop_back();
  CFIE_CHECK_CUDA(cudaEventRecord(*a, c->stream));
}

void prof_end(cfie_ctx* c, int cls, cudaEvent_t a) {
  if (!a) return;
  cudaEvent_t b;
  if (c->pool.empty()) {
    if (cudaEventCreate(&b) != cudaSuccess) return;
  } else {
    b = c->pool.back();
    c->pool.pop_back();
  }
  cudaEventRecord(b, c->stream);
  c->inflight.push_back({cls, a, b});
  if (c->inflight.size() > 4096) prof_harvest(c, true);
}

void prof_harvest(cfie_ctx* c, bool wait) {
  if (wait) cudaStreamSynchronize(c->stream);
  std::vector<cfie_ctx::pending> keep;
  for (auto& p : c->inflight) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->ms[p.cls] += ms;
      c->launches[p.cls] += 1;
      c->pool.push_back(p.a);
      c->pool.push_back(p.b);
    } else {
      keep.push_back(p);
    }
  }
  c->inflight.swap(keep);
}

void apply_inner(cfie_op* op, const double2* x, double2* y, int nrhs) {
  switch (op->prec) {
    case CFIE_FP64:
      matvec_fp64(op, x, y, nrhs);
      break;
    case CFIE_FP32_REFINED:
      matvec_fp32(op, x, y, nrhs);
      break;
    case CFIE_TENSOR_REFINED:
      matvec_stored(op, x, y, nrhs);
      break;
    default:
      throw cfie_error(CFIE_EINVAL, "precision not available for this operator");
  }
}

extern "C" {

cfie_status cfie_ctx_create(int device, void* cuda_stream, cfie_ctx** out) {
  if (!out) return CFIE_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) return CFIE_ECUDA;
  if (device < 0 || device >= count) return CFIE_EINVAL;
  cfie_ctx* c = new (std::nothrow) cfie_ctx();
  if (!c) return CFIE_ENOMEM;
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  cfie_status st = guarded(c, [&] { set_device(c); });
  if (st != CFIE_OK) {
    delete c;
    return st;
  }
  *out = c;
  return CFIE_OK;
}

void cfie_ctx_destroy(cfie_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  prof_harvest(ctx, true);
  for (auto& p : ctx->inflight) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  delete ctx;
}

const char* cfie_last_error(const cfie_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

cfie_status cfie_geometry_circle(cfie_ctx* ctx, double radius, cfie_geom** out) {
  if (!ctx || !out) return CFIE_EINVAL;
  return guarded(ctx, [&] {
    CFIE_REQUIRE(std::isfinite(radius) && radius > 0, "radius must be positive and finite");
    cfie_geom* g = new_geom(ctx, G_CIRCLE);
    g->p0 = radius;
    *out = g;
  });
}

cfie_status cfie_geometry_ellipse(cfie_ctx* ctx, double a, double b, cfie_geom** out) {
  if (!ctx || !out) return CFIE_EINVAL;
  return guarded(ctx, [&] {
    CFIE_REQUIRE(std::isfinite(a) && std::isfinite(b) && a > 0 && b > 0,
                 "ellipse semi-axes must be positive and finite");
    cfie_geom* g = new_geom(ctx, G_ELLIPSE);
    g->p0 = a;
    g->p1 = b;
    *out = g;
  });
}

cfie_status cfie_geometry_fourier_star(cfie_ctx* ctx, int K, const double* a, const double* b,
                                       cfie_geom** out) {
  if (!ctx || !out) return CFIE_EINVAL;
  return guarded(ctx, [&] {
    CFIE_REQUIRE(K >= 1 && K <= 64, "K must be in [1, 64]");
    CFIE_REQUIRE(a && b, "coefficient arrays must not be NULL");
    double bound = 0;
    for (int k = 0; k < K; ++k) {
      CFIE_REQUIRE(std::isfinite(a[k]) && std::isfinite(b[k]), "coefficients must be finite");
      bound += std::fabs(a[k]) + std::fabs(b[k]);
    }
    CFIE_REQUIRE(bound < 1.0, "sum |a_k| + |b_k| must stay below 1 so that r(t) > 0");
    cfie_geom* g = new_geom(ctx, G_STAR);
    g->a.assign(a, a + K);
    g->b.assign(b, b + K);
    *out = g;
  });
}

cfie_status cfie_geometry_kite(cfie_ctx* ctx, cfie_geom** out) {
  if (!ctx || !out) return CFIE_EINVAL;
  return guarded(ctx, [&] { *out = new_geom(ctx, G_KITE); });
}

cfie_status cfie_geometry_samples(cfie_ctx* ctx, int n, const double* z, const double* dz,
                                  const double* ddz, cfie_geom** out) {
  if (!ctx || !out) return CFIE_EINVAL;
  return guarded(ctx, [&] {
    CFIE_REQUIRE(n >= 8 && n % 2 == 0 && n <= (1 << 20), "n must be even and in [8, 2^20]");
    CFIE_REQUIRE(z && dz && ddz, "sample arrays must not be NULL");
    for (int i = 0; i < 2 * n; ++i) {
      CFIE_REQUIRE(std::isfinite(z[i]) && std::isfinite(dz[i]) && std::isfinite(ddz[i]),
                   "samples must be finite");
    }
    for (int i = 0; i < n; ++i)
      CFIE_REQUIRE(dz[2 * i] != 0.0 || dz[2 * i + 1] != 0.0, "z' must not vanish");
    cfie_geom* g = new_geom(ctx, G_SAMPLES);
    g->n_samples = n;
    g->z.assign(z, z + 2 * n);
    g->dz.assign(dz, dz + 2 * n);
    g->ddz.assign(ddz, ddz + 2 * n);
    *out = g;
  });
}

void cfie_geom_destroy(cfie_geom* geom) { delete geom; }

cfie_status cfie_discretise(cfie_geom* geom, int n, double omega, double eta, cfie_bc bc,
                            cfie_precision precision, cfie_layout layout, cfie_op** out) {
  if (!geom || !geom->ctx || !out) return CFIE_EINVAL;
  cfie_ctx* ctx = geom->ctx;
  *out = nullptr;
  cfie_op* op = nullptr;
  cfie_status st = guarded(ctx, [&] {
    CFIE_REQUIRE(n >= 8 && n % 2 == 0 && n <= (1 << 20), "n must be even and in [8, 2^20]");
    CFIE_REQUIRE(geom->kind != G_SAMPLES || geom->n_samples == n,
                 "n must equal the number of caller samples");
    CFIE_REQUIRE(std::isfinite(omega) && omega > 0, "omega must be positive and finite");
    CFIE_REQUIRE(std::isfinite(eta) && eta > 0, "eta must be positive and finite");
    CFIE_REQUIRE(bc == CFIE_SOUND_SOFT || bc == CFIE_SOUND_HARD, "unknown boundary condition");
    CFIE_REQUIRE(precision == CFIE_FP64 || precision == CFIE_FP32_REFINED ||
                     precision == CFIE_TENSOR_REFINED,
                 "unknown precision");
    CFIE_REQUIRE(layout == CFIE_MATRIX_FREE || layout == CFIE_STORED, "unknown layout");
    CFIE_REQUIRE((precision == CFIE_TENSOR_REFINED) == (layout == CFIE_STORED),
                 "the stored layout goes with CFIE_TENSOR_REFINED and only with it");
    set_device(ctx);
    op = new cfie_op();
    op->ctx = ctx;
    op->n = n;
    op->omega = omega;
    op->eta = eta;
    op->h = 2.0 * CFIE_PI / n;
    op->bc = bc;
    op->prec = precision;
    op->layout = layout;
    geometry_sample(op, geom);
    kress_tables(op);
    if (precision != CFIE_FP64) fp32_prepare(op);
    if (layout == CFIE_STORED) stored_prepare(op);
    CFIE_CHECK_CUDA(cudaStreamSynchronize(ctx->stream));
  });
  if (st != CFIE_OK) {
    if (op) cfie_op_destroy(op);
    return st;
  }
  *out = op;
  return CFIE_OK;
}

void cfie_op_destroy(cfie_op* op) {
  if (!op) return;
  cudaSetDevice(op->ctx->device);
  cudaStreamSynchronize(op->ctx->stream);
  if (op->host_res) cudaFreeHost(op->host_res);
  delete op;
}

int cfie_op_n(const cfie_op* op) { return op ? op->n : 0; }

cfie_status cfie_rhs_plane_waves(cfie_op* op, int nrhs, const double* theta, void* f_dev) {
  if (!op) return CFIE_EINVAL;
  return guarded(op->ctx, [&] {
    CFIE_REQUIRE(nrhs >= 1 && nrhs <= 1024, "nrhs must be in [1, 1024]");
    CFIE_REQUIRE(theta, "theta is NULL");
    for (int k = 0; k < nrhs; ++k) CFIE_REQUIRE(std::isfinite(theta[k]), "theta must be finite");
    check_vec(f_dev, "f");
    set_device(op->ctx);
    rhs_plane_waves(op, nrhs, theta, static_cast<double2*>(f_dev));
  });
}

cfie_status cfie_apply(cfie_op* op, const void* x_dev, void* y_dev, int nrhs) {
  if (!op) return CFIE_EINVAL;
  return guarded(op->ctx, [&] {
    CFIE_REQUIRE(nrhs >= 1 && nrhs <= 1024, "nrhs must be in [1, 1024]");
    check_vec(x_dev, "x");
    check_vec(y_dev, "y");
    CFIE_REQUIRE(x_dev != y_dev, "x and y must not overlap");
    set_device(op->ctx);
    apply_inner(op, static_cast<const double2*>(x_dev), static_cast<double2*>(y_dev), nrhs);
    if (op->layout == CFIE_STORED && stored_take_error(op))
      throw cfie_error(CFIE_ETIMEOUT, "tensor-core kernel gave up a bounded wait");
  });
}

cfie_status cfie_apply_fp64(cfie_op* op, const void* x_dev, void* y_dev, int nrhs) {
  if (!op) return CFIE_EINVAL;
  return guarded(op->ctx, [&] {
    CFIE_REQUIRE(nrhs >= 1 && nrhs <= 1024, "nrhs must be in [1, 1024]");
    check_vec(x_dev, "x");
    check_vec(y_dev, "y");
    CFIE_REQUIRE(x_dev != y_dev, "x and y must not overlap");
    set_device(op->ctx);
    matvec_fp64(op, static_cast<const double2*>(x_dev), static_cast<double2*>(y_dev), nrhs);
  });
}

cfie_status cfie_apply_fp64_static(cfie_op* op, const void* x_dev, void* y_dev, int nrhs) {
  if (!op) return CFIE_EINVAL;
  return guarded(op->ctx, [&] {
    CFIE_REQUIRE(nrhs >= 1 && nrhs <= 1024, "nrhs must be in [1, 1024]");
    check_vec(x_dev, "x");
    check_vec(y_dev, "y");
    CFIE_REQUIRE(x_dev != y_dev, "x and y must not overlap");
    set_device(op->ctx);
    matvec_fp64_static(op, static_cast<const double2*>(x_dev), static_cast<double2*>(y_dev),
                       nrhs);
  });
}

cfie_status cfie_gmres_solve(cfie_op* op, const void* f_dev, void* x_dev, int nrhs, double rtol,
                             int restart, int maxit, int* iters_out, double* relres_out) {
  if (!op) return CFIE_EINVAL;
  cfie_status result = CFIE_OK;
  cfie_status st = guarded(op->ctx, [&] {
    CFIE_REQUIRE(nrhs >= 1 && nrhs <= 1024, "nrhs must be in [1, 1024]");
    CFIE_REQUIRE(std::isfinite(rtol) && rtol > 0 && rtol < 1, "rtol must be in (0, 1)");
    CFIE_REQUIRE(restart >= 0 && restart <= 512, "restart must be in [0, 512]");
    CFIE_REQUIRE(maxit >= 1, "maxit must be positive");
    CFIE_REQUIRE(restart > 0 || maxit <= 512, "unrestarted GMRES allows at most 512 steps");
    check_vec(f_dev, "f");
    check_vec(x_dev, "x");
    CFIE_REQUIRE(f_dev != x_dev, "f and x must not overlap");
    set_device(op->ctx);
    gmres_solve(op, static_cast<const double2*>(f_dev), static_cast<double2*>(x_dev), nrhs, rtol,
                restart, maxit, iters_out, relres_out, &result);
    if (op->layout == CFIE_STORED && stored_take_error(op))
      throw cfie_error(CFIE_ETIMEOUT, "tensor-core kernel gave up a bounded wait");
    if (result == CFIE_ENOCONV) op->ctx->err = "GMRES reached maxit before rtol";
  });
  if (st != CFIE_OK) return st;
  return result;
}

cfie_status cfie_op_last_stats(const cfie_op* op, cfie_solve_stats* out) {
  if (!op || !out) return CFIE_EINVAL;
  *out = op->stats;
  return CFIE_OK;
}

cfie_status cfie_ctx_set_profiling(cfie_ctx* ctx, int on) {
  if (!ctx) return CFIE_EINVAL;
  return guarded(ctx, [&] {
    set_device(ctx);
    prof_harvest(ctx, true);
    for (int k = 0; k < CFIE_K_COUNT; ++k) {
      ctx->ms[k] = 0;
      ctx->launches[k] = 0;
    }
    ctx->profiling = on != 0;
  });
}

cfie_status cfie_ctx_kernel_times(cfie_ctx* ctx, double* ms, long long* launches) {
  if (!ctx || !ms || !launches) return CFIE_EINVAL;
  return guarded(ctx, [&] {
    set_device(ctx);
    prof_harvest(ctx, true);
    for (int k = 0; k < CFIE_K_COUNT; ++k) {
      ms[k] = ctx->ms[k];
      launches[k] = ctx->launches[k];
    }
  });
}

long long cfie_launch_count(void) { return g_cfie_launches; }

}  // extern "C"
