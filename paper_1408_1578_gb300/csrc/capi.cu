// C ABI of the CFIE library: argument checks, handle management, dispatch to
// the kernels and per-launch event timing.  Declarations and argument
// conventions are in include/cfie.h.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <new>
#include <tuple>

#include "internal.h"

std::atomic<long long> g_cfie_launches{0};

namespace {

template <class F>
cfie_status guarded(cfie_ctx* ctx, F&& f) {
  stream_scope ss(ctx ? ctx->stream : alloc_stream());
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
  if (!c->profiling || c->prof_suspend > 0) return;
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

namespace {

// Process-wide choice between the two FP32 matvec variants, keyed by
// (boundary condition, n, nrhs): each is timed once with CUDA events on the
// operator's stream and the faster one is kept.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tuned;

int tuned_variant(cfie_op* op, const double2* x, double2* y, int nrhs) {
  if (op->variant) return op->variant;
  // decisions are shared by operators of similar shape (n up to the next power
  // of two, right-hand sides in octaves), so that a server seeing a new n and
  // nrhs with every request does not time both variants every time
  int nb = 1, rb = 1;
  while (nb < op->n) nb *= 2;
  while (rb * 2 <= std::min(nrhs, 64)) rb *= 2;
  const auto key = std::make_tuple((int)op->bc, nb, rb);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
  }
  cudaStream_t st = op->ctx->stream;
  cudaEvent_t e[3];
  for (auto& ev : e) CFIE_CHECK_CUDA(cudaEventCreate(&ev));
  float t[2] = {0.f, 0.f};
  for (int v = 0; v < 2; ++v) {
    auto run = [&] { v == 0 ? matvec_fp32(op, x, y, nrhs) : matvec_fp32_tc(op, x, y, nrhs); };
    run();  // warm-up (plans, attributes)
    CFIE_CHECK_CUDA(cudaEventRecord(e[0], st));
    run();
    CFIE_CHECK_CUDA(cudaEventRecord(e[1], st));
    CFIE_CHECK_CUDA(cudaEventSynchronize(e[1]));
    CFIE_CHECK_CUDA(cudaEventElapsedTime(&t[v], e[0], e[1]));
  }
  for (auto& ev : e) cudaEventDestroy(ev);
  const int choice = t[1] < t[0] ? 2 : 1;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[key] = choice;
  return choice;
}

}  // namespace

void matvec_residual(cfie_op* op, const double2* x, double2* y, int nrhs) {
  if (op->prec != CFIE_FP64 && df_available(op))
    matvec_df(op, x, y, nrhs);
  else
    matvec_fp64(op, x, y, nrhs);
}

void apply_inner(cfie_op* op, const double2* x, double2* y, int nrhs) {
  switch (op->prec) {
    case CFIE_FP64:
      op->stats.matvec_variant = 0;
      matvec_fp64(op, x, y, nrhs);
      break;
    case CFIE_FP32_REFINED:
      op->stats.matvec_variant = tuned_variant(op, x, y, nrhs);
      if (op->stats.matvec_variant == 2)
        matvec_fp32_tc(op, x, y, nrhs);
      else
        matvec_fp32(op, x, y, nrhs);
      break;
    case CFIE_TENSOR_REFINED:
      op->stats.matvec_variant = 3;
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
  cfie_status st = guarded(c, [&] {
    set_device(c);
    // keep freed device buffers in the stream-ordered pool between calls
    // (operators and batches are created and destroyed at every solve)
    cudaMemPool_t pool;
    CFIE_CHECK_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t keep = UINT64_MAX;
    CFIE_CHECK_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
  });
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

cfie_status cfie_discretise_many(int count, cfie_geom* const* geoms, const int* n,
                                 const double* omega, const double* eta, cfie_bc bc,
                                 cfie_precision precision, cfie_layout layout, cfie_op** out) {
  if (count < 1 || !geoms || !n || !omega || !eta || !out || !geoms[0] || !geoms[0]->ctx)
    return CFIE_EINVAL;
  cfie_ctx* ctx = geoms[0]->ctx;
  for (int k = 0; k < count; ++k) out[k] = nullptr;
  for (int k = 0; k < count; ++k)
    if (!geoms[k] || geoms[k]->ctx != ctx) {
      ctx->err = "every geometry must belong to one context";
      return CFIE_EINVAL;
    }
  // each worker sets its operators up on a context and stream of its own
  // (the request server's slots do the same), then hands them to the
  // geometries' context once its stream has finished
  const int K = std::min(count, 8);
  std::vector<cfie_status> st(count, CFIE_OK);
  std::vector<std::string> msg(count);
  std::vector<std::thread> workers;
  auto work = [&](int t) {
    cudaSetDevice(ctx->device);
    cudaStream_t s = nullptr;
    cfie_ctx* wc = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cfie_ctx_create(ctx->device, s, &wc) != CFIE_OK) {
      for (int k = t; k < count; k += K) {
        st[k] = CFIE_ECUDA;
        msg[k] = "could not create a worker stream / context";
      }
      if (s) cudaStreamDestroy(s);
      return;
    }
    for (int k = t; k < count; k += K) {
      try {
        cfie_geom g = *geoms[k];   // the same curve, on the worker's context
        g.ctx = wc;
        st[k] = cfie_discretise(&g, n[k], omega[k], eta[k], bc, precision, layout, &out[k]);
        if (st[k] != CFIE_OK) msg[k] = wc->err;
      } catch (...) {
        st[k] = CFIE_ENOMEM;
        msg[k] = "host allocation failed";
      }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess)
      for (int k = t; k < count; k += K)
        if (st[k] == CFIE_OK) {
          st[k] = CFIE_ECUDA;
          msg[k] = "worker stream failed";
        }
    for (int k = t; k < count; k += K)
      if (out[k]) out[k]->ctx = ctx;
    cfie_ctx_destroy(wc);
    cudaStreamDestroy(s);
  };
  // a worker thread that cannot be started does its share on this thread
  for (int t = 0; t < K; ++t) {
    try {
      workers.emplace_back(work, t);
    } catch (...) {
      work(t);
    }
  }
  for (auto& w : workers) w.join();
  for (int k = 0; k < count; ++k)
    if (st[k] != CFIE_OK) {
      for (int q = 0; q < count; ++q) {
        cfie_op_destroy(out[q]);
        out[q] = nullptr;
      }
      ctx->err = msg[k];
      return st[k];
    }
  ctx->err.clear();
  return CFIE_OK;
}

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
    if (bc == CFIE_SOUND_HARD) fft_prepare(op);
    if (precision != CFIE_FP64) fp32_prepare(op);
    if (precision != CFIE_FP64) df_prepare(op);
    if (precision != CFIE_FP64) fp32_band(op);
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
  stream_scope ss(op->ctx->stream);
  cudaStreamSynchronize(op->ctx->stream);
  krylov_release(op->K);
  gemm_plan_release(op->plan);
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
    if (op->prec == CFIE_FP32_REFINED && tc_take_error(op))
      throw cfie_error(CFIE_ETIMEOUT, "tensor-core kernel gave up a bounded wait");
    if (op->prec != CFIE_FP64 && df_take_error(op))
      throw cfie_error(CFIE_ETIMEOUT, "tensor-core kernel gave up a bounded wait");
  });
}

cfie_status cfie_op_set_variant(cfie_op* op, int variant) {
  if (!op) return CFIE_EINVAL;
  return guarded(op->ctx, [&] {
    CFIE_REQUIRE(variant >= 0 && variant <= 2, "variant must be 0, 1 or 2");
    CFIE_REQUIRE(variant != 2 || op->prec == CFIE_FP32_REFINED,
                 "the tensor-core variant needs a CFIE_FP32_REFINED operator");
    op->variant = variant;
  });
}

cfie_status cfie_apply_residual(cfie_op* op, const void* x_dev, void* y_dev, int nrhs) {
  if (!op) return CFIE_EINVAL;
  return guarded(op->ctx, [&] {
    CFIE_REQUIRE(nrhs >= 1 && nrhs <= 1024, "nrhs must be in [1, 1024]");
    check_vec(x_dev, "x");
    check_vec(y_dev, "y");
    CFIE_REQUIRE(x_dev != y_dev, "x and y must not overlap");
    set_device(op->ctx);
    matvec_residual(op, static_cast<const double2*>(x_dev), static_cast<double2*>(y_dev), nrhs);
    if (op->prec != CFIE_FP64 && df_take_error(op))
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
    cudaStream_t st = op->ctx->stream;
    if (op->ps_nrhs != nrhs) {
      pset_uniform(op->ps, op->n, nrhs, st);
      op->ps_nrhs = nrhs;
    }
    if (op->block_gmres) {
      block_gmres_solve(op, static_cast<const double2*>(f_dev), static_cast<double2*>(x_dev), nrhs,
                        rtol, restart, maxit, iters_out, relres_out, &result, op->bgws);
    } else {
    solve_fns fns;
    fns.inner = [op, nrhs](const double2* a, double2* b) { apply_inner(op, a, b, nrhs); };
    fns.fp64 = [op, nrhs](const double2* a, double2* b) { matvec_residual(op, a, b, nrhs); };
    if (op->dirprec) {
      cfie_dirprec* P = op->dirprec;
      fns.prec = [P, nrhs](const double2* a, double2* b) { dirprec_apply(P, a, b, nrhs); };
    }
    fns.basis32 = op->basis32 != 0;
    gmres_set(st, op->ctx, op->K, op->ps, fns, op->prec != CFIE_FP64,
              static_cast<const double2*>(f_dev), static_cast<double2*>(x_dev), rtol, restart,
              maxit, iters_out, relres_out, &result, op->stats);
    }
    if (op->layout == CFIE_STORED && stored_take_error(op))
      throw cfie_error(CFIE_ETIMEOUT, "tensor-core kernel gave up a bounded wait");
    if (op->prec == CFIE_FP32_REFINED && tc_take_error(op))
      throw cfie_error(CFIE_ETIMEOUT, "tensor-core kernel gave up a bounded wait");
    if (op->prec != CFIE_FP64 && df_take_error(op))
      throw cfie_error(CFIE_ETIMEOUT, "tensor-core kernel gave up a bounded wait");
    if (result == CFIE_ENOCONV) op->ctx->err = "GMRES reached maxit before rtol";
  });
  if (st != CFIE_OK) return st;
  return result;
}

cfie_status cfie_field_eval(cfie_op* op, const void* q_dev, int nrhs, int npts,
                            const void* pts_dev, void* u_dev) {
  if (!op) return CFIE_EINVAL;
  return guarded(op->ctx, [&] {
    CFIE_REQUIRE(nrhs >= 1 && nrhs <= 1024, "nrhs must be in [1, 1024]");
    CFIE_REQUIRE(npts >= 1, "npts must be positive");
    check_vec(q_dev, "q");
    check_vec(pts_dev, "pts");
    check_vec(u_dev, "u");
    CFIE_REQUIRE(u_dev != q_dev && u_dev != pts_dev, "u must not overlap q or pts");
    set_device(op->ctx);
    field_eval(op, static_cast<const double2*>(q_dev), nrhs, npts,
               static_cast<const double2*>(pts_dev), static_cast<double2*>(u_dev));
  });
}

cfie_status cfie_measure_peaks(cfie_ctx* ctx, cfie_peaks* out) {
  if (!ctx || !out) return CFIE_EINVAL;
  return guarded(ctx, [&] {
    set_device(ctx);
    measure_peaks(ctx, out);
  });
}

cfie_status cfie_op_set_residual_variant(cfie_op* op, int variant) {
  if (!op || variant < 0 || variant > 2) return CFIE_EINVAL;
  return guarded(op->ctx, [&] {
    CFIE_REQUIRE(op->prec != CFIE_FP64, "the FP64 precision computes residuals with its own matvec");
    op->res_variant = variant;
  });
}

cfie_status cfie_op_set_inner_basis(cfie_op* op, int fp32) {
  if (!op || (fp32 != 0 && fp32 != 1)) return CFIE_EINVAL;
  op->basis32 = fp32;
  return CFIE_OK;
}

cfie_status cfie_batch_set_inner_basis(cfie_batch* b, int fp32) {
  if (!b || (fp32 != 0 && fp32 != 1)) return CFIE_EINVAL;
  b->basis32 = fp32;
  return CFIE_OK;
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

long long cfie_launch_count(void) { return g_cfie_launches.load(); }

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------
// Whether operator k of a batch has a problem in the running Arnoldi step
// (every operator outside one).  The others' outputs are not read.
static bool batch_live(const cfie_batch* b, size_t k) {
  const std::vector<int>& live = b->K.live;
  if (live.empty()) return true;
  for (int r = 0; r < b->nrhs[k]; ++r)
    if (live[(size_t)b->pfirst[k] + r]) return true;
  return false;
}

// The operators' matvecs are independent: fn(k) for every live operator, on
// up to eight auxiliary streams forked from and joined back into the context
// stream (the operators' kernels launch on ctx->stream, which points at the
// auxiliary stream while that operator's work is issued), timed as one scope
// of class cls.
extern "C++" {
template <class F>
static void batch_each(cfie_batch* b, int cls, F&& fn) {
  cfie_ctx* c = b->ctx;
  std::vector<size_t> ks;
  for (size_t k = 0; k < b->ops.size(); ++k)
    if (batch_live(b, k)) ks.push_back(k);
  const int K = (int)std::min<size_t>(8, ks.size());
  if (K <= 1) {
    for (size_t k : ks) fn(k);
    return;
  }
  while ((int)b->aux.size() < K) {
    cudaStream_t s;
    CFIE_CHECK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    b->aux.push_back(s);
    cudaEvent_t e;
    CFIE_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->aux_ev.push_back(e);
  }
  cudaEvent_t fork;
  CFIE_CHECK_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  cudaStream_t main = c->stream;
  prof_scope ps(c, cls);
  CFIE_CHECK_CUDA(cudaEventRecord(fork, main));
  for (int q = 0; q < K; ++q) CFIE_CHECK_CUDA(cudaStreamWaitEvent(b->aux[q], fork, 0));
  c->prof_suspend++;
  auto join = [&] {
    c->stream = main;
    c->prof_suspend--;
    for (int q = 0; q < K; ++q) {
      cudaEventRecord(b->aux_ev[q], b->aux[q]);
      cudaStreamWaitEvent(main, b->aux_ev[q], 0);
    }
    cudaEventDestroy(fork);
  };
  try {
    for (size_t i = 0; i < ks.size(); ++i) {
      c->stream = b->aux[i % K];
      stream_scope ss(c->stream);
      fn(ks[i]);
    }
  } catch (...) {
    join();
    throw;
  }
  join();
  CFIE_CHECK_CUDA(cudaGetLastError());
}
}  // extern "C++"

static void batch_inner(cfie_batch* b, const double2* x, double2* y) {
  if (b->all_stored) {
    gemm_plan_run(b->plan, b->ctx, x, y);
    return;
  }
  const int cls = b->prec == CFIE_FP64              ? CFIE_K_MATVEC_FP64
                  : b->prec == CFIE_TENSOR_REFINED ? CFIE_K_MATVEC_TENSOR
                                                   : CFIE_K_MATVEC_FP32;
  batch_each(b, cls, [&](size_t k) {
    apply_inner(b->ops[k], x + b->off[k], y + b->off[k], b->nrhs[k]);
  });
}

static void batch_fp64(cfie_batch* b, const double2* x, double2* y) {
  batch_each(b, CFIE_K_MATVEC_FP64, [&](size_t k) {
    matvec_residual(b->ops[k], x + b->off[k], y + b->off[k], b->nrhs[k]);
  });
}

cfie_status cfie_batch_create(cfie_ctx* ctx, int count, cfie_op* const* ops, const int* nrhs,
                              cfie_batch** out) {
  if (!ctx || !out) return CFIE_EINVAL;
  *out = nullptr;
  cfie_batch* b = nullptr;
  cfie_status st = guarded(ctx, [&] {
    CFIE_REQUIRE(count >= 1 && count <= 65535, "count must be in [1, 65535]");
    CFIE_REQUIRE(ops && nrhs, "ops and nrhs must not be NULL");
    set_device(ctx);
    b = new cfie_batch();
    b->ctx = ctx;
    b->all_stored = true;
    std::vector<size_t> poff;
    std::vector<int> plen;
    long long at = 0;
    for (int k = 0; k < count; ++k) {
      CFIE_REQUIRE(ops[k] && ops[k]->ctx == ctx, "every operator must belong to the context");
      CFIE_REQUIRE(nrhs[k] >= 1 && nrhs[k] <= 1024, "nrhs must be in [1, 1024]");
      CFIE_REQUIRE(ops[k]->prec == ops[0]->prec, "operators of a batch share one precision");
      b->ops.push_back(ops[k]);
      b->nrhs.push_back(nrhs[k]);
      b->off.push_back(at);
      b->pfirst.push_back((int)poff.size());
      for (int r = 0; r < nrhs[k]; ++r) {
        poff.push_back((size_t)(at + (long long)r * ops[k]->n));
        plen.push_back(ops[k]->n);
      }
      at += (long long)ops[k]->n * nrhs[k];
      b->all_stored = b->all_stored && ops[k]->layout == CFIE_STORED;
    }
    b->L = (size_t)at;
    b->prec = ops[0]->prec;
    pset_build(b->ps, poff, plen, ctx->stream);
    if (b->all_stored && ctx->tune_batches)
      gemm_plan_tune(b->plan, ctx, b->ops, b->nrhs, b->off, b->L, b->tune_ms);
    else if (b->all_stored)
      gemm_plan_build(b->plan, ctx, b->ops, b->nrhs, b->off, GEMM_DEAL_AUTO);
  });
  if (st != CFIE_OK) {
    if (b) cfie_batch_destroy(b);
    return st;
  }
  *out = b;
  return CFIE_OK;
}

long long cfie_batch_length(const cfie_batch* b) { return b ? (long long)b->L : 0; }

cfie_status cfie_batch_apply(cfie_batch* b, const void* x_dev, void* y_dev) {
  if (!b) return CFIE_EINVAL;
  return guarded(b->ctx, [&] {
    check_vec(x_dev, "x");
    check_vec(y_dev, "y");
    CFIE_REQUIRE(x_dev != y_dev, "x and y must not overlap");
    set_device(b->ctx);
    batch_inner(b, static_cast<const double2*>(x_dev), static_cast<double2*>(y_dev));
    if (b->all_stored && gemm_plan_take_error(b->plan, b->ctx))
      throw cfie_error(CFIE_ETIMEOUT, "tensor-core kernel gave up a bounded wait");
  });
}

cfie_status cfie_batch_gmres_solve(cfie_batch* b, const void* f_dev, void* x_dev, double rtol,
                                   int restart, int maxit, int* iters_out, double* relres_out) {
  if (!b) return CFIE_EINVAL;
  cfie_status result = CFIE_OK;
  cfie_status st = guarded(b->ctx, [&] {
    CFIE_REQUIRE(std::isfinite(rtol) && rtol > 0 && rtol < 1, "rtol must be in (0, 1)");
    CFIE_REQUIRE(restart >= 0 && restart <= 512, "restart must be in [0, 512]");
    CFIE_REQUIRE(maxit >= 1, "maxit must be positive");
    CFIE_REQUIRE(restart > 0 || maxit <= 512, "unrestarted GMRES allows at most 512 steps");
    check_vec(f_dev, "f");
    check_vec(x_dev, "x");
    CFIE_REQUIRE(f_dev != x_dev, "f and x must not overlap");
    set_device(b->ctx);
    solve_fns fns;
    fns.inner = [b](const double2* a, double2* c) { batch_inner(b, a, c); };
    fns.fp64 = [b](const double2* a, double2* c) { batch_fp64(b, a, c); };
    fns.basis32 = b->basis32 != 0;
    gmres_set(b->ctx->stream, b->ctx, b->K, b->ps, fns, b->prec != CFIE_FP64,
              static_cast<const double2*>(f_dev), static_cast<double2*>(x_dev), rtol, restart,
              maxit, iters_out, relres_out, &result, b->stats);
    b->stats.matvec_variant = b->all_stored ? 3 : b->ops.empty() ? 0 : b->ops[0]->stats.matvec_variant;
    b->stats.residual_variant = b->ops.empty() ? 0 : b->ops[0]->stats.residual_variant;
    if (b->all_stored && gemm_plan_take_error(b->plan, b->ctx))
      throw cfie_error(CFIE_ETIMEOUT, "tensor-core kernel gave up a bounded wait");
    for (cfie_op* o : b->ops)
      if (o->prec != CFIE_FP64 && df_take_error(o))
        throw cfie_error(CFIE_ETIMEOUT, "tensor-core kernel gave up a bounded wait");
    if (result == CFIE_ENOCONV) b->ctx->err = "GMRES reached maxit before rtol";
  });
  if (st != CFIE_OK) return st;
  return result;
}

cfie_status cfie_batch_last_stats(const cfie_batch* b, cfie_solve_stats* out) {
  if (!b || !out) return CFIE_EINVAL;
  *out = b->stats;
  return CFIE_OK;
}

void cfie_batch_destroy(cfie_batch* b) {
  if (!b) return;
  cudaSetDevice(b->ctx->device);
  stream_scope ss(b->ctx->stream);
  cudaStreamSynchronize(b->ctx->stream);
  krylov_release(b->K);
  gemm_plan_release(b->plan);
  for (cudaStream_t s : b->aux) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t e : b->aux_ev) cudaEventDestroy(e);
  delete b;
}

}  // extern "C"

// --- directional preconditioner (Section 2) ---------------------------------

cfie_status cfie_dirprec_create(cfie_op* op, cfie_curve kind, const double* params, int nparams,
                                int q, int p, int m_leaf, int t_keep, cfie_dirprec** out) {
  if (!op || !out) return CFIE_EINVAL;
  *out = nullptr;
  cfie_dirprec* P = new (std::nothrow) cfie_dirprec;
  if (!P) return CFIE_ENOMEM;
  cfie_status st = guarded(op->ctx, [&] {
    set_device(op->ctx);
    dirprec_build(P, op, kind, params, nparams, q, p, m_leaf, t_keep);
  });
  if (st != CFIE_OK) {
    stream_scope ss(op->ctx->stream);
    delete P;
    return st;
  }
  *out = P;
  return CFIE_OK;
}

void cfie_dirprec_destroy(cfie_dirprec* P) {
  if (!P) return;
  if (P->ctx) {
    cudaSetDevice(P->ctx->device);
    stream_scope ss(P->ctx->stream);
    cudaStreamSynchronize(P->ctx->stream);
    delete P;
  } else {
    delete P;
  }
}

cfie_status cfie_dirprec_apply(cfie_dirprec* P, const void* x_dev, void* y_dev, int nrhs) {
  if (!P || !P->ctx) return CFIE_EINVAL;
  return guarded(P->ctx, [&] {
    CFIE_REQUIRE(nrhs >= 1 && nrhs <= 1024, "nrhs must be in [1, 1024]");
    check_vec(x_dev, "x");
    check_vec(y_dev, "y");
    CFIE_REQUIRE(x_dev != y_dev, "x and y must not overlap");
    set_device(P->ctx);
    dirprec_apply(P, static_cast<const double2*>(x_dev), static_cast<double2*>(y_dev), nrhs);
  });
}

cfie_status cfie_dirprec_coefficients(const cfie_dirprec* P, int* m, double* e) {
  if (!P || !m) return CFIE_EINVAL;
  *m = dirprec_segments(P, e);
  return CFIE_OK;
}

cfie_status cfie_op_set_preconditioner(cfie_op* op, cfie_dirprec* P) {
  if (!op) return CFIE_EINVAL;
  return guarded(op->ctx, [&] {
    CFIE_REQUIRE(!P || (P->ctx == op->ctx && dirprec_n(P) == op->n),
                 "the preconditioner was built for another operator or context");
    op->dirprec = P;
  });
}

cfie_status cfie_op_set_block_gmres(cfie_op* op, int on) {
  if (!op || (on != 0 && on != 1)) return CFIE_EINVAL;
  op->block_gmres = on;
  return CFIE_OK;
}

cfie_status cfie_batch_tuning(const cfie_batch* b, int* dealing, float* ms) {
  if (!b || !dealing) return CFIE_EINVAL;
  *dealing = b->all_stored ? b->plan.dealing : -1;
  if (ms)
    for (int d = 0; d < 3; ++d) ms[d] = b->tune_ms[d];
  return CFIE_OK;
}

cfie_status cfie_batch_set_dealing(cfie_batch* b, int dealing) {
  if (!b || dealing < 0 || dealing > 2) return CFIE_EINVAL;
  return guarded(b->ctx, [&] {
    CFIE_REQUIRE(b->all_stored, "only a batch of stored operators has a contraction plan");
    set_device(b->ctx);
    gemm_plan_build(b->plan, b->ctx, b->ops, b->nrhs, b->off, dealing);
  });
}
