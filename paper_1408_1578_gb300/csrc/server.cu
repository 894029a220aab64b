// Request server: continuous batching of independent CFIE solves on one GPU.
//
// Requests (an obstacle, a frequency, a boundary condition, a block of
// incidence directions, a target residual) are queued on the host.  A fixed
// set of slots, each a host thread with its own library context and CUDA
// stream, admits queued requests while their estimated device footprint (Krylov
// basis, work vectors, operator tables, near-field band, matvec scratch) fits in
// the HBM budget; a request that arrives while others run is admitted as soon as
// a slot and memory free up, and its kernels overlap on the GPU with the other
// slots' kernels.  With batching on, a free slot takes several compatible
// queued requests at once and solves them as one lockstep batch.  Each slot runs the whole path for its request: geometry and
// Kress tables, plane-wave data, refined GMRES; the Krylov basis stays on the
// device for the life of the solve.  Finished requests keep their solution and
// timing on the host until released.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <numeric>
#include <thread>
#include <unordered_map>

#include "internal.h"

namespace {

using clock_type = std::chrono::steady_clock;

struct request_rec {
  long long ticket = 0;
  cfie_request req{};
  std::vector<double> a, b, theta;
  size_t footprint = 0;
  clock_type::time_point t_submit, t_start, t_done;
  bool started = false, done = false;
  cfie_status status = CFIE_OK;
  int iters_max = 0;
  double relres_max = 0.0;
  std::vector<double2> x;  // solution (n * nrhs), host
  std::string err;
};

size_t footprint_bytes(const cfie_request& r) {
  const size_t n = (size_t)r.n, k = (size_t)r.nrhs;
  const size_t m = (size_t)(r.restart > 0 ? r.restart : r.maxit);
  const size_t vec = n * k * 16;
  const size_t ops = r.bc == CFIE_SOUND_HARD ? 4 : 1;
  // Krylov basis: FP32 for the inner solves of the refined precisions (plus
  // the FP32 work vector and the FP64 matvec input), FP64 otherwise
  size_t f = r.precision == CFIE_FP64 ? vec * (m + 1) : vec / 2 * (m + 2) + vec;
  f += vec * 8;                       // w, r, d, rin, f, x, staging
  f += n * 129 * 8 * 2;               // near-field band (b <= 64), both operators
  f += vec / 2 * (16 * ops + 3);      // FP32 split partials and staging
  f += vec * 4 * ops;                 // FP64 residual partials (a few splits)
  f += n * 200 + ((size_t)64 << 20);  // tables, small buffers, slack
  if (r.precision == CFIE_TENSOR_REFINED) {
    const size_t pitch = (n + 63) / 64 * 64, rows = (n + 127) / 128 * 128;
    f += 8 * rows * pitch;              // stored bf16 hi/lo planes (re, im), whole row blocks
    f += vec * 2;                       // contraction operand and partial sums
  }
  return f;
}

}  // namespace

struct cfie_server {
  int device = 0;
  size_t budget = 0, in_use = 0;
  int slots = 0;
  int batch_max = 1;   // requests a slot takes at once and solves as one batch
  int block_min = 0;   // requests with at least this many right-hand sides ...
  int block_min_n = 0; // ... and nodes: block GMRES (block_min 0: off)
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<request_rec*> queue;
  std::unordered_map<long long, std::unique_ptr<request_rec>> all;
  long long next = 1;
  bool stop = false;
  std::string err;
  long long completed = 0, solves = 0, peak_running = 0, running = 0;
  size_t peak_in_use = 0;
};

namespace {

// The tensor-core form stores its matrix; the others evaluate it on the fly.
cfie_layout layout_of(const cfie_request& q) {
  return q.precision == CFIE_TENSOR_REFINED ? CFIE_STORED : CFIE_MATRIX_FREE;
}

void run_request(cfie_ctx* ctx, request_rec* r, bool block, dbuf& fbuf, dbuf& xbuf) {
  const cfie_request& q = r->req;
  cfie_geom* geom = nullptr;
  cfie_op* op = nullptr;
  auto fail = [&](cfie_status s) {
    r->status = s;
    r->err = cfie_last_error(ctx);
  };
  cfie_status s = cfie_geometry_fourier_star(ctx, q.K, r->a.data(), r->b.data(), &geom);
  if (s != CFIE_OK) return fail(s);
  s = cfie_discretise(geom, q.n, q.omega, q.eta, (cfie_bc)q.bc, (cfie_precision)q.precision,
                      layout_of(q), &op);
  cfie_geom_destroy(geom);
  if (s != CFIE_OK) return fail(s);
  if (block) cfie_op_set_block_gmres(op, 1);
  const size_t len = (size_t)q.n * q.nrhs;
  try {
    fbuf.reserve(sizeof(double2) * len);
    xbuf.reserve(sizeof(double2) * len);
    CFIE_CHECK_CUDA(cudaMemsetAsync(xbuf.p, 0, sizeof(double2) * len, ctx->stream));
  } catch (const cfie_error& e) {
    cfie_op_destroy(op);
    r->status = e.code;
    r->err = e.msg;
    return;
  }
  s = cfie_rhs_plane_waves(op, q.nrhs, r->theta.data(), fbuf.p);
  if (s != CFIE_OK) {
    fail(s);
    cfie_op_destroy(op);
    return;
  }
  std::vector<int> its(q.nrhs);
  std::vector<double> rel(q.nrhs);
  s = cfie_gmres_solve(op, fbuf.p, xbuf.p, q.nrhs, q.rtol, q.restart, q.maxit, its.data(),
                       rel.data());
  r->status = s;
  if (s != CFIE_OK) r->err = cfie_last_error(ctx);
  for (int k = 0; k < q.nrhs; ++k) {
    r->iters_max = std::max(r->iters_max, its[k]);
    r->relres_max = std::max(r->relres_max, rel[k]);
  }
  r->x.resize(len);
  if (cudaMemcpyAsync(r->x.data(), xbuf.p, sizeof(double2) * len, cudaMemcpyDeviceToHost,
                      ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    r->status = CFIE_ECUDA;
    r->err = "copying the solution back failed";
  }
  cfie_op_destroy(op);
}

// Several requests of one slot solved as one batch: their operators in one
// cfie_batch, one lockstep refined GMRES over all their right-hand sides (one
// set of Arnoldi launches and one host synchronisation per step for all of
// them, the matvecs of the operators still iterating issued on concurrent
// streams), each request's solution copied back from its block.
void run_batch(cfie_ctx* ctx, const std::vector<request_rec*>& rs, dbuf& fbuf, dbuf& xbuf) {
  std::vector<cfie_op*> ops;
  std::vector<request_rec*> live;
  std::vector<int> nr;
  for (request_rec* r : rs) {
    const cfie_request& q = r->req;
    cfie_geom* geom = nullptr;
    cfie_op* op = nullptr;
    cfie_status s = cfie_geometry_fourier_star(ctx, q.K, r->a.data(), r->b.data(), &geom);
    if (s == CFIE_OK) {
      s = cfie_discretise(geom, q.n, q.omega, q.eta, (cfie_bc)q.bc, (cfie_precision)q.precision,
                          layout_of(q), &op);
      cfie_geom_destroy(geom);
    }
    if (s != CFIE_OK) {
      r->status = s;
      r->err = cfie_last_error(ctx);
      continue;
    }
    ops.push_back(op);
    live.push_back(r);
    nr.push_back(q.nrhs);
  }
  auto cleanup = [&] {
    for (cfie_op* op : ops) cfie_op_destroy(op);
  };
  if (live.empty()) return;
  cfie_batch* batch = nullptr;
  cfie_status s = cfie_batch_create(ctx, (int)ops.size(), ops.data(), nr.data(), &batch);
  auto fail_all = [&](cfie_status st, const std::string& m) {
    for (request_rec* r : live) {
      r->status = st;
      r->err = m;
    }
  };
  if (s != CFIE_OK) {
    fail_all(s, cfie_last_error(ctx));
    cleanup();
    return;
  }
  const size_t len = (size_t)cfie_batch_length(batch);
  std::vector<size_t> off(live.size(), 0);
  for (size_t k = 1; k < live.size(); ++k) off[k] = off[k - 1] + (size_t)ops[k - 1]->n * nr[k - 1];
  try {
    fbuf.reserve(sizeof(double2) * len);
    xbuf.reserve(sizeof(double2) * len);
    CFIE_CHECK_CUDA(cudaMemsetAsync(xbuf.p, 0, sizeof(double2) * len, ctx->stream));
  } catch (const cfie_error& e) {
    fail_all(e.code, e.msg);
    cfie_batch_destroy(batch);
    cleanup();
    return;
  }
  for (size_t k = 0; k < live.size(); ++k) {
    s = cfie_rhs_plane_waves(ops[k], nr[k], live[k]->theta.data(),
                             fbuf.as<double2>() + off[k]);
    if (s != CFIE_OK) {
      fail_all(s, cfie_last_error(ctx));
      cfie_batch_destroy(batch);
      cleanup();
      return;
    }
  }
  const cfie_request& q0 = live[0]->req;
  std::vector<int> its(len > 0 ? (size_t)std::accumulate(nr.begin(), nr.end(), 0) : 0);
  std::vector<double> rel(its.size());
  s = cfie_batch_gmres_solve(batch, fbuf.p, xbuf.p, q0.rtol, q0.restart, q0.maxit, its.data(),
                             rel.data());
  const std::string msg = s == CFIE_OK ? std::string() : std::string(cfie_last_error(ctx));
  size_t col = 0;
  bool copied = true;
  for (size_t k = 0; k < live.size(); ++k) {
    request_rec* r = live[k];
    r->status = CFIE_OK;
    for (int c = 0; c < nr[k]; ++c, ++col) {
      r->iters_max = std::max(r->iters_max, its[col]);
      r->relres_max = std::max(r->relres_max, rel[col]);
      if (!(rel[col] <= r->req.rtol)) r->status = s == CFIE_OK ? CFIE_ENOCONV : s;
    }
    if (s != CFIE_OK && s != CFIE_ENOCONV) r->status = s;
    if (r->status != CFIE_OK) r->err = msg;
    r->x.resize((size_t)ops[k]->n * nr[k]);
    copied = copied && cudaMemcpyAsync(r->x.data(), xbuf.as<double2>() + off[k],
                                       sizeof(double2) * r->x.size(), cudaMemcpyDeviceToHost,
                                       ctx->stream) == cudaSuccess;
  }
  copied = copied && cudaStreamSynchronize(ctx->stream) == cudaSuccess;
  if (!copied)
    for (request_rec* r : live) {
      r->status = CFIE_ECUDA;
      r->err = "copying the solution back failed";
    }
  cfie_batch_destroy(batch);
  cleanup();
}

void worker_main(cfie_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t stream = nullptr;
  cfie_ctx* ctx = nullptr;
  const bool ok = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cfie_ctx_create(S->device, stream, &ctx) == CFIE_OK;
  // a served batch's shapes rarely repeat: its stored contraction takes the
  // default work dealing instead of timing all three for every batch
  if (ok) ctx->tune_batches = false;
  stream_scope ss(stream);     // the slot's staging buffers live on its stream
  dbuf fbuf, xbuf;
  for (;;) {
    request_rec* r = nullptr;
    std::vector<request_rec*> group;
    bool alone = false;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv_work.wait(lock, [&] {
        if (S->stop) return true;
        for (request_rec* q : S->queue)
          if (q->footprint + S->in_use <= S->budget || S->in_use == 0) return true;
        return false;
      });
      if (S->stop) break;
      // first queued request that fits (an oversized one runs alone on an idle GPU)
      for (auto it = S->queue.begin(); it != S->queue.end(); ++it) {
        if ((*it)->footprint + S->in_use <= S->budget || S->in_use == 0) {
          r = *it;
          S->queue.erase(it);
          break;
        }
      }
      group.push_back(r);
      S->in_use += r->footprint;
      // a request for block GMRES runs alone: one Krylov space over its own
      // right-hand sides
      auto blocked = [&](const request_rec* q) {
        return S->block_min > 0 && q->req.nrhs >= S->block_min && q->req.n >= S->block_min_n;
      };
      alone = blocked(r);
      // with batching, further queued requests of the same solver settings
      // and a similar size (n within a factor of two, so that the lockstep
      // iterations of the group end close together) that fit the budget join
      // this slot's batch, in queue order
      for (auto it = S->queue.begin();
           !alone && it != S->queue.end() && (int)group.size() < S->batch_max;) {
        const cfie_request& q = (*it)->req;
        const cfie_request& q0 = r->req;
        if (q.precision == q0.precision && q.rtol == q0.rtol && q.restart == q0.restart &&
            q.maxit == q0.maxit && q.n <= 2 * q0.n && 2 * q.n >= q0.n && !blocked(*it) &&
            (*it)->footprint + S->in_use <= S->budget) {
          S->in_use += (*it)->footprint;
          group.push_back(*it);
          it = S->queue.erase(it);
        } else {
          ++it;
        }
      }
      S->peak_in_use = std::max(S->peak_in_use, S->in_use);
      S->running += (long long)group.size();
      S->peak_running = std::max(S->peak_running, S->running);
      const auto now = clock_type::now();
      for (request_rec* g : group) {
        g->started = true;
        g->t_start = now;
      }
    }
    if (!ok) {
      for (request_rec* g : group) {
        g->status = CFIE_ECUDA;
        g->err = "slot could not create its CUDA stream / context";
      }
    } else {
      // no exception leaves the slot's thread: a host allocation that fails
      // fails the requests in hand
      try {
        if (group.size() == 1)
          run_request(ctx, r, alone, fbuf, xbuf);
        else
          run_batch(ctx, group, fbuf, xbuf);
      } catch (...) {
        for (request_rec* g : group) {
          g->status = CFIE_ENOMEM;
          g->err = "host allocation failed";
        }
      }
    }
    {
      std::lock_guard<std::mutex> lock(S->mu);
      const auto now = clock_type::now();
      for (request_rec* g : group) {
        g->t_done = now;
        g->done = true;
        S->in_use -= g->footprint;
        S->running--;
        S->completed++;
        if (g->status == CFIE_OK) S->solves += g->req.nrhs;
      }
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  fbuf.release();
  xbuf.release();
  if (stream) cudaStreamSynchronize(stream);
  if (ctx) cfie_ctx_destroy(ctx);
  if (stream) cudaStreamDestroy(stream);
}

double seconds(clock_type::duration d) { return std::chrono::duration<double>(d).count(); }

}  // namespace

extern "C" {

cfie_status cfie_server_create(int device, size_t hbm_budget_bytes, int slots, cfie_server** out) {
  if (!out) return CFIE_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) return CFIE_ECUDA;
  if (device < 0 || device >= count || slots < 1 || slots > 64 || hbm_budget_bytes == 0)
    return CFIE_EINVAL;
  cfie_server* S = new (std::nothrow) cfie_server();
  if (!S) return CFIE_ENOMEM;
  S->device = device;
  S->budget = hbm_budget_bytes;
  S->slots = slots;
  try {
    for (int k = 0; k < slots; ++k) S->workers.emplace_back(worker_main, S);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lock(S->mu);
      S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    delete S;
    return CFIE_ENOMEM;
  }
  *out = S;
  return CFIE_OK;
}

cfie_status cfie_server_submit(cfie_server* S, const cfie_request* req, long long* ticket) {
  if (!S || !req || !ticket) return CFIE_EINVAL;
  const cfie_request& q = *req;
  auto bad = [&](const char* m) {
    std::lock_guard<std::mutex> lock(S->mu);
    S->err = m;
    return CFIE_EINVAL;
  };
  if (q.K < 1 || q.K > 64 || !q.a || !q.b) return bad("K must be in [1, 64] with coefficients");
  if (q.n < 8 || q.n % 2 || q.n > (1 << 20)) return bad("n must be even and in [8, 2^20]");
  if (q.nrhs < 1 || q.nrhs > 1024 || !q.theta) return bad("nrhs must be in [1, 1024] with angles");
  if (!(q.omega > 0) || !(q.eta > 0) || !(q.rtol > 0 && q.rtol < 1)) return bad("omega, eta, rtol");
  if (q.bc != CFIE_SOUND_SOFT && q.bc != CFIE_SOUND_HARD) return bad("unknown boundary condition");
  if (q.precision != CFIE_FP64 && q.precision != CFIE_FP32_REFINED &&
      q.precision != CFIE_TENSOR_REFINED)
    return bad("unknown precision");
  if (q.precision == CFIE_TENSOR_REFINED && q.bc != CFIE_SOUND_SOFT)
    return bad("the stored tensor-core form serves the sound-soft operator");
  if (q.restart < 0 || q.restart > 512 || q.maxit < 1) return bad("restart / maxit");
  auto r = std::make_unique<request_rec>();
  r->req = q;
  r->a.assign(q.a, q.a + q.K);
  r->b.assign(q.b, q.b + q.K);
  r->theta.assign(q.theta, q.theta + q.nrhs);
  r->req.a = nullptr;
  r->req.b = nullptr;
  r->req.theta = nullptr;
  r->footprint = footprint_bytes(q);
  r->t_submit = clock_type::now();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    r->ticket = S->next++;
    *ticket = r->ticket;
    S->queue.push_back(r.get());
    S->all.emplace(r->ticket, std::move(r));
  }
  S->cv_work.notify_one();
  return CFIE_OK;
}

cfie_status cfie_server_poll(cfie_server* S, long long ticket, cfie_result* out, void* x_host) {
  if (!S || !out) return CFIE_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) {
    S->err = "unknown ticket";
    return CFIE_EINVAL;
  }
  const request_rec* r = it->second.get();
  std::memset(out, 0, sizeof(*out));
  out->done = r->done ? 1 : 0;
  out->started = r->started ? 1 : 0;
  if (r->done) {
    out->status = r->status;
    out->iters_max = r->iters_max;
    out->relres_max = r->relres_max;
    out->queued_s = seconds(r->t_start - r->t_submit);
    out->service_s = seconds(r->t_done - r->t_start);
    out->latency_s = seconds(r->t_done - r->t_submit);
    if (x_host && !r->x.empty())
      std::memcpy(x_host, r->x.data(), sizeof(double2) * r->x.size());
  }
  return CFIE_OK;
}

cfie_status cfie_server_wait_all(cfie_server* S, double timeout_s) {
  if (!S) return CFIE_EINVAL;
  std::unique_lock<std::mutex> lock(S->mu);
  const bool all_done = S->cv_done.wait_for(
      lock, std::chrono::duration<double>(timeout_s), [&] {
        if (!S->queue.empty() || S->running) return false;
        return true;
      });
  return all_done ? CFIE_OK : CFIE_ETIMEOUT;
}

cfie_status cfie_server_release(cfie_server* S, long long ticket) {
  if (!S) return CFIE_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end() || !it->second->done) return CFIE_EINVAL;
  S->all.erase(it);
  return CFIE_OK;
}

cfie_status cfie_server_stats(cfie_server* S, cfie_server_counters* out) {
  if (!S || !out) return CFIE_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  out->completed = S->completed;
  out->solves = S->solves;
  out->queued = (long long)S->queue.size();
  out->running = S->running;
  out->peak_running = S->peak_running;
  out->budget_bytes = (long long)S->budget;
  out->in_use_bytes = (long long)S->in_use;
  out->peak_in_use_bytes = (long long)S->peak_in_use;
  return CFIE_OK;
}

cfie_status cfie_server_request_error(cfie_server* S, long long ticket, char* buf, size_t len) {
  if (!S || !buf || len == 0) return CFIE_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) {
    S->err = "unknown ticket";
    return CFIE_EINVAL;
  }
  const request_rec* r = it->second.get();
  const std::string& m = r->done ? r->err : std::string();
  const size_t k = std::min(len - 1, m.size());
  std::memcpy(buf, m.data(), k);
  buf[k] = 0;
  return CFIE_OK;
}

const char* cfie_server_last_error(cfie_server* S) { return S ? S->err.c_str() : "null server"; }

cfie_status cfie_server_set_batching(cfie_server* S, int max_requests) {
  if (!S || max_requests < 1 || max_requests > 256) return CFIE_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  S->batch_max = max_requests;
  return CFIE_OK;
}

cfie_status cfie_server_set_block_gmres(cfie_server* S, int min_rhs, int min_n) {
  if (!S || min_rhs < 0 || min_rhs > 1024 || min_n < 0) return CFIE_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  S->block_min = min_rhs;
  S->block_min_n = min_n;
  return CFIE_OK;
}

void cfie_server_destroy(cfie_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
}

}  // extern "C"
