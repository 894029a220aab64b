// Request server: continuous batching of independent CFIE solves on one GPU.
//
// Requests (an obstacle, a frequency, a boundary condition, a block of
// incidence directions, a target residual) are queued on the host.  A fixed
// set of slots, each a host thread with its own library context and CUDA
// stream, admits queued requests while their estimated device footprint (Krylov
// basis, work vectors, operator tables, near-field band, matvec scratch) fits in
// the HBM budget; a request that arrives while others run is admitted as soon as
// a slot and memory free up, and its kernels overlap on the GPU with the other
// slots' kernels.  Each slot runs the whole path for its request: geometry and
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
  return f;
}

}  // namespace

struct cfie_server {
  int device = 0;
  size_t budget = 0, in_use = 0;
  int slots = 0;
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

void run_request(cfie_ctx* ctx, request_rec* r, dbuf& fbuf, dbuf& xbuf) {
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
                      CFIE_MATRIX_FREE, &op);
  cfie_geom_destroy(geom);
  if (s != CFIE_OK) return fail(s);
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

void worker_main(cfie_server* S) {
  cudaSetDevice(S->device);
  cudaStream_t stream = nullptr;
  cfie_ctx* ctx = nullptr;
  const bool ok = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cfie_ctx_create(S->device, stream, &ctx) == CFIE_OK;
  stream_scope ss(stream);     // the slot's staging buffers live on its stream
  dbuf fbuf, xbuf;
  for (;;) {
    request_rec* r = nullptr;
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
      S->in_use += r->footprint;
      S->peak_in_use = std::max(S->peak_in_use, S->in_use);
      S->running++;
      S->peak_running = std::max(S->peak_running, S->running);
      r->started = true;
      r->t_start = clock_type::now();
    }
    if (ok) {
      run_request(ctx, r, fbuf, xbuf);
    } else {
      r->status = CFIE_ECUDA;
      r->err = "slot could not create its CUDA stream / context";
    }
    {
      std::lock_guard<std::mutex> lock(S->mu);
      r->t_done = clock_type::now();
      r->done = true;
      S->in_use -= r->footprint;
      S->running--;
      S->completed++;
      if (r->status == CFIE_OK) S->solves += r->req.nrhs;
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
  if (q.precision != CFIE_FP64 && q.precision != CFIE_FP32_REFINED)
    return bad("served precisions are CFIE_FP64 and CFIE_FP32_REFINED");
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
