// Eigen-solve server: continuous batching of arb_solve requests on one GPU.
//
// A request (matrix, k, which end, tol, options, optional start block) is queued by
// arb_submit and admitted, in arrival order, as soon as a worker slot is free and its
// HBM footprint (the solver's workspaces, solve_footprint) fits in what the admitted
// requests leave of the budget.  Every slot is a host thread with its own context and
// its own non-blocking CUDA stream, so admitted solves run concurrently on the device;
// a request arriving while others run is admitted the moment a slot and memory free up.
// Workspaces are stream-ordered allocations released after each request, so the device
// memory in use follows the admitted footprints.  Each solve is the same sequence of
// deterministic kernels as a standalone arb_solve, so its result does not depend on what
// else is in flight.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arb_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  arb_ticket ticket = 0;
  arb_mat mat = nullptr;
  int32_t k = 0;
  arb_which which = ARB_SMALLEST;
  double tol = 0.0;
  arb_options opts{};
  std::vector<double> x0;  // empty: drawn from opts.seed
  bool want_vecs = false;
  size_t footprint = 0;
  // results
  std::vector<double> evals, evecs;
  arb_info info{};
  arb_status status = ARB_OK;
  std::string error;
  bool done = false;
  Clock::time_point t_submit, t_start, t_done;
};

}  // namespace

struct arb_server_s {
  int device = 0;
  size_t budget = 0;
  int slots = 0;
  std::vector<std::thread> workers;
  std::vector<arb_ctx> ctxs;
  std::vector<cudaStream_t> streams;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<arb_ticket, std::shared_ptr<Request>> requests;
  size_t in_use = 0;  // footprints of admitted requests
  int busy = 0;
  bool stop = false;
  arb_ticket next_ticket = 1;
  std::string last_error;
};

namespace {

void worker_loop(arb_server srv, int slot) {
  arb_ctx ctx = srv->ctxs[slot];
  cudaSetDevice(srv->device);
  for (;;) {
    std::shared_ptr<Request> req;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      // admission: the oldest queued request, once its footprint fits
      srv->cv_work.wait(lock, [&] {
        return srv->stop || (!srv->queue.empty() && srv->in_use + srv->queue.front()->footprint <= srv->budget);
      });
      if (srv->stop) return;
      req = srv->queue.front();
      srv->queue.pop_front();
      srv->in_use += req->footprint;
      srv->busy++;
      req->t_start = Clock::now();
    }
    const int64_t n = req->mat->n;
    req->evals.assign(req->k, 0.0);
    if (req->want_vecs) req->evecs.assign(static_cast<size_t>(n) * req->k, 0.0);
    arb_status st = arb::solve_on(ctx, req->mat, req->k, req->which, req->tol, &req->opts,
                                  req->x0.empty() ? nullptr : req->x0.data(), 0, req->evals.data(),
                                  req->want_vecs ? req->evecs.data() : nullptr, n, 0, &req->info);
    std::string err = (st == ARB_OK || st == ARB_NOT_CONVERGED) ? std::string() : ctx->last_error;
    // give the memory back before the budget is released
    arb::ws_release_all(ctx);
    cudaStreamSynchronize(ctx->stream);
    {
      std::lock_guard<std::mutex> lock(srv->mu);
      req->status = st;
      req->error = err;
      req->t_done = Clock::now();
      req->done = true;
      srv->in_use -= req->footprint;
      srv->busy--;
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
}

}  // namespace

extern "C" int64_t arb_server_footprint(int64_t n, int64_t nnz, int32_t p, int32_t q, int32_t precision) {
  if (n <= 0 || p <= 0 || q < 0) return -1;
  if (precision != ARB_FP64 && precision != ARB_MIXED && precision != ARB_MIXED_DF) return -1;
  return static_cast<int64_t>(arb::solve_footprint(n, nnz, p, q, precision));
}

extern "C" arb_status arb_server_create(int device, size_t hbm_budget_bytes, int32_t max_slots, arb_server* out) {
  if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) return ARB_INVALID_ARG;
  *out = nullptr;
  auto* srv = new arb_server_s();
  srv->device = device;
  srv->budget = hbm_budget_bytes;
  srv->slots = max_slots;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete srv;
    return ARB_CUDA_ERROR;
  }
  for (int i = 0; i < max_slots; ++i) {
    cudaStream_t s = nullptr;
    arb_ctx ctx = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        arb_ctx_create(&ctx, device, s) != ARB_OK) {
      if (s) cudaStreamDestroy(s);
      for (size_t j = 0; j < srv->ctxs.size(); ++j) {
        arb_ctx_destroy(srv->ctxs[j]);
        cudaStreamDestroy(srv->streams[j]);
      }
      delete srv;
      return ARB_CUDA_ERROR;
    }
    ctx->stream_ordered = true;
    ctx->coop_share = max_slots;
    srv->ctxs.push_back(ctx);
    srv->streams.push_back(s);
  }
  for (int i = 0; i < max_slots; ++i) srv->workers.emplace_back(worker_loop, srv, i);
  *out = srv;
  return ARB_OK;
}

extern "C" arb_status arb_submit(arb_server srv, arb_mat mat, int32_t k, arb_which which, double tol,
                                 const arb_options* opts, const double* x0, int want_evecs, arb_ticket* ticket) {
  if (!srv || !mat || !ticket || k <= 0 || !(tol > 0.0)) return ARB_INVALID_ARG;
  if (mat->device != srv->device) return ARB_INVALID_ARG;
  auto req = std::make_shared<Request>();
  req->mat = mat;
  req->k = k;
  req->which = which;
  req->tol = tol;
  if (opts) {
    req->opts = *opts;
  } else {
    arb_options_default(&req->opts, k);
  }
  const int32_t p = req->opts.p > 0 ? req->opts.p : k + static_cast<int32_t>(std::lround(0.1 * k));
  if (x0) req->x0.assign(x0, x0 + static_cast<size_t>(mat->n) * p);
  req->want_vecs = want_evecs != 0;
  // an adaptive q may grow to q_max (3 by default, and (q+1) p < n): admit for the largest
  int32_t qf = req->opts.q;
  if (req->opts.adapt & ARB_ADAPT_Q) {
    const int64_t fit = (mat->n - 1) / std::max<int32_t>(p, 1) - 1;
    qf = static_cast<int32_t>(std::max<int64_t>(qf, std::min<int64_t>(req->opts.q_max > 0 ? req->opts.q_max : 3, fit)));
  }
  req->footprint = arb::solve_footprint(mat->n, mat->nnz, p, qf, req->opts.precision);
  std::lock_guard<std::mutex> lock(srv->mu);
  if (srv->stop) return ARB_REJECTED;
  if (req->footprint > srv->budget) {
    srv->last_error = "submit: request footprint exceeds the server's HBM budget";
    return ARB_REJECTED;
  }
  req->ticket = srv->next_ticket++;
  req->t_submit = Clock::now();
  srv->requests[req->ticket] = req;
  srv->queue.push_back(req);
  *ticket = req->ticket;
  srv->cv_work.notify_all();
  return ARB_OK;
}

extern "C" arb_status arb_wait(arb_server srv, arb_ticket ticket, int32_t timeout_ms, double* evals, double* evecs,
                               int64_t ldq, arb_info* info, double* latency_s) {
  if (!srv) return ARB_INVALID_ARG;
  std::unique_lock<std::mutex> lock(srv->mu);
  auto it = srv->requests.find(ticket);
  if (it == srv->requests.end()) return ARB_INVALID_ARG;
  std::shared_ptr<Request> req = it->second;
  auto ready = [&] { return req->done; };
  if (timeout_ms < 0) {
    srv->cv_done.wait(lock, ready);
  } else if (!srv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready)) {
    return ARB_TIMEOUT;
  }
  srv->requests.erase(it);
  if (req->status != ARB_OK && req->status != ARB_NOT_CONVERGED) srv->last_error = req->error;
  lock.unlock();
  const int64_t n = req->mat->n;
  if (evecs && !req->want_vecs) return ARB_INVALID_ARG;
  if (evecs && ldq < n) return ARB_INVALID_ARG;
  if (evals) std::copy(req->evals.begin(), req->evals.end(), evals);
  if (evecs)
    for (int32_t c = 0; c < req->k; ++c)
      std::copy(req->evecs.begin() + static_cast<size_t>(c) * n, req->evecs.begin() + static_cast<size_t>(c + 1) * n,
                evecs + static_cast<size_t>(c) * ldq);
  if (info) *info = req->info;
  if (latency_s) *latency_s = std::chrono::duration<double>(req->t_done - req->t_submit).count();
  return req->status;
}

extern "C" arb_status arb_server_destroy(arb_server srv) {
  if (!srv) return ARB_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stop = true;
    for (auto& r : srv->queue) {
      r->status = ARB_REJECTED;
      r->done = true;
    }
    srv->queue.clear();
  }
  srv->cv_work.notify_all();
  srv->cv_done.notify_all();
  for (auto& t : srv->workers) t.join();
  for (size_t i = 0; i < srv->ctxs.size(); ++i) {
    arb_ctx_destroy(srv->ctxs[i]);
    cudaStreamDestroy(srv->streams[i]);
  }
  delete srv;
  return ARB_OK;
}

extern "C" arb_status arb_solve_batched(arb_ctx ctx, int32_t nb, const arb_mat* mats, const int32_t* k,
                                        const arb_which* which, const double* tol, const arb_options* opts,
                                        const double* const* x0, double* const* evals, double* const* evecs,
                                        const int64_t* ldq, arb_info* info, int32_t max_concurrent) {
  if (!ctx || nb < 0 || (nb > 0 && (!mats || !k || !which || !tol || !evals)) || max_concurrent < 1)
    return ARB_INVALID_ARG;
  if (nb == 0) return ARB_OK;
  size_t free_b = 0, total_b = 0;
  if (cudaSetDevice(ctx->device) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess)
    return ARB_CUDA_ERROR;
  arb_server srv = nullptr;
  arb_status st = arb_server_create(ctx->device, static_cast<size_t>(0.9 * free_b), std::min(max_concurrent, nb), &srv);
  if (st != ARB_OK) return st;
  // largest footprints first, so the long solves start early
  std::vector<int32_t> order(nb);
  std::vector<size_t> fp(nb);
  for (int32_t i = 0; i < nb; ++i) {
    order[i] = i;
    arb_options o;
    if (opts) o = opts[i];
    else arb_options_default(&o, k[i]);
    const int32_t p = o.p > 0 ? o.p : k[i] + static_cast<int32_t>(std::lround(0.1 * k[i]));
    fp[i] = arb::solve_footprint(mats[i]->n, mats[i]->nnz, p, o.q, o.precision);
  }
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return fp[a] > fp[b]; });
  std::vector<arb_ticket> tickets(nb, 0);
  arb_status worst = ARB_OK;
  for (int32_t idx : order) {
    st = arb_submit(srv, mats[idx], k[idx], which[idx], tol[idx], opts ? &opts[idx] : nullptr, x0 ? x0[idx] : nullptr,
                    evecs && evecs[idx] ? 1 : 0, &tickets[idx]);
    if (st != ARB_OK) {
      worst = st;
      tickets[idx] = 0;
    }
  }
  for (int32_t i = 0; i < nb; ++i) {
    if (!tickets[i]) continue;
    st = arb_wait(srv, tickets[i], -1, evals[i], evecs ? evecs[i] : nullptr, ldq ? ldq[i] : mats[i]->n,
                  info ? &info[i] : nullptr, nullptr);
    if (st != ARB_OK && (worst == ARB_OK || (worst == ARB_NOT_CONVERGED && st < 0))) worst = st;
  }
  if (worst != ARB_OK && worst != ARB_NOT_CONVERGED) {
    std::lock_guard<std::mutex> lock(srv->mu);
    ctx->last_error = "solve_batched: " + srv->last_error;
  }
  arb_server_destroy(srv);
  return worst;
}
