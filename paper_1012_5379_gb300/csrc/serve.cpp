// Serving loop: continuous batching of Helmholtz solves on one GPU.
//
// Requests (grid, k, theta_beta, host source, host solution buffer, tolerance) are
// queued by any host thread.  One worker thread owns the device.  2D and 3D problems
// are iterated by two runners on two streams that advance independently: whenever a
// runner's stream has finished its outer iteration, the worker reads the states,
// retires converged problems (their solutions are copied back asynchronously), admits
// queued requests (in arrival order up to a bounded overtaking, see admit()) while the
// device-memory budget allows, and
// launches the next iteration of every problem of that dimension together (one launch
// per V-cycle level and per outer kernel for all of them).  Each request runs in a
// problem slot: a handle re-targeted to the request's k and theta_beta.  Idle slots
// of the same shape are reused, so steady-state admission allocates no device memory.
// Each problem's reductions are per problem in a fixed order, so a result does not
// depend on which other requests shared its launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "../../include/helm.h"
#include "engine.h"

namespace helm {

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct ServeRequest {
  long long ticket = 0;
  int dim = 2, n = 0;
  double k = 0, theta_beta = 0, tol = 1e-6;
  const double* b = nullptr;  // borrowed until completion
  double* x = nullptr;        // borrowed until completion
  helm_info info{};
  int status = HELM_EAGAIN;
  double t_submit = 0, t_done = 0;
};

struct Draining {        // a retired request whose solution is still being copied back
  ServeRequest* r;
  int status;
  cudaEvent_t ev;
};

}  // namespace

struct Server {
  helm_serve_opts opts{};
  int device = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServeRequest*> queue;
  std::unordered_map<long long, ServeRequest*> reqs;
  bool stopping = false;
  long long next_ticket = 1;
  helm_serve_counters stats{};
  std::string fatal;

  // worker-owned
  std::map<std::pair<int, int>, std::vector<Handle*>> pool;  // idle slots by (dim, n)
  std::vector<Handle*> all_handles;
  std::unordered_map<Handle*, ServeRequest*> owner;
  size_t bytes_in_use = 0;
  BatchRunner* run[2] = {nullptr, nullptr};
  cudaStream_t st[2] = {nullptr, nullptr};
  cudaStream_t setup_st = nullptr;
  bool inflight[2] = {false, false};
  std::vector<Draining> draining;
  std::vector<cudaEvent_t> free_events;

  helm_opts handle_opts() const {
    helm_opts o{};
    o.nu1 = opts.nu1;
    o.nu2 = opts.nu2;
    o.s = opts.s;
    o.precond_prec = opts.precond_prec;
    o.restart = opts.restart;
    o.maxit = opts.maxit;
    return o;
  }

  static size_t dense_bytes(int dim, int n) {
    return (dim == 3 ? (size_t)n * n * n : (size_t)n * n) * sizeof(double2);
  }

  void finish_request(ServeRequest* r, int status) {
    std::lock_guard<std::mutex> lk(mu);
    r->status = status;
    r->t_done = now_s();
    stats.completed += 1;
    if (status == HELM_ENOMEM || status == HELM_EINVAL) stats.rejected += 1;
    cv_done.notify_all();
  }

  // Free idle slots until `need` more bytes fit in the budget.
  void evict_idle(size_t need) {
    for (auto& kv : pool) {
      while (!kv.second.empty() && bytes_in_use + need > opts.budget_bytes) {
        Handle* h = kv.second.back();
        kv.second.pop_back();
        bytes_in_use -= h->bytes;
        all_handles.erase(std::find(all_handles.begin(), all_handles.end(), h));
        delete h;
      }
    }
  }

  // Admit queued requests while slots and memory allow.  Arrival order is kept, except
  // that a request whose shape has an idle slot, or that fits the free budget, may
  // pass a head that would need slots evicted; the head is passed at most
  // MAX_OVERTAKE times in a row (then idle slots are evicted for it), and only the
  // first WINDOW queued requests are considered.
  static constexpr int WINDOW = 64, MAX_OVERTAKE = 32;
  int head_overtaken = 0;
  size_t estimate(const ServeRequest* r) const {
    return estimate_handle_bytes(r->dim, r->n, opts.precond_prec, opts.s, opts.restart, opts.maxit, 3);
  }
  bool has_idle(const ServeRequest* r) const {
    auto it = pool.find(std::make_pair(r->dim, r->n));
    return it != pool.end() && !it->second.empty();
  }

  int admit() {
    for (;;) {
      ServeRequest* r = nullptr;
      bool evict = false;
      {
        std::lock_guard<std::mutex> lk(mu);
        if (queue.empty()) return HELM_OK;
        const int active = runner_size(run[0]) + runner_size(run[1]);
        if (opts.max_active > 0 && active >= opts.max_active) return HELM_OK;
        const size_t nscan = std::min<size_t>(queue.size(), WINDOW);
        size_t pick = nscan;
        for (size_t i = 0; i < nscan; ++i) {
          const ServeRequest* q = queue[i];
          const size_t est = estimate(q);
          if (has_idle(q) || est > opts.budget_bytes || bytes_in_use + est <= opts.budget_bytes) { pick = i; break; }
          if (i == 0 && (head_overtaken >= MAX_OVERTAKE || active == 0)) { pick = 0; evict = true; break; }
        }
        if (pick == nscan) return HELM_OK;  // wait for completions
        r = queue[pick];
        queue.erase(queue.begin() + pick);
        head_overtaken = pick > 0 ? head_overtaken + 1 : 0;
      }
      const int di = r->dim == 3 ? 1 : 0;
      const auto key = std::make_pair(r->dim, r->n);
      Handle* h = nullptr;
      auto it = pool.find(key);
      if (it != pool.end() && !it->second.empty()) {
        h = it->second.back();
        it->second.pop_back();
        stats.handles_reused += 1;
        TRY(retarget_handle(h, r->k, r->theta_beta, st[di]));
      } else {
        const size_t est = estimate(r);
        if (est > opts.budget_bytes) {
          set_error("request needs more device memory than the serving budget");
          finish_request(r, HELM_ENOMEM);
          continue;
        }
        if (evict && bytes_in_use + est > opts.budget_bytes) evict_idle(est);
        if (bytes_in_use + est > opts.budget_bytes) {  // still no room: back to the head of the queue
          std::lock_guard<std::mutex> lk(mu);
          queue.push_front(r);
          return HELM_OK;
        }
        helm_grid g{};
        g.dim = r->dim;
        g.n = r->n;
        g.ecs_frac = opts.ecs_frac;
        g.theta_gamma = opts.theta_gamma;
        const helm_opts o = handle_opts();
        // set up on a private stream: its synchronisation does not wait for the
        // iteration in flight on the runner's stream
        int rc = setup_handle(&g, nullptr, r->k, r->theta_beta, &o, setup_st, &h);
        if (rc != HELM_OK) {
          finish_request(r, rc);
          continue;
        }
        bytes_in_use += h->bytes;
        all_handles.push_back(h);
        stats.handles_created += 1;
      }
      owner[h] = r;
      // the source goes through the slot's dense staging vector (w, unused until the
      // problem's first outer iteration); stream order protects it
      CUDA_TRY(cudaMemcpyAsync(h->w, r->b, dense_bytes(r->dim, r->n), cudaMemcpyHostToDevice, st[di]));
      TRY(runner_add(run[di], h, (const double2*)h->w, r->tol, st[di]));
    }
  }

  cudaEvent_t take_event() {
    if (free_events.empty()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
      return e;
    }
    cudaEvent_t e = free_events.back();
    free_events.pop_back();
    return e;
  }

  // Converged (or failed) problems: enqueue the solution's conversion and copy to the
  // caller's buffer, and return the slot to the pool (its next use is ordered after
  // the copy on the same stream).
  int retire(int di, const std::vector<std::pair<Handle*, OuterState>>& done) {
    for (const auto& d : done) {
      Handle* h = d.first;
      ServeRequest* r = owner[h];
      owner.erase(h);
      const int status = runner_finish(h, d.second, h->w, st[di], &r->info);
      if (status == HELM_ECUDA) return status;
      CUDA_TRY(cudaMemcpyAsync(r->x, h->w, dense_bytes(h->dim, h->n), cudaMemcpyDeviceToHost, st[di]));
      cudaEvent_t ev = take_event();
      if (!ev) { set_error("cudaEventCreate failed"); return HELM_ECUDA; }
      CUDA_TRY(cudaEventRecord(ev, st[di]));
      draining.push_back({r, status, ev});
      pool[std::make_pair(h->dim, h->n)].push_back(h);
    }
    return HELM_OK;
  }

  // Requests whose solution copy has landed are complete.
  int drain() {
    for (size_t i = 0; i < draining.size();) {
      const cudaError_t q = cudaEventQuery(draining[i].ev);
      if (q == cudaErrorNotReady) { ++i; continue; }
      CUDA_TRY(q);
      free_events.push_back(draining[i].ev);
      finish_request(draining[i].r, draining[i].status);
      draining[i] = draining.back();
      draining.pop_back();
    }
    return HELM_OK;
  }

  void fail_all(int rc) {
    std::lock_guard<std::mutex> lk(mu);
    fatal = helm_last_error();
    for (auto& kv : reqs)
      if (kv.second->status == HELM_EAGAIN) {
        kv.second->status = rc;
        kv.second->t_done = now_s();
      }
    queue.clear();
    cv_done.notify_all();
  }

  // One pass of the worker: collect every runner whose iteration has finished, admit,
  // launch every idle runner's next iteration.
  int step() {
    for (int d = 0; d < 2; ++d) {
      if (!inflight[d]) continue;
      const cudaError_t q = cudaStreamQuery(st[d]);
      if (q == cudaErrorNotReady) continue;
      CUDA_TRY(q);
      std::vector<std::pair<Handle*, OuterState>> done;
      TRY(runner_collect(run[d], st[d], &done));
      inflight[d] = false;
      TRY(retire(d, done));
    }
    TRY(drain());
    TRY(admit());
    for (int d = 0; d < 2; ++d) {
      if (inflight[d] || runner_size(run[d]) == 0) continue;
      TRY(runner_iterate(run[d], st[d]));
      inflight[d] = true;
    }
    const int active = runner_size(run[0]) + runner_size(run[1]);
    std::lock_guard<std::mutex> lk(mu);
    stats.active = active;
    stats.queued = (int)queue.size();
    stats.peak_active = std::max(stats.peak_active, active);
    stats.bytes_in_use = bytes_in_use;
    stats.peak_bytes = std::max(stats.peak_bytes, bytes_in_use);
    return HELM_OK;
  }

  void loop() {
    cudaSetDevice(device);
    int rc = HELM_OK;
    for (int d = 0; d < 2 && rc == HELM_OK; ++d) {
      if (cudaStreamCreateWithFlags(&st[d], cudaStreamNonBlocking) != cudaSuccess) {
        set_error("cudaStreamCreate failed");
        rc = HELM_ECUDA;
      }
      run[d] = runner_create(opts.precond_prec);
    }
    if (rc == HELM_OK && cudaStreamCreateWithFlags(&setup_st, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("cudaStreamCreate failed");
      rc = HELM_ECUDA;
    }
    while (rc == HELM_OK) {
      rc = step();
      if (rc != HELM_OK) break;
      if (inflight[0] || inflight[1] || !draining.empty()) {
        std::this_thread::yield();
        continue;
      }
      std::unique_lock<std::mutex> lk(mu);
      if (stopping && queue.empty()) break;
      if (queue.empty()) cv_work.wait_for(lk, std::chrono::milliseconds(2));
    }
    if (rc != HELM_OK) fail_all(rc);
    for (int d = 0; d < 2; ++d)
      if (st[d]) cudaStreamSynchronize(st[d]);
    for (int d = 0; d < 2; ++d) {
      if (run[d]) runner_destroy(run[d]);
      run[d] = nullptr;
    }
    for (Handle* h : all_handles) delete h;
    all_handles.clear();
    pool.clear();
    for (auto& dr : draining) cudaEventDestroy(dr.ev);
    for (cudaEvent_t e : free_events) cudaEventDestroy(e);
    for (int d = 0; d < 2; ++d)
      if (st[d]) cudaStreamDestroy(st[d]);
    if (setup_st) cudaStreamDestroy(setup_st);
  }
};

int serve_start(const helm_serve_opts* opts, Server** out) {
  if (!out) { set_error("out must not be NULL"); return HELM_EINVAL; }
  helm_serve_opts o{};
  if (opts) o = *opts;
  if (o.budget_bytes == 0) o.budget_bytes = (size_t)120 << 30;
  if (o.precond_prec == 0) o.precond_prec = HELM_C64;
  if (o.restart <= 0) o.restart = 40;
  if (o.maxit <= 0) o.maxit = 400;
  if (o.nu1 <= 0 && o.nu2 <= 0) { o.nu1 = 1; o.nu2 = 1; }
  if (o.s <= 0) o.s = 3;
  if (o.ecs_frac <= 0) o.ecs_frac = 0.125;
  if (o.theta_gamma <= 0) o.theta_gamma = 0.5;
  if (o.precond_prec != HELM_C64 && o.precond_prec != HELM_C128) {
    set_error("precond_prec must be HELM_C64 or HELM_C128");
    return HELM_EINVAL;
  }
  if (o.nu1 < 0 || o.nu2 < 0 || o.nu1 > 8 || o.nu2 > 8 || o.s > SMAX || o.ecs_frac >= 0.5 ||
      !(o.theta_gamma < M_PI / 2) || o.max_active < 0) {
    set_error("invalid serving options (nu1, nu2, s, ecs_frac, theta_gamma or max_active)");
    return HELM_EINVAL;
  }
  Server* s = new Server();
  s->opts = o;
  cudaGetDevice(&s->device);
  s->worker = std::thread([s]() { s->loop(); });
  *out = s;
  return HELM_OK;
}

int serve_submit(Server* s, int dim, int n, double k, double theta_beta, const double* b_host, double* x_host,
                 double tol, long long* ticket) {
  if (!s || !b_host || !x_host || !ticket) { set_error("NULL argument"); return HELM_EINVAL; }
  if ((dim != 2 && dim != 3) || n < 3 || !(tol > 0) || !(theta_beta >= 0 && theta_beta < M_PI / 2) ||
      !std::isfinite(k)) {
    set_error("invalid request (dim, n, tol, theta_beta or k)");
    return HELM_EINVAL;
  }
  if (((n + 1) & n) != 0) { set_error("served grids need n + 1 a power of two"); return HELM_EINVAL; }
  ServeRequest* r = new ServeRequest();
  r->dim = dim;
  r->n = n;
  r->k = k;
  r->theta_beta = theta_beta;
  r->tol = tol;
  r->b = b_host;
  r->x = x_host;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) {
    delete r;
    set_error("server is stopping");
    return HELM_EINVAL;
  }
  r->ticket = s->next_ticket++;
  r->t_submit = now_s();
  s->reqs[r->ticket] = r;
  s->queue.push_back(r);
  s->stats.submitted += 1;
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return HELM_OK;
}

static int take_result(Server* s, ServeRequest* r, helm_info* info, double* latency) {
  if (info) *info = r->info;
  if (latency) *latency = r->t_done - r->t_submit;
  const int status = r->status;
  s->reqs.erase(r->ticket);
  delete r;
  return status;
}

int serve_poll(Server* s, long long ticket, helm_info* info, double* latency) {
  if (!s) { set_error("NULL server"); return HELM_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) { set_error("unknown ticket"); return HELM_EINVAL; }
  if (it->second->status == HELM_EAGAIN) return HELM_EAGAIN;
  return take_result(s, it->second, info, latency);
}

int serve_wait(Server* s, long long ticket, double timeout_s, helm_info* info, double* latency) {
  if (!s) { set_error("NULL server"); return HELM_EINVAL; }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) { set_error("unknown ticket"); return HELM_EINVAL; }
  ServeRequest* r = it->second;
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(std::max(0.0, timeout_s)));
  while (r->status == HELM_EAGAIN) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && r->status == HELM_EAGAIN) {
      set_error("wait timed out");
      return HELM_ETIMEOUT;
    }
  }
  return take_result(s, r, info, latency);
}

int serve_stats(Server* s, helm_serve_counters* out) {
  if (!s || !out) { set_error("NULL argument"); return HELM_EINVAL; }
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  build_stats(&out->group_builds, &out->graph_builds, &out->build_s);
  return HELM_OK;
}

int serve_stop(Server* s) {
  if (!s) return HELM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    s->cv_work.notify_one();
  }
  if (s->worker.joinable()) s->worker.join();
  const bool failed = !s->fatal.empty();
  if (failed) set_error(s->fatal);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return failed ? HELM_ECUDA : HELM_OK;
}

}  // namespace helm
