// ccmc_server.cpp -- continuous-batching server of independent simulations.
//
// Requests (one lattice each: shape, seed, density, sweeps, parameters) are
// admitted as memory and slots free up, under a device-memory budget.  Every
// admitted simulation keeps its lattice and random-stream position resident on
// the GPU.  A scheduler thread advances all admitted simulations in slices: one
// slice is one batched sweep launch (small lattices share one persistent
// shared-memory launch, large ones run beside it), each simulation advancing
// by as many sweeps as fit a slice's time budget.  New requests join at the
// next slice boundary while the others keep running; finished ones leave and
// free their memory.  The random streams are keyed by (seed, sweep, site), so a
// request's result is the same whether it ran alone or in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ccmc.h"
#include "ccmc_fault.h"
#include "ccmc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
  uint64_t ticket;
  ccmc_request req;
  double t_submit;
};

struct Running {
  uint64_t ticket;
  ccmc_request req;
  ccmc_lattice *lat;
  int64_t remaining;
  size_t bytes;
  double t_submit, t_start;
};

struct Finished {
  ccmc_result res;
  std::vector<ccmc_obs> series;
};

size_t request_bytes(const ccmc_request &r) {
  const int64_t Cx = r.Lx / 4, Cy = r.Ly / 4, W = (Cx + 15) / 16;
  const int64_t words = 16 * Cy * W * 4;
  const int64_t ring = r.obs_every > 0 ? 64 * std::min<int64_t>(r.nsweeps / r.obs_every + 1, 1 << 16) : 64;
  const int64_t state = r.state_out ? (int64_t)r.Lx * r.Ly : 0;
  return (size_t)(words + ring + state + (128 << 10));  // tables, control, partials
}

// Estimated wall time of one sweep, for sizing slices: a latency floor for
// lattices held by one CTA, plus a throughput term.
double sweep_us(const ccmc_request &r) {
  return 12.0 + 5e-6 * (double)r.Lx * (double)r.Ly;
}

}  // namespace

struct ccmc_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;
  std::vector<Running> active;
  std::unordered_map<uint64_t, Finished> done;
  std::unordered_map<uint64_t, int> state;  // 1 queued, 2 running
  uint64_t next_ticket = 1;
  size_t budget = 0, in_use = 0;
  int max_active = 0;
  double slice_ms = 20.0;
  bool stopping = false;
  int device = 0;
  ccmc_batch *batch = nullptr;
  cudaStream_t stream = nullptr;
  std::thread worker;
  Clock::time_point t0;
  ccmc_server_stats st{};

  double now() const {
    return std::chrono::duration<double>(Clock::now() - t0).count();
  }
  void run();
  void finish(Running &r, int status);
};

void ccmc_server::finish(Running &r, int status) {
  Finished f{};
  f.res.status = status;
  f.res.submit_s = r.t_submit;
  f.res.start_s = r.t_start;
  if (status == CCMC_OK) {
    ccmc_obs o{};
    int rc = ccmc_observables(r.lat, &o);
    if (rc == CCMC_OK && r.req.state_out) rc = ccmc_get_state(r.lat, r.req.state_out);
    if (rc == CCMC_OK && r.req.obs_every > 0) {
      const int64_t cap = std::min<int64_t>(r.req.nsweeps / r.req.obs_every + 1, 1 << 16);
      f.series.resize((size_t)cap);
      int64_t n = 0;
      rc = ccmc_obs_series(r.lat, f.series.data(), cap, &n);
      f.series.resize((size_t)n);
    }
    f.res.status = rc;
    f.res.final_obs = o;
    f.res.site_updates = (int64_t)r.req.Lx * r.req.Ly * r.req.nsweeps;
  }
  ccmc_lattice_destroy(r.lat);
  f.res.done_s = now();
  std::lock_guard<std::mutex> lock(mu);
  in_use -= r.bytes;
  state.erase(r.ticket);
  if (f.res.status == CCMC_OK) {
    ++st.completed;
    st.site_updates += f.res.site_updates;
  } else {
    ++st.failed;
  }
  done[r.ticket] = std::move(f);
  cv_done.notify_all();
}

void ccmc_server::run() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<Pending> admit;
    {
      std::unique_lock<std::mutex> lock(mu);
      cv_work.wait(lock, [&] { return stopping || !queue.empty() || !active.empty(); });
      if (stopping && queue.empty() && active.empty()) break;
      // admission: first come, first served, while slots and budget allow
      size_t planned = in_use;
      while (!queue.empty() && (int)(active.size() + admit.size()) < max_active) {
        Pending &p = queue.front();
        const size_t bytes = request_bytes(p.req);
        if (bytes > budget || ccmc::fault_injected("admit")) {  // can never fit
          Finished f{};
          f.res.status = CCMC_E_BUDGET;
          f.res.submit_s = p.t_submit;
          f.res.done_s = now();
          state.erase(p.ticket);
          done[p.ticket] = f;
          ++st.rejected;
          queue.pop_front();
          cv_done.notify_all();
          continue;
        }
        if (planned + bytes > budget) break;
        planned += bytes;
        admit.push_back(p);
        state[p.ticket] = 2;
        queue.pop_front();
      }
      in_use = planned;
    }
    for (Pending &p : admit) {
      Running r{p.ticket, p.req, nullptr, p.req.nsweeps, request_bytes(p.req), p.t_submit, now()};
      int rc = ccmc_lattice_create(p.req.Lx, p.req.Ly, nullptr,
                                   p.req.obs_every > 0 ? std::min<int64_t>(p.req.nsweeps / p.req.obs_every + 1, 1 << 16) : 1,
                                   &r.lat);
      if (rc == CCMC_OK) rc = ccmc_init_constrained(r.lat, p.req.seed, p.req.n, p.req.charged_frac);
      if (rc != CCMC_OK) {
        if (!r.lat) {
          std::lock_guard<std::mutex> lock(mu);
          in_use -= r.bytes;
          state.erase(r.ticket);
          Finished f{};
          f.res.status = rc;
          f.res.submit_s = r.t_submit;
          f.res.done_s = now();
          done[r.ticket] = f;
          ++st.failed;
          cv_done.notify_all();
        } else {
          finish(r, rc);
        }
        continue;
      }
      active.push_back(r);
    }
    if (active.empty()) continue;
    // one slice: every active simulation advances by what fits the time budget
    const int n = (int)active.size();
    std::vector<ccmc_lattice *> lats(n);
    std::vector<int64_t> sw(n);
    std::vector<double> beta(n), Delta(n), V(n), J(n);
    std::vector<int> every(n);
    for (int i = 0; i < n; ++i) {
      Running &r = active[i];
      int64_t q = (int64_t)(slice_ms * 1e3 / sweep_us(r.req));
      if (q < 1) q = 1;
      if (r.req.obs_every > 1) q = std::max<int64_t>(r.req.obs_every, q / r.req.obs_every * r.req.obs_every);
      lats[i] = r.lat;
      sw[i] = std::min(r.remaining, q);
      beta[i] = r.req.beta;
      Delta[i] = r.req.Delta;
      V[i] = r.req.V;
      J[i] = r.req.J;
      every[i] = r.req.obs_every;
    }
    int rc = ccmc::batch_run(batch, lats, sw.data(), beta.data(), Delta.data(), V.data(), J.data(),
                             every.data(), false);
    if (rc == CCMC_OK && cudaStreamSynchronize(stream) != cudaSuccess) rc = CCMC_E_CUDA;
    for (int i = 0; i < n && rc == CCMC_OK; ++i) rc = ccmc_sync(lats[i]);
    {
      std::lock_guard<std::mutex> lock(mu);
      ++st.slices;
    }
    std::vector<Running> still;
    for (int i = 0; i < n; ++i) {
      Running &r = active[i];
      r.remaining -= sw[i];
      if (rc != CCMC_OK)
        finish(r, rc);
      else if (r.remaining == 0)
        finish(r, CCMC_OK);
      else
        still.push_back(r);
    }
    active.swap(still);
  }
}

extern "C" {

int ccmc_server_start(size_t hbm_budget_bytes, int max_active, double slice_ms,
                      ccmc_server **out) {
  if (!out || hbm_budget_bytes == 0 || max_active < 1 || max_active > 4096 || !(slice_ms > 0.0))
    return CCMC_E_INVAL;
  *out = nullptr;
  ccmc_server *s = new (std::nothrow) ccmc_server();
  if (!s) return CCMC_E_NOMEM;
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  s->slice_ms = slice_ms;
  s->t0 = Clock::now();
  cudaGetDevice(&s->device);
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    return CCMC_E_CUDA;
  }
  int rc = ccmc::batch_new(max_active, s->stream, &s->batch);
  if (rc != CCMC_OK) {
    cudaStreamDestroy(s->stream);
    delete s;
    return rc;
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return CCMC_OK;
}

int ccmc_server_submit(ccmc_server *s, const ccmc_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return CCMC_E_INVAL;
  if (req->Lx < 4 || req->Ly < 4 || (req->Lx & 3) || (req->Ly & 3) ||
      (int64_t)req->Lx * req->Ly > ((int64_t)1 << 30) || req->nsweeps < 0 ||
      !(req->beta >= 0.0) || req->obs_every < 0)
    return CCMC_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stopping) return CCMC_E_STATE;
  const uint64_t t = s->next_ticket++;
  s->queue.push_back(Pending{t, *req, s->now()});
  s->state[t] = 1;
  ++s->st.submitted;
  *ticket = t;
  s->cv_work.notify_one();
  return CCMC_OK;
}

int ccmc_server_poll(ccmc_server *s, uint64_t ticket, ccmc_result *out) {
  if (!s || !out) return CCMC_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->done.find(ticket);
  if (it != s->done.end()) {
    *out = it->second.res;
    return CCMC_OK;
  }
  return s->state.count(ticket) ? CCMC_PENDING : CCMC_E_NOTFOUND;
}

int ccmc_server_wait(ccmc_server *s, uint64_t ticket, ccmc_result *out, double timeout_s) {
  if (!s || !out) return CCMC_E_INVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  if (!s->done.count(ticket) && !s->state.count(ticket)) return CCMC_E_NOTFOUND;
  const bool ok = s->cv_done.wait_for(
      lock, std::chrono::duration<double>(timeout_s < 0 ? 0 : timeout_s),
      [&] { return s->done.count(ticket) > 0; });
  if (!ok) return CCMC_E_TIMEOUT;
  *out = s->done[ticket].res;
  return CCMC_OK;
}

int ccmc_server_series(ccmc_server *s, uint64_t ticket, ccmc_obs *out, int64_t cap,
                       int64_t *n_written) {
  if (!s || !n_written || cap < 0 || (cap > 0 && !out)) return CCMC_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) return s->state.count(ticket) ? CCMC_PENDING : CCMC_E_NOTFOUND;
  const auto &v = it->second.series;
  const int64_t n = std::min<int64_t>(cap, (int64_t)v.size());
  if (n > 0) std::memcpy(out, v.data(), sizeof(ccmc_obs) * (size_t)n);
  *n_written = n;
  return CCMC_OK;
}

int ccmc_server_release(ccmc_server *s, uint64_t ticket) {
  if (!s) return CCMC_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  return s->done.erase(ticket) ? CCMC_OK : CCMC_E_NOTFOUND;
}

int ccmc_server_stats_get(ccmc_server *s, ccmc_server_stats *out) {
  if (!s || !out) return CCMC_E_INVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->st;
  out->queued = (int64_t)s->queue.size();
  out->active = (int64_t)(s->state.size() - s->queue.size());
  out->bytes_in_use = (int64_t)s->in_use;
  return CCMC_OK;
}

int ccmc_server_stop(ccmc_server *s) {
  if (!s) return CCMC_E_INVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  ccmc_batch_destroy(s->batch);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return CCMC_OK;
}

}  // extern "C"
