// ccmc_server.cpp -- continuous-batching server of independent simulations.
//
// Requests (one lattice each: shape, seed, density, sweeps, parameters) are
// admitted as memory and slots free up, under a device-memory budget.  Every
// admitted simulation keeps its lattice and random-stream position resident on
// the GPU.  A scheduler thread advances all admitted simulations in slices: one
// slice is one batched sweep launch (small lattices share one persistent
// shared-memory launch, large ones run beside it on their own streams), each
// simulation advancing by as many sweeps as fit a slice's time budget.
//
// The GPU never waits for the host: the scheduler keeps two slices queued, so
// slice k + 1 is on the device before slice k ends; a request is created and
// initialised by work queued on its own stream (lattice memory comes from a
// stream-ordered pool, so no call synchronises the device); a request that
// finishes in a slice has its results (latest exact recount, status, the
// observable ring and the final state when asked) copied into pinned host
// buffers by work queued behind its last sweep, and the scheduler collects
// them once that work's event has fired, then retires the lattice.  The
// random streams are keyed by (seed, sweep, site), so a request's result is
// the same whether it ran alone or in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ccmc.h"
#include "ccmc_fault.h"
#include "ccmc_internal.h"
#include "ccmc_trace.h"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kSlicesInFlight = 2;

struct Pending {
  uint64_t ticket;
  ccmc_request req;
  double t_submit;
};

struct Running {
  uint64_t ticket;
  ccmc_request req;
  ccmc_lattice *lat;
  int64_t remaining;  // sweeps not yet queued
  size_t bytes;
  double t_submit, t_start;
};

// A request whose last sweep is queued: its results are on their way to
// pinned host buffers; `ready` fires when they have landed.
struct Retiring {
  Running r;
  cudaEvent_t ready;
  int64_t *pin;  // rec (8), status, count
  int64_t *ring;
  uint8_t *state;
  size_t ring_bytes, state_bytes;
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

int64_t ring_records(const ccmc_request &r) {
  return r.obs_every > 0 ? std::min<int64_t>(r.nsweeps / r.obs_every + 1, 1 << 16) : 1;
}

// Estimated wall time of one sweep, for sizing slices: a latency floor for
// lattices held by one CTA, plus a throughput term.
double sweep_us(const ccmc_request &r) {
  return 12.0 + 5e-6 * (double)r.Lx * (double)r.Ly;
}

// Pinned host buffers, cached by power-of-two size (allocating pinned memory
// is slow and may synchronise; retired buffers are reused).
class PinnedCache {
 public:
  void *get(size_t bytes) {
    const size_t c = size_class(bytes);
    auto &v = free_[c];
    if (!v.empty()) {
      void *p = v.back();
      v.pop_back();
      return p;
    }
    void *p = nullptr;
    if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void *p, size_t bytes) {
    if (p) free_[size_class(bytes)].push_back(p);
  }
  ~PinnedCache() {
    for (auto &kv : free_)
      for (void *p : kv.second) cudaFreeHost(p);
  }

 private:
  static size_t size_class(size_t b) {
    size_t c = 256;
    while (c < b) c <<= 1;
    return c;
  }
  std::map<size_t, std::vector<void *>> free_;
};

}  // namespace

struct ccmc_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;
  std::unordered_map<uint64_t, Finished> done;
  std::unordered_map<uint64_t, int> state;  // 1 queued, 2 running
  uint64_t next_ticket = 1;
  size_t budget = 0, in_use = 0;
  int max_active = 0;
  int active_count = 0;  // admitted and not yet finished (scheduler's count)
  double slice_ms = 20.0;
  bool stopping = false;
  int device = 0;
  ccmc_batch *batch = nullptr;
  cudaStream_t stream = nullptr;  // the batch's stream
  cudaStream_t marker = nullptr;  // waits for a slice's work; its events end slices
  std::thread worker;
  Clock::time_point t0;
  ccmc_server_stats st{};

  // scheduler-thread state
  std::vector<Running> active;
  std::vector<Retiring> retiring;
  std::deque<cudaEvent_t> slices;   // end events of the queued slices
  std::vector<cudaEvent_t> events;  // idle events for reuse
  PinnedCache pinned;

  double now() const {
    return std::chrono::duration<double>(Clock::now() - t0).count();
  }
  cudaEvent_t event() {
    if (!events.empty()) {
      cudaEvent_t e = events.back();
      events.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
  void run();
  void publish(uint64_t ticket, Finished &&f, size_t bytes);
  void fail(Running &r, int status);
  void retire(Running &r);
  bool collect(Retiring &x);
};

// Hand a result to the waiting clients and release the request's budget.
void ccmc_server::publish(uint64_t ticket, Finished &&f, size_t bytes) {
  f.res.done_s = now();
  std::lock_guard<std::mutex> lock(mu);
  in_use -= bytes;
  state.erase(ticket);
  --active_count;
  if (f.res.status == CCMC_OK) {
    ++st.completed;
    st.site_updates += f.res.site_updates;
  } else {
    ++st.failed;
  }
  done[ticket] = std::move(f);
  cv_done.notify_all();
}

void ccmc_server::fail(Running &r, int status) {
  Finished f{};
  f.res.status = status;
  f.res.submit_s = r.t_submit;
  f.res.start_s = r.t_start;
  if (r.lat) ccmc_lattice_destroy(r.lat);
  r.lat = nullptr;
  publish(r.ticket, std::move(f), r.bytes);
}

// Queue the copies of a finished request's results behind its last sweep.
void ccmc_server::retire(Running &r) {
  Retiring x{r, event(), nullptr, nullptr, nullptr, 0, 0};
  x.pin = static_cast<int64_t *>(pinned.get(sizeof(int64_t) * 10));
  if (r.req.obs_every > 0) {
    x.ring_bytes = sizeof(int64_t) * 8 * (size_t)ccmc::ring_capacity(r.lat);
    x.ring = static_cast<int64_t *>(pinned.get(x.ring_bytes));
  }
  if (r.req.state_out) {
    x.state_bytes = (size_t)r.req.Lx * r.req.Ly;
    x.state = static_cast<uint8_t *>(pinned.get(x.state_bytes));
  }
  int rc = CCMC_OK;
  if (!x.ready || !x.pin || (r.req.obs_every > 0 && !x.ring) || (r.req.state_out && !x.state))
    rc = CCMC_E_NOMEM;
  if (rc == CCMC_OK)
    rc = ccmc::export_async(r.lat, x.pin, x.pin + 8, x.pin + 9, x.ring, x.state, x.ready);
  if (rc != CCMC_OK) {
    pinned.put(x.pin, sizeof(int64_t) * 10);
    pinned.put(x.ring, x.ring_bytes);
    pinned.put(x.state, x.state_bytes);
    if (x.ready) events.push_back(x.ready);
    fail(r, rc);
    return;
  }
  retiring.push_back(x);
}

// A retiring request whose results have landed: publish them.  False while
// they are still on their way.
bool ccmc_server::collect(Retiring &x) {
  const cudaError_t q = cudaEventQuery(x.ready);
  if (q == cudaErrorNotReady) return false;
  Running &r = x.r;
  Finished f{};
  f.res.submit_s = r.t_submit;
  f.res.start_s = r.t_start;
  f.res.status = q == cudaSuccess ? (x.pin[8] == 0 ? CCMC_OK : CCMC_E_TIMEOUT) : CCMC_E_CUDA;
  if (q != cudaSuccess) cudaGetLastError();
  if (f.res.status == CCMC_OK) {
    ccmc::obs_of_record(r.lat, x.pin, &f.res.final_obs);
    f.res.site_updates = (int64_t)r.req.Lx * r.req.Ly * r.req.nsweeps;
    if (x.ring) {
      f.series.resize((size_t)ring_records(r.req));
      f.series.resize((size_t)ccmc::series_of_ring(r.lat, x.ring, x.pin[9], f.series.data(),
                                                    (int64_t)f.series.size()));
    }
    if (x.state) std::memcpy(r.req.state_out, x.state, x.state_bytes);
  }
  pinned.put(x.pin, sizeof(int64_t) * 10);
  pinned.put(x.ring, x.ring_bytes);
  pinned.put(x.state, x.state_bytes);
  events.push_back(x.ready);
  ccmc_lattice_destroy(r.lat);  // its stream's work is done: no wait
  r.lat = nullptr;
  publish(r.ticket, std::move(f), r.bytes);
  return true;
}

void ccmc_server::run() {
  cudaSetDevice(device);
  for (;;) {
    // (1) admission: first come, first served, while slots and budget allow
    std::vector<Pending> admit;
    {
      std::unique_lock<std::mutex> lock(mu);
      auto has_work = [&] {
        return stopping || !queue.empty() || !active.empty() || !retiring.empty() ||
               !slices.empty();
      };
      if (active.empty() && retiring.empty() && slices.empty())
        cv_work.wait(lock, has_work);
      if (stopping && queue.empty() && active.empty() && retiring.empty() && slices.empty())
        break;
      size_t planned = in_use;
      while (!queue.empty() && active_count + (int)admit.size() < max_active) {
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
      active_count += (int)admit.size();
    }
    for (Pending &p : admit) {
      Running r{p.ticket, p.req, nullptr, p.req.nsweeps, request_bytes(p.req), p.t_submit, now()};
      int rc = ccmc::lattice_new(p.req.Lx, p.req.Ly, nullptr, ring_records(p.req), false, &r.lat);
      if (rc == CCMC_OK)
        rc = ccmc::init_constrained_async(r.lat, p.req.seed, p.req.n, p.req.charged_frac);
      if (rc != CCMC_OK) {
        fail(r, rc);
        continue;
      }
      if (r.remaining == 0)
        retire(r);
      else
        active.push_back(r);
    }

    // (2) results that have landed
    for (size_t i = 0; i < retiring.size();) {
      if (collect(retiring[i])) {
        retiring[i] = retiring.back();
        retiring.pop_back();
      } else {
        ++i;
      }
    }

    // (3) at most kSlicesInFlight slices queued: wait for the oldest
    while ((int)slices.size() >= kSlicesInFlight ||
           (!slices.empty() && active.empty())) {
      cudaEventSynchronize(slices.front());
      events.push_back(slices.front());
      slices.pop_front();
    }
    if (active.empty()) {
      if (!retiring.empty()) std::this_thread::sleep_for(std::chrono::microseconds(100));
      continue;
    }

    // (4) the next slice: every active simulation advances by what fits the
    // time budget; those it finishes retire behind it
    ccmc::TraceRange trace("server slice");
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
    int rc = ccmc::batch_run(batch, lats, sw.data(), beta.data(), Delta.data(), V.data(),
                             J.data(), every.data(), false);
    cudaEvent_t end = event();
    if (rc == CCMC_OK && !end) rc = CCMC_E_CUDA;
    // the slice ends when every lattice's stream has done its part
    for (int i = 0; i < n && rc == CCMC_OK; ++i) {
      cudaEvent_t e = event();
      if (!e || cudaEventRecord(e, ccmc::lattice_stream(lats[i])) != cudaSuccess ||
          cudaStreamWaitEvent(marker, e, 0) != cudaSuccess)
        rc = CCMC_E_CUDA;
      if (e) events.push_back(e);  // a recorded event may be recorded again later
    }
    if (rc == CCMC_OK && cudaEventRecord(end, marker) != cudaSuccess) rc = CCMC_E_CUDA;
    if (end) {
      if (rc == CCMC_OK)
        slices.push_back(end);
      else
        events.push_back(end);
    }
    {
      std::lock_guard<std::mutex> lock(mu);
      ++st.slices;
    }
    std::vector<Running> still;
    for (int i = 0; i < n; ++i) {
      Running &r = active[i];
      r.remaining -= sw[i];
      if (rc != CCMC_OK)
        fail(r, rc);
      else if (r.remaining == 0)
        retire(r);
      else
        still.push_back(r);
    }
    active.swap(still);
  }
  for (cudaEvent_t e : events) cudaEventDestroy(e);
  events.clear();
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
  if (cudaStreamCreateWithFlags(&s->marker, cudaStreamNonBlocking) != cudaSuccess) {
    cudaStreamDestroy(s->stream);
    delete s;
    return CCMC_E_CUDA;
  }
  int rc = ccmc::batch_new(max_active, s->stream, &s->batch);
  if (rc != CCMC_OK) {
    cudaStreamDestroy(s->stream);
    cudaStreamDestroy(s->marker);
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
  out->active = (int64_t)s->active_count;
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
  if (s->marker) cudaStreamDestroy(s->marker);
  delete s;
  return CCMC_OK;
}

}  // extern "C"
