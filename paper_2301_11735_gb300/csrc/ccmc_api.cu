// ccmc_api.cu -- the C ABI of libccmc (declared in include/ccmc.h): handle
// lifecycle, parameter tables, the sweep driver and state transfer.  Host code
// only; the kernels live in ccmc_kernels.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/ccmc.h"
#include "ccmc_fault.h"
#include "ccmc_internal.h"
#include "ccmc_map.h"
#include "ccmc_state.h"
#include "ccmc_trace.h"

using namespace ccmc;

#define CK(call)                                \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return CCMC_E_CUDA;  \
  } while (0)

namespace {

// A sweep of the graph path is captured as a chunk of `sweeps` sweeps; with
// obs_every in [1, 16] the chunk holds a recount after every obs_every-th
// sweep and is replayed only when the run is aligned to obs_every.
struct GraphEntry {
  int sweeps = 0;
  int obs_every = 0;
  cudaGraphExec_t exec = nullptr;
};

constexpr int kChunk = 16;
// Lock-step groups: at least kLockstepMin lattices, each with fewer than
// kLockstepMaxWords a-words per phase.  Measured on GB300: 16 lattices of
// 1024^2 run faster in lock step than on their own streams; 8 of 2048^2 or
// 4 of 4096^2 run faster on their own streams, whose phases fill each other's
// tails.
constexpr int kLockstepMin = 8;
constexpr int64_t kLockstepMaxWords = 16384;

// Lattice memory comes from a library-owned stream-ordered pool per device
// (allocations and frees queued on the lattice's stream, memory kept cached
// in the pool): creating and destroying lattices then never synchronises the
// device, which a server admitting and retiring simulations while others run
// depends on.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaMemPool_t lattice_pool(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = p;
  }
  return g_pool[dev];
}

// bytes of device memory for a lattice of device dev, ordered on stream s
bool dalloc(void **p, size_t bytes, int dev, cudaStream_t s) {
  cudaMemPool_t pool = lattice_pool(dev);
  if (!pool || cudaMallocFromPoolAsync(p, bytes, pool, s) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

void dfree(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

}  // namespace

struct ccmc_lattice {
  Geo g{};
  int h = 1;  // Feistel half width: 4^h >= N
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  uint32_t *d_words = nullptr;
  int64_t *d_ctl = nullptr;
  int64_t *d_partials = nullptr;
  int64_t *d_ring = nullptr;
  int64_t ring_cap = 0;
  int64_t *d_hist = nullptr;
  int nbins = 0;
  void *d_tables = nullptr;
  DevTables t{};
  uint8_t *d_bytes = nullptr;
  int *d_flag = nullptr;
  bool initialised = false;
  uint64_t seed = 0;
  int64_t phases_done = 0;  // global phase index of the next phase
  bool have_params = false;
  double params[4] = {0, 0, 0, 0};  // beta, Delta, V, J
  LaunchCfg cfg{};
  std::vector<GraphEntry> graphs;
  int32_t *d_maps = nullptr;  // paper-map mode: uploaded pairs
  int64_t map_cap = 0;        // int32 entries held by d_maps
  cudaEvent_t map_ev = nullptr;
};

namespace {

int validate_shape(int Lx, int Ly) {
  if (Lx < 4 || Ly < 4 || (Lx & 3) || (Ly & 3)) return CCMC_E_INVAL;
  if ((int64_t)Lx * (int64_t)Ly > ((int64_t)1 << 30)) return CCMC_E_INVAL;
  return CCMC_OK;
}

void set_seed(ccmc_lattice *h, uint64_t seed) {
  h->seed = seed;
  h->g.k0 = (uint32_t)(seed & 0xFFFFFFFFu);
  h->g.k1 = (uint32_t)(seed >> 32);
}

void drop_graphs(ccmc_lattice *h) {
  for (auto &e : h->graphs)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  h->graphs.clear();
}

int upload_params_on(ccmc_lattice *h, double beta, double Delta, double V, double J,
                     cudaStream_t st) {
  if (h->have_params && h->params[0] == beta && h->params[1] == Delta && h->params[2] == V &&
      h->params[3] == J)
    return CCMC_OK;
  std::vector<uint32_t> thr32(kTableN);
  std::vector<uint16_t> thrT(kThrT, 0);
  build_thresholds(beta, Delta, V, J, thr32.data());
  for (int i = 0; i < kTableN; ++i) thrT[i] = threshold_level(thr32[i]);
  CK(cudaMemcpyAsync(h->t.thr32, thr32.data(), sizeof(uint32_t) * kTableN,
                     cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h->t.thrT, thrT.data(), sizeof(uint16_t) * kThrT, cudaMemcpyHostToDevice,
                     st));
  // pageable sources: the copies are staged before the calls return
  h->have_params = true;
  h->params[0] = beta;
  h->params[1] = Delta;
  h->params[2] = V;
  h->params[3] = J;
  return CCMC_OK;
}

int upload_params(ccmc_lattice *h, double beta, double Delta, double V, double J) {
  return upload_params_on(h, beta, Delta, V, J, h->stream);
}

// Queue `sweeps` sweeps starting at phase offset 0 of the control block's base;
// obs_every > 0: a recount after every obs_every-th of them (the caller aligns).
int enqueue_chunk(ccmc_lattice *h, int sweeps, int obs_every) {
  for (int s = 0; s < sweeps; ++s) {
    for (int p = 0; p < 8; ++p) CK(launch_phase(h->g, h->t, 8LL * s + p, h->cfg, h->stream));
    if (obs_every > 0 && (s + 1) % obs_every == 0)
      CK(launch_recount(h->g, h->d_partials, h->d_ring, h->ring_cap, h->d_hist, h->nbins, s + 1,
                        h->stream));
  }
  CK(launch_advance(h->d_ctl, 8LL * sweeps, h->stream));
  return CCMC_OK;
}

int run_graph(ccmc_lattice *h, int sweeps, int obs_every) {
  GraphEntry *hit = nullptr;
  for (auto &e : h->graphs)
    if (e.sweeps == sweeps && e.obs_every == obs_every) hit = &e;
  if (!hit) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_chunk(h, sweeps, obs_every);
    const cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
    if (rc != CCMC_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return CCMC_E_CUDA;
    }
    GraphEntry e;
    e.sweeps = sweeps;
    e.obs_every = obs_every;
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return CCMC_E_CUDA;
    h->graphs.push_back(e);
    hit = &h->graphs.back();
  }
  CK(cudaGraphLaunch(hit->exec, h->stream));
  return CCMC_OK;
}

// Drives nsweeps sweeps from absolute sweep index sweeps_done: replayable
// chunks of G sweeps (chunk(G, obs): G a multiple of obs when 0 < obs <= 16,
// started aligned to obs) where possible, single directly launched sweeps
// (single(obs_due)) to align or finish.
template <typename Chunk, typename Single>
int drive_sweeps(int64_t sweeps_done, int64_t nsweeps, int obs_every, Chunk chunk, Single single) {
  int64_t s = 0;
  while (s < nsweeps) {
    const int64_t abs_sweep = sweeps_done + s;
    const int64_t remaining = nsweeps - s;
    if (obs_every > 0 && obs_every <= kChunk) {
      const int g = obs_every * (kChunk / obs_every);
      if (abs_sweep % obs_every == 0 && remaining >= g) {
        const int rc = chunk(g, obs_every);
        if (rc) return rc;
        s += g;
        continue;
      }
    } else {
      const int64_t dist = obs_every > 0 ? obs_every - abs_sweep % obs_every : INT64_MAX;
      if (remaining >= kChunk && dist > kChunk) {
        const int rc = chunk(kChunk, 0);
        if (rc) return rc;
        s += kChunk;
        continue;
      }
    }
    const int rc = single(obs_every > 0 && (abs_sweep + 1) % obs_every == 0);
    if (rc) return rc;
    s += 1;
  }
  return CCMC_OK;
}

int write_recount_latest(ccmc_lattice *h) {
  CK(launch_recount(h->g, h->d_partials, nullptr, 0, nullptr, 0, 0, h->stream));
  return CCMC_OK;
}

void fill_obs(const ccmc_lattice *h, const int64_t *rec, ccmc_obs *o) {
  o->sweeps_done = rec[0];
  o->Nc = rec[1];
  o->BV = rec[2];
  o->BJ = rec[3];
  o->M = rec[4];
  o->M_stag = rec[5];
  o->S_sum = rec[6];
  o->S_stag = rec[7];
  const double Delta = h->params[1], V = h->params[2], J = h->params[3];
  o->E = Delta * (double)rec[1] + V * (double)rec[2] + (0.25 * J) * (double)rec[3];
}

int check_status(ccmc_lattice *h) {
  int64_t st = 0;
  CK(cudaMemcpyAsync(&st, h->d_ctl + kCtlStatus, sizeof(int64_t), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return st == 0 ? CCMC_OK : CCMC_E_TIMEOUT;
}

}  // namespace

int ccmc::lattice_new(int Lx, int Ly, void *cuda_stream, int64_t obs_capacity, bool wait,
                      ccmc_lattice **out) {
  if (!out) return CCMC_E_INVAL;
  *out = nullptr;
  int rc = validate_shape(Lx, Ly);
  if (rc) return rc;
  if (fault_injected("alloc")) return CCMC_E_NOMEM;
  ccmc_lattice *h = new (std::nothrow) ccmc_lattice();
  if (!h) return CCMC_E_NOMEM;
  Geo &g = h->g;
  g.Lx = Lx;
  g.Ly = Ly;
  g.Cx = Lx / 4;
  g.Cy = Ly / 4;
  g.W = (g.Cx + 15) / 16;
  g.cstride = (int64_t)g.Cy * g.W;
  const uint64_t N = (uint64_t)Lx * (uint64_t)Ly;
  g.rej = (0 - N) % N;
  h->cfg.phase_grid_cap = phase_resident_grid((g.Cx & 15) == 0);
  if (tile_path_ok(g) && !std::getenv("CCMC_NO_TILE")) {
    h->cfg.tile_grid = tile_resident_grid();
    h->cfg.tile_grid_small = tile_resident_grid_small();
    // CCMC_TILE_GRID=n (tests): the pipelined tile kernel with at most n CTAs,
    // so that small lattices take several tiles per CTA
    if (const char *e = std::getenv("CCMC_TILE_GRID")) {
      const int n = std::atoi(e);
      if (n > 0 && h->cfg.tile_grid > 0) {
        h->cfg.tile_grid = n < h->cfg.tile_grid ? n : h->cfg.tile_grid;
        h->cfg.tile_grid_small = 0;
      }
    }
  }
  while (((int64_t)1 << (2 * h->h)) < (int64_t)N) ++h->h;
  h->ring_cap = obs_capacity > 0 ? obs_capacity : 4096;
  cudaGetDevice(&h->device);
  auto fail = [&](int code) {
    ccmc_lattice_destroy(h);
    return code;
  };
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(CCMC_E_CUDA);
    h->own_stream = true;
  }
  const int np = recount_grid(g);
  const int dev = h->device;
  const size_t tb = sizeof(uint32_t) * (kTableN + 2 * kMoveN) + sizeof(uint16_t) * kThrT;
  if (!dalloc((void **)&h->d_words, sizeof(uint32_t) * 16 * g.cstride, dev, h->stream) ||
      !dalloc((void **)&h->d_ctl, sizeof(int64_t) * kCtlWords, dev, h->stream) ||
      !dalloc((void **)&h->d_partials, sizeof(int64_t) * 7 * np, dev, h->stream) ||
      !dalloc((void **)&h->d_ring, sizeof(int64_t) * 8 * h->ring_cap, dev, h->stream) ||
      !dalloc((void **)&h->d_flag, sizeof(int), dev, h->stream) ||
      !dalloc(&h->d_tables, tb, dev, h->stream))
    return fail(CCMC_E_NOMEM);
  // the threshold levels and the move table one after another (a multiple of
  // 16 bytes from a 256-byte aligned base): the tile kernels copy them into
  // shared memory with one bulk copy; thr32 after them
  char *p = (char *)h->d_tables;
  h->t.thrT = (uint16_t *)p;
  p += sizeof(uint16_t) * kThrT;
  h->t.trans = (uint32_t *)p;
  p += sizeof(uint32_t) * 2 * kMoveN;
  h->t.thr32 = (uint32_t *)p;
  g.words = h->d_words;
  g.ctl = h->d_ctl;
  uint32_t tr[2 * kMoveN];
  if (!build_transitions(tr)) return fail(CCMC_E_INVAL);
  if (cudaMemcpyAsync(h->t.trans, tr, sizeof(tr), cudaMemcpyHostToDevice, h->stream) !=
          cudaSuccess ||
      cudaMemsetAsync(h->d_words, 0, sizeof(uint32_t) * 16 * g.cstride, h->stream) !=
          cudaSuccess ||
      launch_set_ctl(h->d_ctl, 0, h->stream) != cudaSuccess ||
      (wait && cudaStreamSynchronize(h->stream) != cudaSuccess))
    return fail(CCMC_E_CUDA);
  *out = h;
  return CCMC_OK;
}

static int ensure_bytes(ccmc_lattice *h) {
  if (h->d_bytes) return CCMC_OK;
  const size_t N = (size_t)h->g.Lx * h->g.Ly;
  if (!dalloc((void **)&h->d_bytes, N, h->device, h->stream)) return CCMC_E_NOMEM;
  return CCMC_OK;
}

int ccmc::init_counts_async(ccmc_lattice *h, uint64_t seed, int64_t n_plus, int64_t n_minus) {
  if (!h) return CCMC_E_INVAL;
  const int64_t N = (int64_t)h->g.Lx * h->g.Ly;
  if (n_plus < 0 || n_minus < 0 || n_plus + n_minus > N) return CCMC_E_INVAL;
  set_seed(h, seed);
  CK(launch_set_ctl(h->d_ctl, 0, h->stream));
  CK(launch_init(h->g, h->h, n_plus, n_minus, h->stream));
  if (h->d_hist) CK(cudaMemsetAsync(h->d_hist, 0, sizeof(int64_t) * 3 * h->nbins, h->stream));
  h->phases_done = 0;
  h->initialised = true;
  return CCMC_OK;
}

int ccmc::init_constrained_async(ccmc_lattice *h, uint64_t seed, double n, double charged_frac) {
  if (!h) return CCMC_E_INVAL;
  if (!std::isfinite(n)) return CCMC_E_INVAL;
  if (charged_frac < 0.0) charged_frac = 0.3;
  if (!std::isfinite(charged_frac)) return CCMC_E_INVAL;
  const int64_t N = (int64_t)h->g.Lx * h->g.Ly;
  const int64_t Q = std::llround(n * (double)N);
  int64_t C = std::llround(charged_frac * (double)N);
  const int64_t aQ = Q < 0 ? -Q : Q;
  if (C < aQ) C = aQ;
  if ((C - Q) & 1) C += 1;
  if (C > N) return CCMC_E_INVAL;
  return init_counts_async(h, seed, (C + Q) / 2, (C - Q) / 2);
}

int ccmc::export_async(ccmc_lattice *h, int64_t *rec, int64_t *status, int64_t *count,
                       int64_t *ring, uint8_t *state, cudaEvent_t ready) {
  if (!h || !rec || !status || !h->initialised) return CCMC_E_INVAL;
  int rc = write_recount_latest(h);
  if (rc) return rc;
  CK(cudaMemcpyAsync(rec, h->d_ctl + kCtlLatest, sizeof(int64_t) * 8, cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaMemcpyAsync(status, h->d_ctl + kCtlStatus, sizeof(int64_t), cudaMemcpyDeviceToHost,
                     h->stream));
  if (ring) {
    if (!count) return CCMC_E_INVAL;
    CK(cudaMemcpyAsync(count, h->d_ctl + kCtlObsCount, sizeof(int64_t), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaMemcpyAsync(ring, h->d_ring, sizeof(int64_t) * 8 * h->ring_cap,
                       cudaMemcpyDeviceToHost, h->stream));
  }
  if (state) {
    rc = ensure_bytes(h);
    if (rc) return rc;
    CK(launch_unpack(h->g, h->d_bytes, h->stream));
    CK(cudaMemcpyAsync(state, h->d_bytes, (size_t)h->g.Lx * h->g.Ly, cudaMemcpyDeviceToHost,
                       h->stream));
  }
  CK(cudaEventRecord(ready, h->stream));
  return CCMC_OK;
}

void ccmc::obs_of_record(const ccmc_lattice *h, const int64_t *rec, ccmc_obs *out) {
  int64_t r[8];
  std::memcpy(r, rec, sizeof(r));
  r[0] = h->phases_done / 8;
  fill_obs(h, r, out);
}

int64_t ccmc::series_of_ring(const ccmc_lattice *h, const int64_t *ring, int64_t count,
                             ccmc_obs *out, int64_t cap) {
  const int64_t held = count < h->ring_cap ? count : h->ring_cap;
  int64_t n = 0;
  for (int64_t r = count - held; r < count && n < cap; ++r, ++n)
    fill_obs(h, ring + 8 * (r % h->ring_cap), out + n);
  return n;
}

int64_t ccmc::ring_capacity(const ccmc_lattice *h) { return h->ring_cap; }

cudaStream_t ccmc::lattice_stream(const ccmc_lattice *h) { return h->stream; }

extern "C" {

const char *ccmc_strerror(int code) {
  switch (code) {
    case CCMC_OK: return "ok";
    case CCMC_E_INVAL: return "invalid argument";
    case CCMC_E_NOMEM: return "out of memory";
    case CCMC_E_CUDA: return "CUDA error";
    case CCMC_E_TIMEOUT: return "device wait timed out";
    case CCMC_E_BUDGET: return "memory budget exhausted";
    case CCMC_E_STATE: return "call out of order";
    case CCMC_E_NOTFOUND: return "not found";
    default: return "unknown error";
  }
}

int ccmc_threshold_table(double beta, double Delta, double V, double J, uint32_t *out) {
  if (!out || !(beta >= 0.0) || !std::isfinite(Delta) || !std::isfinite(V) ||
      !std::isfinite(J))
    return CCMC_E_INVAL;
  build_thresholds(beta, Delta, V, J, out);
  return CCMC_OK;
}

int ccmc_lattice_create(int Lx, int Ly, void *cuda_stream, int64_t obs_capacity,
                        ccmc_lattice **out) {
  return lattice_new(Lx, Ly, cuda_stream, obs_capacity, true, out);
}

int ccmc_lattice_destroy(ccmc_lattice *h) {
  if (!h) return CCMC_E_INVAL;
  if (h->stream) cudaStreamSynchronize(h->stream);  // this lattice's work only
  drop_graphs(h);
  dfree(h->d_words, h->stream);
  dfree(h->d_ctl, h->stream);
  dfree(h->d_partials, h->stream);
  dfree(h->d_ring, h->stream);
  dfree(h->d_hist, h->stream);
  dfree(h->d_tables, h->stream);
  dfree(h->d_bytes, h->stream);
  dfree(h->d_flag, h->stream);
  dfree(h->d_maps, h->stream);
  if (h->map_ev) cudaEventDestroy(h->map_ev);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return CCMC_OK;
}

int ccmc_init_counts(ccmc_lattice *h, uint64_t seed, int64_t n_plus, int64_t n_minus) {
  const int rc = init_counts_async(h, seed, n_plus, n_minus);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return CCMC_OK;
}

int ccmc_init_constrained(ccmc_lattice *h, uint64_t seed, double n, double charged_frac) {
  const int rc = init_constrained_async(h, seed, n, charged_frac);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return CCMC_OK;
}

int ccmc_sweep(ccmc_lattice *h, int64_t nsweeps, double beta, double Delta, double V, double J,
               int obs_every) {
  if (!h || nsweeps < 0) return CCMC_E_INVAL;
  if (!(beta >= 0.0) || !std::isfinite(Delta) || !std::isfinite(V) || !std::isfinite(J))
    return CCMC_E_INVAL;
  if (!h->initialised) return CCMC_E_STATE;
  if (fault_injected("launch")) return CCMC_E_CUDA;
  TraceRange trace("ccmc_sweep");
  int rc = upload_params(h, beta, Delta, V, J);
  if (rc) return rc;
  if (nsweeps > 0 && h->phases_done % 8) {
    // finish the sweep that ccmc_phases left open; it counts as the first one
    const int64_t rest = 8 - h->phases_done % 8;
    rc = ccmc_phases(h, rest, beta, Delta, V, J);
    if (rc) return rc;
    if (obs_every > 0 && (h->phases_done / 8) % obs_every == 0)
      CK(launch_recount(h->g, h->d_partials, h->d_ring, h->ring_cap, h->d_hist, h->nbins, 0,
                        h->stream));
    --nsweeps;
  }
  rc = drive_sweeps(
      h->phases_done / 8, nsweeps, obs_every,
      [&](int g, int obs) { return run_graph(h, g, obs); },
      [&](bool obs_due) {
        for (int p = 0; p < 8; ++p) CK(launch_phase(h->g, h->t, p, h->cfg, h->stream));
        if (obs_due)
          CK(launch_recount(h->g, h->d_partials, h->d_ring, h->ring_cap, h->d_hist, h->nbins, 1,
                            h->stream));
        CK(launch_advance(h->d_ctl, 8, h->stream));
        return CCMC_OK;
      });
  if (rc) return rc;
  h->phases_done += 8 * nsweeps;
  return CCMC_OK;
}

int ccmc_phases(ccmc_lattice *h, int64_t nphases, double beta, double Delta, double V,
                double J) {
  if (!h || nphases < 0) return CCMC_E_INVAL;
  if (!(beta >= 0.0) || !std::isfinite(Delta) || !std::isfinite(V) || !std::isfinite(J))
    return CCMC_E_INVAL;
  if (!h->initialised) return CCMC_E_STATE;
  if (fault_injected("launch")) return CCMC_E_CUDA;
  int rc = upload_params(h, beta, Delta, V, J);
  if (rc) return rc;
  for (int64_t p = 0; p < nphases; ++p) {
    CK(launch_phase(h->g, h->t, 0, h->cfg, h->stream));
    CK(launch_advance(h->d_ctl, 1, h->stream));
  }
  h->phases_done += nphases;
  return CCMC_OK;
}

int ccmc_sync(ccmc_lattice *h) {
  if (!h) return CCMC_E_INVAL;
  return check_status(h);
}

int ccmc_map_apply(ccmc_lattice *h, const int32_t *pairs, int64_t map0, int64_t nmaps,
                   double beta, double Delta, double V, double J) {
  if (!h || map0 < 0 || nmaps < 0 || (nmaps > 0 && !pairs) || !(beta >= 0.0) ||
      !std::isfinite(Delta) || !std::isfinite(V) || !std::isfinite(J))
    return CCMC_E_INVAL;
  if (!h->initialised) return CCMC_E_STATE;
  if (nmaps == 0) return CCMC_OK;
  const int64_t P = ccmc_map_size(h->g.Lx, h->g.Ly);
  const int64_t N = (int64_t)h->g.Lx * h->g.Ly;
  if (nmaps > ((int64_t)1 << 40) / (2 * P)) return CCMC_E_INVAL;
  const int64_t n = 2 * P * nmaps;
  // the kernel addresses the lattice with these indices: reject any outside it
  for (int64_t i = 0; i < n; ++i)
    if (pairs[i] < 0 || pairs[i] >= N) return CCMC_E_INVAL;
  if (!h->map_ev && cudaEventCreateWithFlags(&h->map_ev, cudaEventDisableTiming) != cudaSuccess)
    return CCMC_E_CUDA;
  if (n > h->map_cap) {
    dfree(h->d_maps, h->stream);  // after the earlier maps' work on the stream
    h->d_maps = nullptr;
    h->map_cap = 0;
    if (!dalloc((void **)&h->d_maps, sizeof(int32_t) * n, h->device, h->stream))
      return CCMC_E_NOMEM;
    h->map_cap = n;
  }
  int rc = upload_params(h, beta, Delta, V, J);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h->d_maps, pairs, sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->stream));
  CK(cudaEventRecord(h->map_ev, h->stream));
  for (int64_t k = 0; k < nmaps; ++k)
    CK(launch_map(h->g, h->d_maps + 2 * P * k, P, (uint64_t)(map0 + k), h->t, h->stream));
  // the caller may reuse `pairs` once the copy has run
  CK(cudaEventSynchronize(h->map_ev));
  return CCMC_OK;
}

int ccmc_observables(ccmc_lattice *h, ccmc_obs *out) {
  if (!h || !out) return CCMC_E_INVAL;
  if (!h->initialised) return CCMC_E_STATE;
  int rc = write_recount_latest(h);
  if (rc) return rc;
  int64_t rec[8];
  CK(cudaMemcpyAsync(rec, h->d_ctl + kCtlLatest, sizeof(rec), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  rec[0] = h->phases_done / 8;
  fill_obs(h, rec, out);
  return check_status(h);
}

int ccmc_obs_series(ccmc_lattice *h, ccmc_obs *out, int64_t cap, int64_t *n_written) {
  if (!h || !n_written || cap < 0 || (cap > 0 && !out)) return CCMC_E_INVAL;
  int64_t cnt = 0;
  CK(cudaMemcpyAsync(&cnt, h->d_ctl + kCtlObsCount, sizeof(int64_t), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const int64_t held = cnt < h->ring_cap ? cnt : h->ring_cap;
  const int64_t first = cnt - held;
  std::vector<int64_t> ring((size_t)(8 * h->ring_cap));
  CK(cudaMemcpyAsync(ring.data(), h->d_ring, sizeof(int64_t) * 8 * h->ring_cap,
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  int64_t n = 0;
  for (int64_t r = first; r < cnt && n < cap; ++r, ++n)
    fill_obs(h, ring.data() + 8 * (r % h->ring_cap), out + n);
  *n_written = n;
  return CCMC_OK;
}

int ccmc_hist_enable(ccmc_lattice *h, int nbins) {
  if (!h || nbins < 1 || nbins > (1 << 20)) return CCMC_E_INVAL;
  CK(cudaStreamSynchronize(h->stream));
  drop_graphs(h);  // captured recounts hold the old histogram pointer
  dfree(h->d_hist, h->stream);
  h->d_hist = nullptr;
  h->nbins = 0;
  if (!dalloc((void **)&h->d_hist, sizeof(int64_t) * 3 * nbins, h->device, h->stream))
    return CCMC_E_NOMEM;
  h->nbins = nbins;
  CK(cudaMemsetAsync(h->d_hist, 0, sizeof(int64_t) * 3 * nbins, h->stream));
  return CCMC_OK;
}

int ccmc_hist_get(ccmc_lattice *h, int64_t *out) {
  if (!h || !out) return CCMC_E_INVAL;
  if (!h->d_hist) return CCMC_E_STATE;
  CK(cudaMemcpyAsync(out, h->d_hist, sizeof(int64_t) * 3 * h->nbins, cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CCMC_OK;
}


int ccmc_get_state(ccmc_lattice *h, uint8_t *host_out) {
  if (!h || !host_out) return CCMC_E_INVAL;
  if (!h->initialised) return CCMC_E_STATE;
  int rc = ensure_bytes(h);
  if (rc) return rc;
  const size_t N = (size_t)h->g.Lx * h->g.Ly;
  CK(launch_unpack(h->g, h->d_bytes, h->stream));
  CK(cudaMemcpyAsync(host_out, h->d_bytes, N, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CCMC_OK;
}

int ccmc_get_state_packed(ccmc_lattice *h, uint8_t *host_out) {
  if (!h || !host_out) return CCMC_E_INVAL;
  if (!h->initialised) return CCMC_E_STATE;
  int rc = ensure_bytes(h);
  if (rc) return rc;
  const size_t nb = (size_t)h->g.Lx * h->g.Ly / 4;
  CK(launch_unpack2(h->g, h->d_bytes, h->stream));
  CK(cudaMemcpyAsync(host_out, h->d_bytes, nb, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CCMC_OK;
}

int ccmc_set_state_packed(ccmc_lattice *h, const uint8_t *host_in, uint64_t seed,
                          int64_t sweeps_done) {
  if (!h || !host_in || sweeps_done < 0 || sweeps_done > ((int64_t)1 << 59)) return CCMC_E_INVAL;
  int rc = ensure_bytes(h);
  if (rc) return rc;
  const size_t nb = (size_t)h->g.Lx * h->g.Ly / 4;
  // every 2-bit code is a state: nothing to validate, nothing to wait for
  CK(cudaMemcpyAsync(h->d_bytes, host_in, nb, cudaMemcpyHostToDevice, h->stream));
  set_seed(h, seed);
  CK(launch_pack2(h->g, h->d_bytes, h->stream));
  CK(launch_set_ctl(h->d_ctl, 8 * sweeps_done, h->stream));
  if (h->d_hist) CK(cudaMemsetAsync(h->d_hist, 0, sizeof(int64_t) * 3 * h->nbins, h->stream));
  h->phases_done = 8 * sweeps_done;
  h->initialised = true;
  return CCMC_OK;
}

int ccmc_set_state(ccmc_lattice *h, const uint8_t *host_in, uint64_t seed, int64_t sweeps_done) {
  if (!h || !host_in || sweeps_done < 0) return CCMC_E_INVAL;
  int rc = ensure_bytes(h);
  if (rc) return rc;
  const size_t N = (size_t)h->g.Lx * h->g.Ly;
  int zero = 0, bad = 0;
  CK(cudaMemcpyAsync(h->d_flag, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_bytes, host_in, N, cudaMemcpyHostToDevice, h->stream));
  set_seed(h, seed);
  CK(launch_pack(h->g, h->d_bytes, h->d_flag, h->stream));
  CK(launch_set_ctl(h->d_ctl, 8 * sweeps_done, h->stream));
  if (h->d_hist) CK(cudaMemsetAsync(h->d_hist, 0, sizeof(int64_t) * 3 * h->nbins, h->stream));
  CK(cudaMemcpyAsync(&bad, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (bad) {
    h->initialised = false;
    return CCMC_E_INVAL;
  }
  h->phases_done = 8 * sweeps_done;
  h->initialised = true;
  return CCMC_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Batches: many lattices swept together.  Lattices whose packed words fit the
// resident limit run in one persistent resident_kernel launch on the batch
// stream (each CTA holds a whole lattice in shared memory); larger ones run the
// per-phase path on their own streams at the same time.
struct ccmc_batch {
  std::vector<ccmc_lattice *> lats;
  int cap = 0;  // largest number of lattices one launch may hold
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  JobDesc *d_jobs = nullptr;
  int *d_queue = nullptr;
  int threads = 256;
  int64_t resident_max_sites = (int64_t)1 << 18;
  int ctas_per_sm = 2;
  int max_tpw = 4;
  int sms = 152;
  cudaEvent_t ev = nullptr;
  std::vector<cudaEvent_t> lat_ev;
  MultiJob *d_multi = nullptr;  // lock-step groups of large lattices
  struct MultiGraph {
    std::vector<ccmc_lattice *> members;
    int sweeps, obs_every;
    int64_t off;
    cudaGraphExec_t exec;
  };
  std::vector<MultiGraph> graphs;
};

namespace {
JobDesc job_of(ccmc_lattice *h, int64_t nsweeps, int obs_every) {
  JobDesc d{};
  d.g = h->g;
  d.thrT = h->t.thrT;
  d.thr32 = h->t.thr32;
  d.trans = h->t.trans;
  d.nsweeps = nsweeps;
  d.ring = h->d_ring;
  d.ring_cap = h->ring_cap;
  d.hist = h->d_hist;
  d.nbins = h->nbins;
  d.obs_every = obs_every;
  return d;
}
}  // namespace

namespace {

struct MultiGroup {
  std::vector<ccmc_lattice *> m;
  int64_t off;  // first slot in d_multi
  int grid;
  bool aligned;
  bool tiled;  // every member takes the tile-staged phase
};

int enqueue_multi_chunk(ccmc_batch *b, const MultiGroup &G, int sweeps, int obs_every) {
  for (int s = 0; s < sweeps; ++s) {
    for (int p = 0; p < 8; ++p)
      CK(G.tiled ? launch_phase_tile_multi(b->d_multi + G.off, (int)G.m.size(), G.grid,
                                           8LL * s + p, b->stream)
                 : launch_phase_multi(b->d_multi + G.off, (int)G.m.size(), G.grid, G.aligned,
                                      8LL * s + p, b->stream));
    if (obs_every > 0 && (s + 1) % obs_every == 0)
      for (ccmc_lattice *h : G.m)
        CK(launch_recount(h->g, h->d_partials, h->d_ring, h->ring_cap, h->d_hist, h->nbins,
                          s + 1, b->stream));
  }
  for (ccmc_lattice *h : G.m) CK(launch_advance(h->d_ctl, 8LL * sweeps, b->stream));
  return CCMC_OK;
}

int run_multi_graph(ccmc_batch *b, const MultiGroup &G, int sweeps, int obs_every) {
  for (auto &e : b->graphs)
    if (e.members == G.m && e.sweeps == sweeps && e.obs_every == obs_every && e.off == G.off) {
      CK(cudaGraphLaunch(e.exec, b->stream));
      return CCMC_OK;
    }
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue_multi_chunk(b, G, sweeps, obs_every);
  const cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
  if (rc != CCMC_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return CCMC_E_CUDA;
  }
  ccmc_batch::MultiGraph e{G.m, sweeps, obs_every, G.off, nullptr};
  const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return CCMC_E_CUDA;
  b->graphs.push_back(e);
  CK(cudaGraphLaunch(e.exec, b->stream));
  return CCMC_OK;
}

// Sweep a lock-step group (same position, sweeps, observable interval and
// alignment) with one phase launch per phase for all of them.
int run_multi(ccmc_batch *b, MultiGroup &G, int64_t nsweeps, int obs_every) {
  int64_t words = 0, tiles = 0;
  for (ccmc_lattice *h : G.m) words += (int64_t)h->g.Cy * h->g.W;
  for (ccmc_lattice *h : G.m) tiles += G.tiled ? tile_count(h->g) : 0;
  const int wave = G.tiled ? G.m[0]->cfg.tile_grid : phase_resident_grid(G.aligned);
  // tile path: the same number of tiles per CTA for every member, as few as
  // one wave of CTAs allows
  int64_t per_cta = G.tiled ? (tiles + wave - 1) / wave : 1;
  if (G.tiled)
    for (;;) {
      int64_t ctas = 0;
      for (ccmc_lattice *h : G.m) ctas += (tile_count(h->g) + per_cta - 1) / per_cta;
      if (ctas <= wave) break;
      ++per_cta;
    }
  std::vector<MultiJob> jobs;
  int begin = 0;
  for (ccmc_lattice *h : G.m) {
    const int64_t w = (int64_t)h->g.Cy * h->g.W;
    int share;
    if (G.tiled) {
      share = (int)((tile_count(h->g) + per_cta - 1) / per_cta);
    } else {
      share = (int)((double)wave * (double)w / (double)words);
      const int64_t need = (w + 255) / 256;  // more CTAs than a word each would idle
      if (share > need) share = (int)need;
      if (share < 1) share = 1;
    }
    MultiJob j{};
    j.g = h->g;
    j.thrT = h->t.thrT;
    j.thr32 = h->t.thr32;
    j.trans = h->t.trans;
    j.cta_begin = begin;
    j.cta_count = share;
    begin += share;
    jobs.push_back(j);
  }
  G.grid = begin;
  CK(cudaMemcpyAsync(b->d_multi + G.off, jobs.data(), sizeof(MultiJob) * jobs.size(),
                     cudaMemcpyHostToDevice, b->stream));
  const int rc = drive_sweeps(
      G.m[0]->phases_done / 8, nsweeps, obs_every,
      [&](int g, int obs) { return run_multi_graph(b, G, g, obs); },
      [&](bool obs_due) {
        for (int p = 0; p < 8; ++p)
          CK(G.tiled ? launch_phase_tile_multi(b->d_multi + G.off, (int)G.m.size(), G.grid, p,
                                               b->stream)
                     : launch_phase_multi(b->d_multi + G.off, (int)G.m.size(), G.grid, G.aligned,
                                          p, b->stream));
        if (obs_due)
          for (ccmc_lattice *h : G.m)
            CK(launch_recount(h->g, h->d_partials, h->d_ring, h->ring_cap, h->d_hist, h->nbins,
                              1, b->stream));
        for (ccmc_lattice *h : G.m) CK(launch_advance(h->d_ctl, 8, b->stream));
        return CCMC_OK;
      });
  if (rc) return rc;
  for (ccmc_lattice *h : G.m) h->phases_done += 8 * nsweeps;
  return CCMC_OK;
}

}  // namespace

namespace ccmc {

int batch_run(ccmc_batch *b, const std::vector<ccmc_lattice *> &lats, const int64_t *nsweeps,
              const double *beta, const double *Delta, const double *V, const double *J,
              const int *obs_every, bool lockstep) {
  const int n = (int)lats.size();
  if (n > b->cap) return CCMC_E_INVAL;
  TraceRange trace("ccmc_batch_run");
  for (int i = 0; i < n; ++i) {
    if (nsweeps[i] < 0 || !(beta[i] >= 0.0) || !std::isfinite(Delta[i]) ||
        !std::isfinite(V[i]) || !std::isfinite(J[i]))
      return CCMC_E_INVAL;
    ccmc_lattice *h = lats[i];
    if (!h || !h->initialised || h->phases_done % 8) return CCMC_E_STATE;
    for (int k = 0; k < i; ++k)
      if (lats[k] == h) return CCMC_E_INVAL;  // a lattice may appear once
  }
  std::vector<JobDesc> jobs;
  std::vector<int> resident;
  for (int i = 0; i < n; ++i) {
    ccmc_lattice *h = lats[i];
    const int64_t sites = 16 * h->g.cstride * 16;  // padded sites held in words
    if (nsweeps[i] == 0 || sites > b->resident_max_sites) continue;
    // order the batch stream after work already queued on this lattice's stream
    if (h->stream != b->stream) {
      CK(cudaEventRecord(b->lat_ev[i], h->stream));
      CK(cudaStreamWaitEvent(b->stream, b->lat_ev[i], 0));
    }
    int rc = upload_params_on(h, beta[i], Delta[i], V[i], J[i], b->stream);
    if (rc) return rc;
    jobs.push_back(job_of(h, nsweeps[i], obs_every[i]));
    jobs.back().max_tpw = b->max_tpw;
    resident.push_back(i);
  }
  if (!jobs.empty()) {
    // When there are more lattices than CTAs resident at once, those whose
    // words fit one warp's share of the CTA's shared memory run one a warp
    // (eight in a CTA of 256 threads): run by a whole CTA they would leave
    // most of its threads idle through every phase and hold back the lattices
    // queued behind them.  With CTAs to spare, a whole CTA runs each lattice
    // (its eight phase schedules drawn in parallel, its tables in shared
    // memory: 10.3 against 13.6 us a sweep for a 16x16 lattice alone).
    // One-warp lattices come last; before them, and among them, largest
    // first, so that the queue hands the longest jobs out before the short
    // ones.
    int64_t max_words = 0;
    for (const JobDesc &j : jobs) max_words = std::max(max_words, 16 * j.g.cstride);
    const int64_t warp_words = resident_warp_words(b->threads, max_words);
    const int64_t resident_ctas =
        (int64_t)b->sms *
        std::min(b->ctas_per_sm, resident_ctas_per_sm(b->threads, max_words));
    const bool pack = (int64_t)jobs.size() > resident_ctas;
    for (JobDesc &j : jobs) j.warp = pack && 16 * j.g.cstride <= warp_words ? 1 : 0;
    std::vector<int> order(jobs.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
      if (jobs[x].warp != jobs[y].warp) return jobs[x].warp < jobs[y].warp;
      const int64_t wx = (int64_t)jobs[x].g.Lx * jobs[x].g.Ly * jobs[x].nsweeps;
      const int64_t wy = (int64_t)jobs[y].g.Lx * jobs[y].g.Ly * jobs[y].nsweeps;
      return wx > wy;
    });
    std::vector<JobDesc> sorted;
    for (int k : order) sorted.push_back(jobs[k]);
    CK(cudaMemcpyAsync(b->d_jobs, sorted.data(), sizeof(JobDesc) * sorted.size(),
                       cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemsetAsync(b->d_queue, 0, sizeof(int), b->stream));
    int grid = b->sms * b->ctas_per_sm;
    if (grid > (int)sorted.size()) grid = (int)sorted.size();
    CK(launch_resident(b->d_jobs, (int)sorted.size(), b->d_queue, grid, b->threads, max_words,
                       b->stream));
    CK(cudaEventRecord(b->ev, b->stream));
    for (int i : resident) {
      ccmc_lattice *h = lats[i];
      h->phases_done += 8 * nsweeps[i];
      if (h->stream != b->stream) CK(cudaStreamWaitEvent(h->stream, b->ev, 0));
    }
  }
  // The large lattices: those at the same position with the same sweeps,
  // observable interval and alignment advance in lock-step with one phase
  // launch for all of them (on the batch stream); the others run the per-phase
  // path on their own streams.  Both overlap the resident launch.
  std::vector<char> used(n, 0);
  int64_t off = 0;
  for (int i = 0; i < n; ++i) {
    ccmc_lattice *h = lats[i];
    const int64_t sites = 16 * h->g.cstride * 16;
    if (used[i] || nsweeps[i] == 0 || sites <= b->resident_max_sites) continue;
    MultiGroup G{{h}, off, 0, (h->g.Cx & 15) == 0, h->cfg.tile_grid > 0};
    used[i] = 1;
    auto small = [](const ccmc_lattice *x) { return (int64_t)x->g.Cy * x->g.W < kLockstepMaxWords; };
    for (int k = i + 1; k < n && lockstep && small(h); ++k) {
      ccmc_lattice *o = lats[k];
      if (used[k] || nsweeps[k] != nsweeps[i] || obs_every[k] != obs_every[i] ||
          o->phases_done != h->phases_done || ((o->g.Cx & 15) == 0) != G.aligned ||
          (o->cfg.tile_grid > 0) != G.tiled || !small(o) ||
          16 * o->g.cstride * 16 <= b->resident_max_sites)
        continue;
      G.m.push_back(o);
      used[k] = 1;
    }
    // Few or large lattices run on their own streams (see kLockstepMin).
    if ((int)G.m.size() < kLockstepMin) {
      for (ccmc_lattice *o : G.m) {
        const int k = (int)(std::find(lats.begin(), lats.end(), o) - lats.begin());
        const int rc = ccmc_sweep(o, nsweeps[k], beta[k], Delta[k], V[k], J[k], obs_every[k]);
        if (rc) return rc;
      }
      continue;
    }
    for (ccmc_lattice *o : G.m) {
      const int k = (int)(std::find(lats.begin(), lats.end(), o) - lats.begin());
      if (o->stream != b->stream) {
        CK(cudaEventRecord(b->lat_ev[k], o->stream));
        CK(cudaStreamWaitEvent(b->stream, b->lat_ev[k], 0));
      }
      const int rc = upload_params_on(o, beta[k], Delta[k], V[k], J[k], b->stream);
      if (rc) return rc;
    }
    const int rc = run_multi(b, G, nsweeps[i], obs_every[i]);
    if (rc) return rc;
    off += (int64_t)G.m.size();
    CK(cudaEventRecord(b->ev, b->stream));
    for (ccmc_lattice *o : G.m)
      if (o->stream != b->stream) CK(cudaStreamWaitEvent(o->stream, b->ev, 0));
  }
  return CCMC_OK;
}

}  // namespace ccmc

extern "C" {

int ccmc_batch_create(int count, ccmc_lattice *const *lattices, void *cuda_stream,
                      ccmc_batch **out) {
  if (!out || count < 1 || !lattices) return CCMC_E_INVAL;
  *out = nullptr;
  for (int i = 0; i < count; ++i)
    if (!lattices[i]) return CCMC_E_INVAL;
  if (ccmc::fault_injected("alloc")) return CCMC_E_NOMEM;
  const int rc = ccmc::batch_new(count, (cudaStream_t)cuda_stream, out);
  if (rc != CCMC_OK) return rc;
  (*out)->lats.assign(lattices, lattices + count);
  return CCMC_OK;
}

}  // extern "C"

int ccmc::batch_new(int cap, cudaStream_t stream, ccmc_batch **out) {
  if (!out || cap < 1) return CCMC_E_INVAL;
  *out = nullptr;
  ccmc_batch *b = new (std::nothrow) ccmc_batch();
  if (!b) return CCMC_E_NOMEM;
  b->cap = cap;
  const int count = cap;
  void *cuda_stream = (void *)stream;
  auto fail = [&](int code) {
    ccmc_batch_destroy(b);
    return code;
  };
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail(CCMC_E_CUDA);
    b->own_stream = true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int64_t max_words = optin / 4 - kResTableWords - 64;
  if (b->resident_max_sites / 4 > max_words) b->resident_max_sites = max_words * 4;
  if (cudaMalloc(&b->d_jobs, sizeof(JobDesc) * count) != cudaSuccess ||
      cudaMalloc(&b->d_multi, sizeof(MultiJob) * count) != cudaSuccess ||
      cudaMalloc(&b->d_queue, sizeof(int)) != cudaSuccess)
    return fail(CCMC_E_NOMEM);
  if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess)
    return fail(CCMC_E_CUDA);
  b->lat_ev.assign(count, nullptr);
  for (auto &e : b->lat_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return fail(CCMC_E_CUDA);
  *out = b;
  return CCMC_OK;
}

extern "C" {

int ccmc_batch_destroy(ccmc_batch *b) {
  if (!b) return CCMC_E_INVAL;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto &e : b->graphs)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  cudaFree(b->d_jobs);
  cudaFree(b->d_multi);
  cudaFree(b->d_queue);
  if (b->ev) cudaEventDestroy(b->ev);
  for (auto e : b->lat_ev)
    if (e) cudaEventDestroy(e);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return CCMC_OK;
}

int ccmc_batch_config(ccmc_batch *b, int resident_threads, int64_t resident_max_sites,
                      int ctas_per_sm, int max_threads_per_word) {
  if (!b) return CCMC_E_INVAL;
  if (resident_threads != 64 && resident_threads != 128 && resident_threads != 256 &&
      resident_threads != 512)
    return CCMC_E_INVAL;
  if (max_threads_per_word != 1 && max_threads_per_word != 2 && max_threads_per_word != 4)
    return CCMC_E_INVAL;
  if (resident_max_sites < 0 || ctas_per_sm < 1 || ctas_per_sm > 32) return CCMC_E_INVAL;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int64_t max_words = optin / 4 - kResTableWords - 64;
  if (resident_max_sites / 4 > max_words) return CCMC_E_INVAL;
  b->threads = resident_threads;
  b->resident_max_sites = resident_max_sites;
  b->ctas_per_sm = ctas_per_sm;
  b->max_tpw = max_threads_per_word;
  return CCMC_OK;
}

int ccmc_batch_sweep(ccmc_batch *b, const int64_t *nsweeps, const double *beta,
                     const double *Delta, const double *V, const double *J, int obs_every) {
  if (!b || !nsweeps || !beta || !Delta || !V || !J) return CCMC_E_INVAL;
  if (ccmc::fault_injected("launch")) return CCMC_E_CUDA;
  std::vector<int> every(b->lats.size(), obs_every);
  return ccmc::batch_run(b, b->lats, nsweeps, beta, Delta, V, J, every.data(), true);
}

int ccmc_batch_sync(ccmc_batch *b) {
  if (!b) return CCMC_E_INVAL;
  CK(cudaStreamSynchronize(b->stream));
  for (ccmc_lattice *h : b->lats) {
    const int rc = check_status(h);
    if (rc) return rc;
  }
  return CCMC_OK;
}

int ccmc_selftest_wait(uint32_t polls) {
  if (polls == 0 || polls > (1u << 24)) return CCMC_E_INVAL;
  int *d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return CCMC_E_NOMEM;
  int status = 0;
  int rc = CCMC_OK;
  if (cudaMemset(d, 0, sizeof(int)) != cudaSuccess ||
      ccmc::launch_wait_selftest(polls, d, 0) != cudaSuccess ||
      cudaMemcpy(&status, d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = CCMC_E_CUDA;
  cudaFree(d);
  if (rc) return rc;
  return status ? CCMC_E_TIMEOUT : CCMC_OK;
}

int ccmc_philox_device(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                       uint32_t k1, int64_t count, uint32_t *out) {
  if (!out || count < 0 || count > ((int64_t)1 << 28)) return CCMC_E_INVAL;
  if (count == 0) return CCMC_OK;
  uint32_t *d = nullptr;
  if (cudaMalloc(&d, sizeof(uint32_t) * 4 * count) != cudaSuccess) return CCMC_E_NOMEM;
  int rc = CCMC_OK;
  if (launch_philox(c0, c1, c2, c3, k0, k1, count, d, 0) != cudaSuccess ||
      cudaMemcpy(out, d, sizeof(uint32_t) * 4 * count, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = CCMC_E_CUDA;
  cudaFree(d);
  return rc;
}

}  // extern "C"
