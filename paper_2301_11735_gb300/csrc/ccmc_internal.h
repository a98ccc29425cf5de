// ccmc_internal.h -- library-internal types shared by the host API and the
// kernels (plain C++, no device code).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/ccmc.h"

struct ccmc_lattice;
struct ccmc_batch;

namespace ccmc {

constexpr uint32_t TAG_SCHED = 1u;    // phase schedule
constexpr uint32_t TAG_MOVE = 2u;     // per 8 pairs: a 16-bit field a pair
constexpr uint32_t TAG_SLOW = 3u;     // per pair: acceptance word, choice fallback
constexpr uint32_t TAG_FEISTEL = 4u;  // initial placement
constexpr uint32_t TAG_SIGN = 5u;     // initial spin signs

constexpr int kDB = 20;                 // |dBV|, |dBJ| <= 20 when Lx, Ly >= 4
constexpr int kNB = 2 * kDB + 1;        // 41
constexpr int kTableN = 3 * kNB * kNB;  // dQ in {-2, 0, 2}: 5043 thresholds

// Control block of a lattice (int64 words in device memory).
enum CtlSlot : int {
  kCtlPhaseBase = 0,  // global phase index of the next phase with offset 0
  kCtlObsCount = 1,   // records written to the ring so far
  kCtlTicket = 2,     // arrival counter of the recount's last-block reduction
  kCtlStatus = 3,     // device-side error flag
  kCtlLatest = 4,     // 8 words: the last recount record
  kCtlTileClaim = 12,  // 2 words: tile claims of the tile-staged phases of even
                       // and odd P (phase P's low 32 bits above the claim count)
  kCtlWords = 16
};

// Lattice geometry as seen by the kernels.
struct Geo {
  uint32_t *words;  // 16 classes x Cy rows x W words
  int64_t *ctl;     // control block
  int Lx, Ly, Cx, Cy, W;
  int64_t cstride;  // Cy * W words per class
  uint32_t k0, k1;  // Philox key = seed
  uint64_t rej;     // 2^64 mod (Lx Ly): Lemire rejection bound
};

// Per-lattice parameter tables in device memory (built on the host).
struct DevTables {
  uint16_t *thrT;   // kThrT: threshold levels T = floor(5461 thr / 2^32), 5461 for
                    // thr = 0xFFFFFFFF (fast path)
  uint32_t *trans;  // kMoveN x 2 words: move entries (see kMoveN), directly after thrT
  uint32_t *thr32;  // kTableN: full thresholds (exact path)
};

// The fast path's threshold level of a 32-bit threshold: a field's w = v / 12
// (in [0, 5461)) below it accepts, above it rejects, equal to it is a tie.
__host__ __device__ inline uint16_t threshold_level(uint32_t thr) {
  return thr == 0xFFFFFFFFu ? (uint16_t)5461 : (uint16_t)(((uint64_t)thr * 5461u) >> 32);
}

// Move entries: one uint2 per (r, near, pc), entry (2 r + near) * 16 + (pc ^ r), i.e.
// at byte offset 256 r + 128 near + 8 (pc ^ r) -- r the pair's choice field mod 12
// (12 is a multiple of both q-set sizes, 4 and 6), near whether the partner is a
// nearest neighbour, pc = 4 code_a + code_b the pair state.
constexpr int kTransN = 16 * 12;     // entries of one kind (far or near)
constexpr int kMoveN = 2 * kTransN;  // both kinds
constexpr int kThrT = (kTableN + 7) / 8 * 8;  // 16-bit levels, padded to 16 bytes

struct LaunchCfg {
  int phase_grid_cap = 152 * 3;  // one resident wave of phase_kernel (set at create)
  int tile_grid = 0;             // > 0: tile-staged phases, this many CTAs at most
  int tile_grid_small = 0;       // one wave of the compact tile kernel (16-bit tops)
};

// One lattice of a resident batch launch (device array, filled on the host).
struct JobDesc {
  Geo g;                    // the lattice in global memory
  const uint16_t *thrT;     // its tables
  const uint32_t *thr32;
  const uint32_t *trans;
  int64_t nsweeps;          // sweeps to run in this launch
  int64_t *ring;            // observable ring (records every obs_every sweeps)
  int64_t ring_cap;
  int64_t *hist;            // histograms (nullptr: none)
  int nbins;
  int obs_every;
  int max_tpw;              // threads a word: the most of 4, 2, 1 (at most max_tpw) that
                            // take a phase's words in one pass of the CTA, else 1
  int warp;                 // 1: run by one warp of a CTA, the lattice in that warp's
                            // share of the shared memory (the launch's warp_words)
};

// One lattice of a lock-step multi-lattice phase launch: CTAs
// [cta_begin, cta_begin + cta_count) of the grid work on it.
struct MultiJob {
  Geo g;
  const uint16_t *thrT;
  const uint32_t *thr32;
  const uint32_t *trans;
  int cta_begin, cta_count;
};

// Shared memory of the resident kernel besides the lattice words.
constexpr int kResTableWords = kThrT / 2 + 2 * kMoveN;

// Host-side table builders (ccmc_tables.cpp).
void build_thresholds(double beta, double Delta, double V, double J, uint32_t *thr32);
// Returns false if some entry could index outside the threshold table.
bool build_transitions(uint32_t *trans);

// Launchers (ccmc_kernels.cu).
cudaError_t launch_init(const Geo &g, int h, int64_t n_plus, int64_t n_minus, cudaStream_t s);
cudaError_t launch_phase(const Geo &g, const DevTables &t, int64_t p_off, const LaunchCfg &cfg,
                         cudaStream_t s);
int recount_grid(const Geo &g);
// CTAs of phase_kernel that fit the device at once (one wave).
int phase_resident_grid(bool aligned);
// Whether a lattice can take the tile-staged phase kernel, and its one wave.
bool tile_path_ok(const Geo &g);
int tile_resident_grid();
// One wave of the compact tile kernel (more CTAs per SM), 0 if unavailable.
int tile_resident_grid_small();
// One colour phase of every lattice in d_jobs (all aligned or all not).
cudaError_t launch_phase_multi(const MultiJob *d_jobs, int njobs, int grid, bool aligned,
                               int64_t p_off, cudaStream_t s);
// One tile-staged phase of every lattice in d_jobs (all take the tile path;
// their tables one staged block each, as launch_phase requires).
cudaError_t launch_phase_tile_multi(const MultiJob *d_jobs, int njobs, int grid, int64_t p_off,
                                    cudaStream_t s);
// Tiles of one tile-staged phase of lattice g.
int tile_count(const Geo &g);
cudaError_t launch_recount(const Geo &g, int64_t *partials, int64_t *ring, int64_t ring_cap,
                           int64_t *hist, int nbins, int64_t sweep_off, cudaStream_t s);
cudaError_t launch_advance(int64_t *ctl, int64_t phases, cudaStream_t s);
cudaError_t launch_set_ctl(int64_t *ctl, int64_t phase_base, cudaStream_t s);
cudaError_t launch_unpack(const Geo &g, uint8_t *out, cudaStream_t s);
cudaError_t launch_pack(const Geo &g, const uint8_t *in, int *bad, cudaStream_t s);
// Resident batch kernel: grid CTAs of `threads` threads take jobs from *queue
// (zeroed by the caller) until njobs are done; max_words bounds 16 Cy W of
// the jobs a whole CTA runs.  Jobs with `warp` set come last in d_jobs and
// have 16 Cy W <= resident_warp_words(threads, max_words).
cudaError_t launch_resident(const JobDesc *d_jobs, int njobs, int *d_queue, int grid, int threads,
                            int64_t max_words, cudaStream_t s);
// Words of one warp's share of a resident CTA's shared memory, and the
// resident CTAs of `threads` threads an SM holds at once.
int64_t resident_warp_words(int threads, int64_t max_words);
int resident_ctas_per_sm(int threads, int64_t max_words);
int64_t resident_smem_bytes(int64_t max_words);
cudaError_t launch_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                          uint32_t k1, int64_t count, uint32_t *out, cudaStream_t s);

// ccmc_lattice_create without the final wait (wait false): the lattice's
// memory, tables and zeroed state are queued on its stream.
int lattice_new(int Lx, int Ly, void *cuda_stream, int64_t obs_capacity, bool wait,
                ccmc_lattice **out);

// ccmc_init_counts / ccmc_init_constrained without the final wait.
int init_counts_async(ccmc_lattice *h, uint64_t seed, int64_t n_plus, int64_t n_minus);
int init_constrained_async(ccmc_lattice *h, uint64_t seed, double n, double charged_frac);

// What a finished simulation reports, copied to pinned host memory by work
// queued on its stream (then `ready` recorded there): rec (8 int64), the
// latest exact recount (its word 0 is replaced by the sweeps done); status,
// the device-side error flag; count and ring (8 int64 a record, ring_cap
// records), the observable ring, when ring is not null; state (Lx Ly bytes),
// the site codes, when state is not null.
int export_async(ccmc_lattice *h, int64_t *rec, int64_t *status, int64_t *count, int64_t *ring,
                 uint8_t *state, cudaEvent_t ready);
// The observables of a record exported by export_async (its E from the
// lattice's parameters), and the records of an exported ring, oldest first.
void obs_of_record(const ccmc_lattice *h, const int64_t *rec, ccmc_obs *out);
int64_t series_of_ring(const ccmc_lattice *h, const int64_t *ring, int64_t count, ccmc_obs *out,
                       int64_t cap);
int64_t ring_capacity(const ccmc_lattice *h);
cudaStream_t lattice_stream(const ccmc_lattice *h);

// A batch with no fixed members, room for `cap` lattices, on `stream`.
int batch_new(int cap, cudaStream_t stream, ccmc_batch **out);

// Sweep a list of lattices (at most the batch's capacity) with per-lattice
// sweeps, parameters and observable intervals through the batch machinery.
// lockstep: large lattices at the same position may share phase launches
// (the launches are captured once per group and replayed, so the list should
// be the same on every call).
int batch_run(ccmc_batch *b, const std::vector<ccmc_lattice *> &lats, const int64_t *nsweeps,
              const double *beta, const double *Delta, const double *V, const double *J,
              const int *obs_every, bool lockstep);

}  // namespace ccmc
