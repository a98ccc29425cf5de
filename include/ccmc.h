/*
 * ccmc.h -- C ABI of libccmc: the charge-conserving coupled-pair Metropolis
 * sweep of Budrin et al. ("The Parallel Monte Carlo Algorithm Implementation on
 * GPU for the Systems with an Ising Hamiltonian under the Condition of a
 * Constant Charge Density"), on one NVIDIA GB300 (sm_103a).
 *
 * Model (Sec. 2.1).  An Lx x Ly square lattice with periodic edges; each site
 * is magnetic (S = 0, s = +-1/2, sigma = 2 s = +-1) or charged (S = +-1).
 *   E = Delta sum_i S_i^2 + V sum_<ij> S_i S_j + (J/4) sum_<ij> sigma_i sigma_j
 * (Eq. 3), every bond counted once, under the constraint sum_i S_i = n N
 * (Eq. 2), which every move of the library keeps exactly.
 *
 * Site codes used by every host buffer of this API (one byte per site, site
 * (x, y) at index y * Lx + x):
 *   0 : s = +1/2    1 : s = -1/2    2 : S = +1    3 : S = -1
 *
 * Conventions.
 *   - Return value: CCMC_OK (0) or a negative CCMC_E_* code; ccmc_strerror()
 *     names it.  A failed call leaves the handle usable unless it returns
 *     CCMC_E_CUDA, after which only ccmc_*_destroy is meaningful.
 *   - Memory: the library owns all device memory of a handle (allocated in
 *     *_create, freed in *_destroy).  The caller owns every host buffer it
 *     passes; the library never keeps a host pointer after a call returns.
 *   - Streams: every device operation of a handle is issued on the stream given
 *     at creation (NULL: a stream the library creates).  Calls that return host
 *     data synchronise that stream; ccmc_sweep returns as soon as the work is
 *     queued.  A handle must not be used from two host threads at once.
 *   - Lx and Ly must be multiples of 4 and at least 4 (the colour schedule
 *     works on residue classes mod 4), and Lx * Ly <= 2^30.
 */
#ifndef CCMC_H
#define CCMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CCMC_OK 0
#define CCMC_E_INVAL (-1)   /* bad argument: shape, counts, NaN parameter, ... */
#define CCMC_E_NOMEM (-2)   /* device or host allocation failed                */
#define CCMC_E_CUDA (-3)    /* a CUDA runtime call or kernel launch failed     */
#define CCMC_E_TIMEOUT (-4) /* a bounded device wait gave up                   */
#define CCMC_E_BUDGET (-5)  /* admission refused: the memory budget is full    */
#define CCMC_E_STATE (-6)   /* call out of order (e.g. sweep before init)      */
#define CCMC_E_NOTFOUND (-7)/* unknown ticket or handle                        */
#define CCMC_PENDING 1      /* ccmc_server_poll: the request has not finished   */

/* Observables after a sweep (Sec. 2.2 and Eq. 3).  All integer terms are exact
 * recounts of the lattice: Nc = sum S^2, BV = sum_bonds S S, BJ = sum_bonds
 * sigma sigma, M = sum sigma, M_stag = sum (-1)^(x+y) sigma, S_sum = sum S
 * (always n N), S_stag = sum (-1)^(x+y) S.  E = Delta Nc + V BV + (J/4) BJ,
 * evaluated in FP64 on the host with the parameters of the last sweep. */
typedef struct {
  int64_t sweeps_done, Nc, BV, BJ, M, M_stag, S_sum, S_stag;
  double E;
} ccmc_obs;

typedef struct ccmc_lattice ccmc_lattice;

/* Allocate an Lx x Ly lattice on the current CUDA device (Lx, Ly multiples of
 * 4, at least 4, Lx Ly <= 2^30).  cuda_stream is a cudaStream_t (NULL: the
 * library creates one).  The observable ring holds the last obs_capacity
 * records (<= 0: 4096).  Device memory comes from a stream-ordered pool the
 * library keeps per device (allocated and freed in order on the lattice's
 * stream, cached for reuse until the process exits), so creating and
 * destroying lattices never synchronises the device.  Returns once the
 * lattice is ready.  Errors: E_INVAL, E_NOMEM, E_CUDA. */
int ccmc_lattice_create(int Lx, int Ly, void *cuda_stream, int64_t obs_capacity,
                        ccmc_lattice **out);
/* Waits for the work queued on the lattice's stream, then releases it. */
int ccmc_lattice_destroy(ccmc_lattice *h);

/* Constrained initial state (Sec. 3.1, stage 1).  Q = llround(n N);
 * C = max(llround(charged_frac N), |Q|), plus one when C - Q is odd;
 * N+ = (C + Q)/2 sites get S = +1 and N- = (C - Q)/2 get S = -1, placed by a
 * seeded Feistel permutation of the site indices; the remaining sites are
 * magnetic with seeded random signs.  charged_frac < 0 means 0.3.  Resets the
 * sweep counter and the observable ring.  Errors: E_INVAL (C > N, NaN). */
int ccmc_init_constrained(ccmc_lattice *h, uint64_t seed, double n, double charged_frac);
/* Same placement with explicit counts N+ = n_plus, N- = n_minus. */
int ccmc_init_counts(ccmc_lattice *h, uint64_t seed, int64_t n_plus, int64_t n_minus);

/* Run nsweeps sweeps of the coupled-pair Metropolis algorithm (Sec. 3.1-3.2)
 * at inverse temperature beta (k = 1) with couplings Delta, V, J.  A sweep is 8
 * colour phases; phase P (counted from the initial state) updates every pair
 * (a, a + r) with a = a0 (mod 4) for a class a0 and an offset r drawn from the
 * counter-based generator, so no two pairs of a phase interact (the paper's
 * "map").  After every sweep whose 1-based index is a multiple of obs_every
 * (<= 0: never) the lattice is recounted into the observable ring.  Results
 * depend only on (seed, sweep index, site), not on launch shape.
 * Errors: E_INVAL (beta < 0 or NaN, non-finite couplings), E_STATE. */
int ccmc_sweep(ccmc_lattice *h, int64_t nsweeps, double beta, double Delta, double V, double J,
               int obs_every);

/* Run nphases colour phases, each launched on its own.  One phase is the
 * paper's "step" (Sec. 5: the processing of one map); a sweep is 8 phases, and
 * ccmc_sweep(h, s, ...) equals ccmc_phases(h, 8 s, ...) without observables.
 * The phase counter continues across both calls, so they can be mixed; the
 * sweep count of a record is the completed phases / 8.  Errors as ccmc_sweep. */
int ccmc_phases(ccmc_lattice *h, int64_t nphases, double beta, double Delta, double V, double J);

/* ---- Batches of replicas (several independent lattices of uneven size). ----
 * A batch groups existing, initialised lattices (each with its own size,
 * seed and parameters; Sec. 3.2 runs "several copies of the lattice").
 * ccmc_batch_sweep advances lattice i by nsweeps[i] sweeps at (beta[i],
 * Delta[i], V[i], J[i]).  Lattices of at most resident_max_sites sites run
 * together in one persistent launch on the batch stream: each CTA keeps a
 * whole lattice and its tables in shared memory and runs all its sweeps,
 * taking lattices from a work queue largest first.  Larger lattices run the
 * per-phase path at the same time: eight or more of them at the same sweep
 * count with fewer than 16384 class-row words a phase (below 2048^2) advance
 * in lock step, one launch per phase for all of them on the batch stream; the
 * others each on their own stream.  Every lattice ends in
 * exactly the state ccmc_sweep would give it (same random streams), and its
 * observable ring gets the same records.  Ordering: the batch waits for work
 * already queued on each lattice's stream, and each lattice's stream waits for
 * the batch.  Errors: E_INVAL, E_STATE (a lattice not initialised, or left in
 * the middle of a sweep by ccmc_phases). */
typedef struct ccmc_batch ccmc_batch;
int ccmc_batch_create(int count, ccmc_lattice *const *lattices, void *cuda_stream,
                      ccmc_batch **out);
int ccmc_batch_destroy(ccmc_batch *b);
/* Launch shape of the resident launch (autotuner knobs; results do not depend
 * on them): threads per CTA (64, 128, 256 or 512), the largest lattice (in
 * sites) kept in shared memory, CTAs per SM of the persistent grid, and the
 * most threads that share one packed word (16 pairs) of a lattice: 1, 2 or 4
 * (each lattice takes the most, up to this, that still covers a phase's words
 * in one pass of its CTA).  Errors: E_INVAL (a value out of range, or a
 * resident limit beyond the device's shared memory). */
int ccmc_batch_config(ccmc_batch *b, int resident_threads, int64_t resident_max_sites,
                      int ctas_per_sm, int max_threads_per_word);
int ccmc_batch_sweep(ccmc_batch *b, const int64_t *nsweeps, const double *beta,
                     const double *Delta, const double *V, const double *J, int obs_every);
/* Wait for the batch stream and every member's stream; reports device errors. */
int ccmc_batch_sync(ccmc_batch *b);

/* ---- Serving: a continuous-batching request loop of independent runs. ----
 * A request is one simulation: an Lx x Ly lattice initialised as by
 * ccmc_init_constrained(seed, n, charged_frac), then nsweeps sweeps at
 * (beta, Delta, V, J), recording observables every obs_every sweeps (0: none).
 * state_out, if not NULL, is a host buffer of Lx * Ly bytes that receives the
 * final lattice; it must stay valid until the request finishes.  Requests are
 * admitted first come first served while fewer than max_active are running and
 * their device memory fits the budget (a request that can never fit finishes
 * with E_BUDGET).  Admitted simulations stay resident on the GPU; a scheduler
 * thread advances all of them in slices of about slice_ms (each slice is one
 * batched launch, ccmc_batch_*), so requests that arrive while others run
 * join at the next slice and leave as soon as they are done.  Results equal
 * those of running each request alone.  Times are seconds since the server
 * started (host clock). */
typedef struct {
  int Lx, Ly;
  uint64_t seed;
  double n, charged_frac;
  int64_t nsweeps;
  double beta, Delta, V, J;
  int obs_every;
  uint8_t *state_out;
} ccmc_request;

typedef struct {
  int status;            /* CCMC_OK or the error that ended the request */
  ccmc_obs final_obs;    /* observables after the last sweep            */
  int64_t site_updates;  /* Lx * Ly * nsweeps                           */
  double submit_s, start_s, done_s;
} ccmc_result;

typedef struct {
  int64_t submitted, queued, active, completed, rejected, failed, slices, site_updates,
      bytes_in_use;
} ccmc_server_stats;

typedef struct ccmc_server ccmc_server;
int ccmc_server_start(size_t hbm_budget_bytes, int max_active, double slice_ms,
                      ccmc_server **out);
int ccmc_server_submit(ccmc_server *s, const ccmc_request *req, uint64_t *ticket);
/* CCMC_OK and *out filled once the request finished, CCMC_PENDING before,
 * E_NOTFOUND for an unknown (or released) ticket. */
int ccmc_server_poll(ccmc_server *s, uint64_t ticket, ccmc_result *out);
/* Block up to timeout_s seconds for the request; E_TIMEOUT if it is not done. */
int ccmc_server_wait(ccmc_server *s, uint64_t ticket, ccmc_result *out, double timeout_s);
/* Observable records of a finished request (as ccmc_obs_series). */
int ccmc_server_series(ccmc_server *s, uint64_t ticket, ccmc_obs *out, int64_t cap,
                       int64_t *n_written);
/* Forget a finished request's result. */
int ccmc_server_release(ccmc_server *s, uint64_t ticket);
int ccmc_server_stats_get(ccmc_server *s, ccmc_server_stats *out);
/* Stop accepting requests, finish every queued and running one, then free
 * everything. */
int ccmc_server_stop(ccmc_server *s);

/* Recount the current lattice and return its observables (synchronises). */
int ccmc_observables(ccmc_lattice *h, ccmc_obs *out);
/* Copy the ring's records, oldest first, into out[0 .. cap); *n_written gets
 * their number.  Records whose index fell out of the ring are lost. */
int ccmc_obs_series(ccmc_lattice *h, ccmc_obs *out, int64_t cap, int64_t *n_written);

/* Histograms (per recount in the ring) of M, M_stag and S_stag over nbins
 * equal bins of [-N, N]: bin = (x + N) nbins / (2N + 1).  Enabling clears
 * them; out receives 3 * nbins int64 (M, M_stag, S_stag). */
int ccmc_hist_enable(ccmc_lattice *h, int nbins);
int ccmc_hist_get(ccmc_lattice *h, int64_t *out);

/* Lattice state as N bytes of site codes (synchronises). */
int ccmc_get_state(ccmc_lattice *h, uint8_t *host_out);
/* Load a state (checkpoint / resume): host_in holds N site codes; seed and
 * sweeps_done fix the random stream, so resuming reproduces the trajectory
 * bit for bit.  Errors: E_INVAL (code > 3). */
int ccmc_set_state(ccmc_lattice *h, const uint8_t *host_in, uint64_t seed, int64_t sweeps_done);

/* Compact state, 2 bits a site in row-major order: site i = y * Lx + x is
 * the code (as in ccmc_get_state) at bits 2 (i mod 4) .. 2 (i mod 4) + 1 of
 * byte i / 4; Lx * Ly / 4 bytes (Lx is a multiple of 4, so each row is Lx / 4
 * whole bytes).  A quarter of the byte-per-site form: for checkpoints and for
 * streaming lattices in and out of the GPU.
 *
 * ccmc_get_state_packed: host-returning (synchronises the lattice's stream).
 * ccmc_set_state_packed: stream-ordered, it returns once the work is queued
 * on the lattice's stream; the copy reads host_in later, so the buffer must
 * stay valid and unchanged until the next call that synchronises the lattice
 * (ccmc_sync, ccmc_observables, ccmc_get_state...).  Every byte is a valid
 * input (all four 2-bit codes are states).  seed and sweeps_done as in
 * ccmc_set_state.  Errors: E_INVAL, E_STATE (get before any state), E_NOMEM,
 * E_CUDA. */
int ccmc_get_state_packed(ccmc_lattice *h, uint8_t *host_out);
int ccmc_set_state_packed(ccmc_lattice *h, const uint8_t *host_in, uint64_t seed,
                          int64_t sweeps_done);

/* Block until the handle's queued work is done; reports a device-side error. */
int ccmc_sync(ccmc_lattice *h);

/* Observables of a lattice the caller keeps in device memory, computed without
 * allocating anything -- for callers that cannot let a library allocate device
 * memory during the call (a server that reserved its whole memory budget up
 * front, or a latency-critical path that must not pay for cudaMalloc/cudaFree).
 * The paper has no counterpart; it is a service of this library.
 *   d_state: Lx * Ly site codes (device memory, site (x, y) at y * Lx + x);
 *   d_out:   7 int64 in device memory, receives Nc, BV, BJ, M, M_stag, S_sum,
 *            S_stag of Eq. 3 by definition: the 2 Lx Ly right and down bonds
 *            of the torus (on a 2-wide torus both bonds joining the same two
 *            sites count), M_stag and S_stag with the sign of (x + y) mod 2.
 *            For the shapes ccmc_lattice_create accepts these are exactly
 *            what ccmc_observables reports; other shapes (odd sides, 2-wide
 *            tori) are accepted too.
 * The reduction's scratch is a fixed static device array of 64 KB (1024 block
 * partials and a counter) that every GPU loading the library holds until exit;
 * lattices of any size up to Lx * Ly = 2^30 fit it (larger: E_INVAL), and
 * Lx, Ly >= 2.  The first call on a device looks up that array's address with
 * the device current and keeps it for the life of the process; make that
 * first call before any stream capture, and do not call this function on a
 * device after resetting it (cudaDeviceReset) in the same process: the kept
 * address then belongs to the destroyed context.  The work
 * is queued on cuda_stream (NULL: the legacy default stream); synchronise before
 * reading d_out.  All calls share the one array, so calls that overlap on the
 * GPU (different streams, or another host thread) race and must not be issued.
 * Errors: E_INVAL (null pointer or size), E_CUDA. */
int ccmc_recount_noalloc(const uint8_t *d_state, int Lx, int Ly, int64_t *d_out,
                         void *cuda_stream);

/* Host-only: the acceptance thresholds the sweep uses (Sec. 3.1, "otherwise
 * the classical Metropolis algorithm"), for dQ in {-2, 0, 2} and dBV, dBJ in
 * [-20, 20]: out[((dQ + 2)/2 * 41 + dBV + 20) * 41 + dBJ + 20] =
 * 0xFFFFFFFF if dE <= 0, else min(floor(2^32 exp(-beta dE)), 0xFFFFFFFE), with
 * dE = Delta dQ + V dBV + (J/4) dBJ in FP64.  A move is accepted iff its
 * threshold is 0xFFFFFFFF or a uniform 32-bit word is below it.  out holds
 * 5043 entries.  No GPU needed. */
int ccmc_threshold_table(double beta, double Delta, double V, double J, uint32_t *out);

/* Diagnostic (the paper has no counterpart): the bounded-wait self-test.  One
 * CTA waits on a device barrier that nothing completes, giving up after
 * `polls` polls (1 .. 2^24), records the timeout and returns, as every wait of
 * the phase kernels does; the call then returns CCMC_E_TIMEOUT and the CUDA
 * context stays usable.  Errors: E_INVAL (polls out of range), E_NOMEM,
 * E_CUDA.  Host-side failures can be injected with the environment variable
 * CCMC_FAULT (comma-separated): "alloc" makes ccmc_lattice_create and
 * ccmc_batch_create return E_NOMEM before allocating anything, "launch" makes
 * ccmc_sweep, ccmc_phases and ccmc_batch_sweep return E_CUDA before queuing
 * anything (the handle stays usable), "admit" makes the server refuse every
 * request at admission (result status E_BUDGET). */
int ccmc_selftest_wait(uint32_t polls);

/* Diagnostic: Philox4x32-10 on the device for counters (c0 + i mod 2^32, c1,
 * c2, c3), i < count, key (k0, k1); out receives 4 * count words (host buffer
 * owned by the caller), counter by counter.  Synchronous on the default stream.
 * Errors: E_INVAL (out NULL, count < 0 or count > 2^28), E_NOMEM, E_CUDA. */
int ccmc_philox_device(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                       uint32_t k1, int64_t count, uint32_t *out);

/* Diagnostics (the paper has no counterpart): measured read bandwidth of the
 * current device's on-chip memories, the peaks against which the shared-memory
 * and L2 paths' rooflines are stated.  ccmc_peak_smem_read: every SM's
 * resident CTAs stream conflict-free 16-byte reads of their own shared-memory
 * buffer (32 KB each); ccmc_peak_l2_read: all SMs stream 16-byte reads that
 * bypass L1 over a device buffer of buffer_bytes (1 MiB .. 1 GiB; pick one
 * that L2 holds), after a pass that brings it into L2.  Each times one launch
 * with CUDA events after a warm-up launch, synchronously on the legacy default
 * stream, and writes bytes per second.  Errors: E_INVAL (null pointer, size
 * out of range), E_NOMEM, E_CUDA. */
int ccmc_peak_smem_read(double *bytes_per_s);
int ccmc_peak_l2_read(int64_t buffer_bytes, double *bytes_per_s);

/* ---- Paper-faithful map mode (Sec. 3.2, the algorithm for building a map) --
 * The paper's own parallel scheme: maps of non-interacting pairs built on the
 * host by random marking, copied to the GPU and processed one after another,
 * each pair of a map by its own thread.  ccmc_sweep's colour phases replace it
 * in this library; the mode is kept to compare both (statistics, and the cost
 * of host generation plus transfer).
 *
 * A map of an Lx x Ly lattice holds P = max(1, floor(Lx Ly / 10)) pairs.  It is
 * built with an array of N flags, all clear: draw a site until it is unmarked
 * and mark it (a), the same for b (b may be a neighbour of a), append (a, b),
 * mark the four nearest neighbours of a and of b, and repeat until P pairs are
 * listed.  Draw d of map m uses words 2 (d mod 2) and 2 (d mod 2) + 1 of
 * Philox4x32-10(seed; d / 2, m_lo, m_hi, 10) as a 64-bit x: the site is the
 * high half of x * N, redrawn when the low half is below 2^64 mod N. */

/* Pairs per map, max(1, floor(Lx Ly / 10)); E_INVAL if Lx or Ly < 2. */
int64_t ccmc_map_size(int Lx, int Ly);

/* Host-only (no GPU needed): builds maps map0 .. map0 + nmaps - 1 for the
 * given seed into pairs_out, caller-owned, 2 * P * nmaps int32: for each pair
 * the site indices y * Lx + x of a, then b; map k starts at pairs_out + 2 P k.
 * nthreads host threads build maps in parallel (<= 0: one per core); the
 * result does not depend on it.  Lx, Ly >= 2, Lx * Ly <= 2^31.
 * Errors: E_INVAL, E_NOMEM. */
int ccmc_maps_build(int Lx, int Ly, uint64_t seed, int64_t map0, int64_t nmaps,
                    int32_t *pairs_out, int nthreads);

/* Applies maps map0 .. map0 + nmaps - 1 (host memory, laid out as
 * ccmc_maps_build writes them for this lattice's shape) to the lattice at
 * (beta, Delta, V, J): the pairs are copied into device memory the lattice
 * owns and one kernel per map makes the coupled-pair move of Sec. 3.1 for
 * every pair of the map.  Pair p of map m draws its move word from
 * Philox4x32-10(seed; p, m_lo, m_hi, 11) and, when the choice field is >= 65532
 * or the acceptance needs the low half, its slow words from (p, m_lo, m_hi,
 * 12), with the choice and acceptance rules of ccmc_sweep; the seed is the
 * lattice's.  Every index must lie in [0, Lx Ly) (checked: E_INVAL); maps that
 * do not come from ccmc_maps_build may break the sampling but not memory
 * safety.  The work is queued on the lattice's stream; the call returns once
 * `pairs` has been copied.  The colour-phase position is unchanged; read the
 * result with ccmc_observables or ccmc_get_state.
 * Errors: E_INVAL, E_STATE (not initialised), E_NOMEM, E_CUDA. */
int ccmc_map_apply(ccmc_lattice *h, const int32_t *pairs, int64_t map0, int64_t nmaps,
                   double beta, double Delta, double V, double J);

const char *ccmc_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
