/*
 * ccmc_oracle.h -- the CPU oracle's own interface.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package's smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  The CUDA library has
 * its own, separately written implementation of every step below; the two
 * share no header, helper, table or constant generator.
 *
 * Model (Budrin et al., "The Parallel Monte Carlo Algorithm Implementation on
 * GPU for the Systems with an Ising Hamiltonian under the Condition of a
 * Constant Charge Density", Sec. 2.1, Eqs. (1)-(3)):
 *   an Lx x Ly periodic square lattice, every site in one of four states,
 *   stored one byte per site, site (x, y) at index y*Lx + x:
 *     0 : magnetic, s = +1/2 (sigma = +1, S = 0)
 *     1 : magnetic, s = -1/2 (sigma = -1, S = 0)
 *     2 : charge S = +1      (sigma = 0)
 *     3 : charge S = -1      (sigma = 0)
 *   E = Delta * sum_i S_i^2 + V * sum_<ij> S_i S_j + (J/4) * sum_<ij> sigma_i sigma_j
 *   with every bond counted once (the right and the down bond of each site),
 *   and the constraint sum_i S_i = n N (Eq. 2).
 */
#ifndef CCMC_ORACLE_H
#define CCMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Counter-space tags (fourth counter word) of the independent random streams. */
#define ORACLE_TAG_SCHED 1u   /* phase schedule (class a0 and offset r)     */
#define ORACLE_TAG_MOVE 2u    /* per 8 pairs: a 16-bit field each          */
#define ORACLE_TAG_SLOW 3u    /* per pair: acceptance word, choice fallback */
#define ORACLE_TAG_FEISTEL 4u /* initial-state placement permutation        */
#define ORACLE_TAG_SIGN 5u    /* initial spin signs of magnetic sites       */
#define ORACLE_TAG_SEQ 6u     /* sequential random-pair mode: pair + field  */
#define ORACLE_TAG_SEQSLOW 7u /* sequential random-pair mode: slow words    */
#define ORACLE_TAG_NN 8u      /* short-range pair mode: pair + field       */
#define ORACLE_TAG_NNSLOW 9u  /* short-range pair mode: slow words         */
#define ORACLE_TAG_MAP 10u    /* paper maps: random-marking site draws      */
#define ORACLE_TAG_MAPMOVE 11u /* paper maps: per pair, the 16-bit field    */
#define ORACLE_TAG_MAPSLOW 12u /* paper maps: per pair, slow words          */
#define ORACLE_TAG_PENALTY 13u /* penalty-function baseline: single sites   */

/* Threshold table: dQ in [-2,2], dBV and dBJ in [-ORACLE_DB, ORACLE_DB]. */
#define ORACLE_DB 24
#define ORACLE_NB (2 * ORACLE_DB + 1)
#define ORACLE_TABLE_SIZE (5 * ORACLE_NB * ORACLE_NB)

/* Observable record: sweeps_done, Nc, BV, BJ, M, M_stag, S_sum, S_stag. */
#define ORACLE_REC 8

/* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Counters (ctr[0] + i mod 2^32, ctr[1], ctr[2], ctr[3]) for i < count, in order. */
void oracle_philox_block(const uint32_t ctr[4], const uint32_t key[2], int64_t count,
                         uint32_t *out);

/* Charge counts from (n, c): Q = llround(n N), C = max(llround(c N), |Q|),
 * C += 1 when C - Q is odd; N+ = (C + Q)/2, N- = (C - Q)/2.  Returns 0, or -1
 * when C > N or the inputs are not finite. */
int oracle_charge_counts(int64_t N, double n, double c, int64_t *Q, int64_t *n_plus,
                         int64_t *n_minus);

/* Rank of site i (0 <= i < N) under the seeded Feistel permutation of [0, N). */
int64_t oracle_feistel_rank(uint64_t seed, int64_t N, int64_t i);

/* Exact-count initial state: rank < N+ -> S=+1, rank < N+ + N- -> S=-1,
 * otherwise magnetic with a seeded sign.  Returns 0 or -1 on bad counts. */
int oracle_init_counts(int Lx, int Ly, uint64_t seed, int64_t n_plus, int64_t n_minus,
                       uint8_t *st);

/* Acceptance thresholds, ORACLE_TABLE_SIZE entries. */
void oracle_threshold_table(double beta, double Delta, double V, double J, uint32_t *table);
int oracle_table_index(int dQ, int dBV, int dBJ);

/* 1 if the offset (rx, ry) is in the allowed set R of the colour schedule. */
int oracle_offset_allowed(int Lx, int Ly, int rx, int ry);
/* Schedule of global phase P: class (a0x, a0y) and offset (rx, ry). */
void oracle_schedule(int Lx, int Ly, uint64_t seed, uint64_t P, int *a0x, int *a0y, int *rx,
                     int *ry);

/* Integer energy-term changes of moving sites a, b to codes na, nb. */
void oracle_pair_delta(const uint8_t *st, int Lx, int Ly, int a, int b, int na, int nb,
                       int out[3]);

/* One coupled-pair Metropolis move on sites a and b.  The low 16 bits of F
 * are the pair's random field (choice and the acceptance word's top part,
 * see ccmc_oracle.c); the SLOW words are drawn from Philox(key, slow_ctr)
 * when needed.  Returns 1 if the lattice changed. */
int oracle_pair_move(uint8_t *st, int Lx, int Ly, int a, int b, uint32_t F,
                     const uint32_t key[2], const uint32_t slow_ctr[4], const uint32_t *table);

/* Full recount: out = {Nc, BV, BJ, M, M_stag, S_sum, S_stag}. */
void oracle_recount(const uint8_t *st, int Lx, int Ly, int64_t out[7]);

/* One colour phase (global phase index P). */
void oracle_phase(uint8_t *st, int Lx, int Ly, uint64_t seed, uint64_t P, const uint32_t *table);

/* nsweeps colour-ordered sweeps starting at sweep index sweep0; a record is
 * written after every obs_every-th sweep (obs_every <= 0: none). */
int64_t oracle_sweeps(uint8_t *st, int Lx, int Ly, uint64_t seed, int64_t sweep0,
                      int64_t nsweeps, double beta, double Delta, double V, double J,
                      int obs_every, int64_t *records);

/* Sequential random-pair mode: floor(N/2) moves per sweep, each on a uniform
 * ordered pair a != b.  Any Lx, Ly >= 2. */
int64_t oracle_sequential_sweeps(uint8_t *st, int Lx, int Ly, uint64_t seed, int64_t sweep0,
                                 int64_t nsweeps, double beta, double Delta, double V, double J,
                                 int obs_every, int64_t *records);
/* Short-range pair mode (Sec. 3.2's abandoned first version): partner b is a
 * uniformly chosen nearest neighbour of a uniformly chosen a; N/2 moves per
 * sweep.  A negative control for tests, not a method of the library. */
int64_t oracle_neighbour_sweeps(uint8_t *st, int Lx, int Ly, uint64_t seed, int64_t sweep0,
                                int64_t nsweeps, double beta, double Delta, double V, double J,
                                int obs_every, int64_t *records);

/* Paper-faithful maps (Sec. 3.2): P = max(1, floor(N/10)) non-interacting
 * pairs built by random marking; map m's pairs as site indices y*Lx + x,
 * a then b, into pairs[2P].  Returns 0, or -1 if memory runs out. */
int64_t oracle_map_size(int Lx, int Ly);
int oracle_map_build(int Lx, int Ly, uint64_t seed, int64_t m, int32_t *pairs);

/* Applies maps map0 .. map0 + nmaps - 1 in turn, each pair of a map once (in
 * list order; the pairs do not interact).  Records after map m when
 * (m + 1) % obs_every == 0, with sweeps_done = m + 1 (maps done). */
int64_t oracle_map_sweeps(uint8_t *st, int Lx, int Ly, uint64_t seed, int64_t map0, int64_t nmaps,
                          double beta, double Delta, double V, double J, int obs_every,
                          int64_t *records);

/* Change of the integer energy terms (dNc, dBV, dBJ) of Eq. (3) when site a
 * alone goes from its current code to code nc: dNc = S'^2 - S^2, dBV = dS x
 * (sum of S over a's four neighbours), dBJ = dsigma x (sum of sigma over them),
 * each neighbour counted once per bond (twice on a 2-wide torus). */
void oracle_site_delta(const uint8_t *st, int Lx, int Ly, int a, int nc, int out[3]);

/* Penalty-function baseline (Sec. 2.2): single-site Metropolis with the extra
 * energy -mu sum S, mu <- mu + kappa (nN - sum S)/N after every sweep (the
 * adjustment rule is this oracle's reading).  *mu is read and updated.
 * Pinned by its single-site energy change against a full recount, and at
 * kappa = 0 (fixed mu) by the exact grand-canonical averages of 3 x 3 and
 * 4 x 2 tori; the adjustment rule itself has no exact reference.  It has no
 * GPU counterpart. */
int64_t oracle_penalty_sweeps(uint8_t *st, int Lx, int Ly, uint64_t seed, int64_t sweep0,
                              int64_t nsweeps, double beta, double Delta, double V, double J,
                              double n, double *mu, double kappa, int obs_every,
                              int64_t *records, double *mu_trace);

/* Exact enumeration of the states with sum S = Q (N <= 16): histogram over
 * (Nc, BV, BJ) with bins [Nc][BV + 2N][BJ + 2N] of size (N+1) x (4N+1) x (4N+1);
 * count, and integer sums of M^2, |M|, M_stag^2 per bin (Lx <= 4).  Returns the
 * number of states, or -1 for an unsupported shape. */
int64_t oracle_enumerate(int Lx, int Ly, int Q, int64_t *count, int64_t *m2, int64_t *mabs,
                         int64_t *mstag2);

#ifdef __cplusplus
}
#endif
#endif
