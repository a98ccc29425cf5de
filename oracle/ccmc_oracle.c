/*
 * ccmc_oracle.c -- plain, single-threaded CPU oracle for the charge-conserving
 * coupled-pair Metropolis method (Budrin et al., Sec. 3).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package's smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  It shares nothing with
 * the CUDA library: the library's Philox, initial state, threshold table,
 * schedule, move and recount are written separately and must agree with this
 * file bit for bit.
 *
 * Lattice: one byte per site, site (x, y) at y*Lx + x, codes
 *   0: s=+1/2 (sigma=+1, S=0)   1: s=-1/2 (sigma=-1, S=0)
 *   2: S=+1                     3: S=-1
 * Every floating-point step is written out in the order it is evaluated; the
 * file is compiled with -ffp-contract=off.
 */
#include "ccmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10.  Round: multiply words 0 and 2 by the two Philox multipliers,
 * swap the halves across the pairs and mix in the key; the key is advanced by
 * the two Weyl constants after every round (Salmon et al., SC'11, Sec. 4). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

/* A block of counters (ctr[0] + i mod 2^32, ctr[1], ctr[2], ctr[3]), i < count:
 * out receives 4 * count words, one call of the generator each. */
void oracle_philox_block(const uint32_t ctr[4], const uint32_t key[2], int64_t count,
                         uint32_t *out) {
  for (int64_t i = 0; i < count; ++i) {
    const uint32_t c[4] = {ctr[0] + (uint32_t)i, ctr[1], ctr[2], ctr[3]};
    oracle_philox4x32_10(c, key, out + 4 * i);
  }
}

static void seed_key(uint64_t seed, uint32_t key[2]) {
  key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(seed >> 32);
}

/* ------------------------------------------------------------------------ */
/* Site values (Sec. 2.1): charge S and sigma = 2 (1 - S^2) s. */
static const int CODE_S[4] = {0, 0, 1, -1};
static const int CODE_SIGMA[4] = {1, -1, 0, 0};

/* Two-site configurations for each pair charge q, in the order the paper lists
 * them (Sec. 3.1): (S_a or s_a, S_b or s_b) as codes (a, b). */
static const uint8_t SET_QP1[4][2] = {{2, 0}, {2, 1}, {0, 2}, {1, 2}};
static const uint8_t SET_QM1[4][2] = {{3, 0}, {3, 1}, {0, 3}, {1, 3}};
static const uint8_t SET_Q0[6][2] = {{2, 3}, {3, 2}, {0, 0}, {1, 1}, {0, 1}, {1, 0}};

/* ------------------------------------------------------------------------ */
/* Initial state (Sec. 3.1, stage 1: a configuration with the given charge). */
int oracle_charge_counts(int64_t N, double n, double c, int64_t *Q, int64_t *n_plus,
                         int64_t *n_minus) {
  if (!isfinite(n) || !isfinite(c) || N <= 0) return -1;
  double qn = n * (double)N;
  double cn = c * (double)N;
  int64_t q = llround(qn);
  int64_t cc = llround(cn);
  int64_t aq = q < 0 ? -q : q;
  if (cc < aq) cc = aq;
  if (((cc - q) % 2 + 2) % 2 == 1) cc += 1;
  if (cc > N || cc < 0) return -1;
  *Q = q;
  *n_plus = (cc + q) / 2;
  *n_minus = (cc - q) / 2;
  return 0;
}

static int feistel_half_bits(int64_t N) {
  int h = 1;
  while (((int64_t)1 << (2 * h)) < N) ++h;
  return h;
}

/* Balanced four-round Feistel network on [0, 4^h); round function = low h bits
 * of the first Philox word keyed by the seed, counter (R, round, 0, tag). */
static uint64_t feistel_once(const uint32_t key[2], int h, uint64_t x) {
  uint64_t mask = ((uint64_t)1 << h) - 1;
  uint64_t L = x >> h, R = x & mask;
  for (uint32_t round = 0; round < 4; ++round) {
    uint32_t ctr[4] = {(uint32_t)R, round, 0u, ORACLE_TAG_FEISTEL};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    uint64_t F = (uint64_t)w[0] & mask;
    uint64_t newL = R;
    uint64_t newR = L ^ F;
    L = newL;
    R = newR;
  }
  return (L << h) | R;
}

int64_t oracle_feistel_rank(uint64_t seed, int64_t N, int64_t i) {
  uint32_t key[2];
  seed_key(seed, key);
  int h = feistel_half_bits(N);
  /* cycle-walk: apply the permutation until the value lands inside [0, N) */
  uint64_t y = feistel_once(key, h, (uint64_t)i);
  while (y >= (uint64_t)N) y = feistel_once(key, h, y);
  return (int64_t)y;
}

int oracle_init_counts(int Lx, int Ly, uint64_t seed, int64_t n_plus, int64_t n_minus,
                       uint8_t *st) {
  int64_t N = (int64_t)Lx * Ly;
  if (Lx < 2 || Ly < 2 || n_plus < 0 || n_minus < 0 || n_plus + n_minus > N) return -1;
  uint32_t key[2];
  seed_key(seed, key);
  for (int64_t i = 0; i < N; ++i) {
    int64_t rank = oracle_feistel_rank(seed, N, i);
    uint8_t code;
    if (rank < n_plus) {
      code = 2;
    } else if (rank < n_plus + n_minus) {
      code = 3;
    } else {
      uint32_t ctr[4] = {(uint32_t)(i >> 7), 0u, 0u, ORACLE_TAG_SIGN};
      uint32_t w[4];
      oracle_philox4x32_10(ctr, key, w);
      code = (uint8_t)((w[(i >> 5) & 3] >> (i & 31)) & 1u);
    }
    st[i] = code;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Metropolis acceptance (Sec. 3.1: otherwise the classical algorithm):
 * accept with probability min(1, exp(-beta dE)), as a 32-bit threshold.
 * dE = Delta dQ + V dBV + (J/4) dBJ (Eq. 3). */
int oracle_table_index(int dQ, int dBV, int dBJ) {
  return ((dQ + 2) * ORACLE_NB + (dBV + ORACLE_DB)) * ORACLE_NB + (dBJ + ORACLE_DB);
}

static uint32_t threshold_of(double beta, double Delta, double V, double J, int dQ, int dBV,
                             int dBJ) {
  double t1 = Delta * (double)dQ;
  double t2 = V * (double)dBV;
  double t3 = t1 + t2;
  double t4 = 0.25 * J;
  double t5 = t4 * (double)dBJ;
  double dE = t3 + t5;
  if (dE <= 0.0) return 0xFFFFFFFFu;
  double x = -beta * dE;
  double p = exp(x);
  if (p >= 1.0) return 0xFFFFFFFFu;
  double s = ldexp(p, 32);
  double f = floor(s);
  if (f >= 4294967295.0) return 0xFFFFFFFEu;
  return (uint32_t)f;
}

void oracle_threshold_table(double beta, double Delta, double V, double J, uint32_t *table) {
  for (int dQ = -2; dQ <= 2; ++dQ)
    for (int dBV = -ORACLE_DB; dBV <= ORACLE_DB; ++dBV)
      for (int dBJ = -ORACLE_DB; dBJ <= ORACLE_DB; ++dBJ)
        table[oracle_table_index(dQ, dBV, dBJ)] = threshold_of(beta, Delta, V, J, dQ, dBV, dBJ);
}

/* ------------------------------------------------------------------------ */
/* Colour schedule: a phase is the set of pairs (a, a + r) with a = a0 mod 4.
 * Allowed offsets: r != 0 whose residue mod 4 is not 0 or a unit vector, plus
 * the four exact nearest-neighbour offsets. */
int oracle_offset_allowed(int Lx, int Ly, int rx, int ry) {
  rx = ((rx % Lx) + Lx) % Lx;
  ry = ((ry % Ly) + Ly) % Ly;
  if (rx == 0 && ry == 0) return 0;
  if (ry == 0 && (rx == 1 || rx == Lx - 1)) return 1;
  if (rx == 0 && (ry == 1 || ry == Ly - 1)) return 1;
  int mx = rx % 4, my = ry % 4;
  if (mx == 0 && my == 0) return 0;
  if (my == 0 && (mx == 1 || mx == 3)) return 0;
  if (mx == 0 && (my == 1 || my == 3)) return 0;
  return 1;
}

void oracle_schedule(int Lx, int Ly, uint64_t seed, uint64_t P, int *a0x, int *a0y, int *rx,
                     int *ry) {
  uint32_t key[2];
  seed_key(seed, key);
  uint64_t N = (uint64_t)Lx * (uint64_t)Ly;
  uint64_t reject_below = (0 - N) % N; /* 2^64 mod N */
  for (uint32_t attempt = 0; attempt < 64; ++attempt) {
    uint32_t ctr[4] = {attempt, (uint32_t)P, (uint32_t)(P >> 32), ORACLE_TAG_SCHED};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    uint64_t x = ((uint64_t)w[2] << 32) | (uint64_t)w[1];
    unsigned __int128 m = (unsigned __int128)x * (unsigned __int128)N;
    uint64_t lo = (uint64_t)m;
    if (lo < reject_below) continue;
    uint64_t idx = (uint64_t)(m >> 64);
    int cx = (int)(idx % (uint64_t)Lx);
    int cy = (int)(idx / (uint64_t)Lx);
    if (!oracle_offset_allowed(Lx, Ly, cx, cy)) continue;
    *a0x = (int)(w[0] & 3u);
    *a0y = (int)((w[0] >> 2) & 3u);
    *rx = cx;
    *ry = cy;
    return;
  }
  *a0x = 0;
  *a0y = 0;
  *rx = 2;
  *ry = 2;
}

/* ------------------------------------------------------------------------ */
/* Neighbours of site a in the order left, right, up, down (periodic). */
static void neighbours(int Lx, int Ly, int a, int nb[4]) {
  int x = a % Lx, y = a / Lx;
  nb[0] = y * Lx + (x + Lx - 1) % Lx;
  nb[1] = y * Lx + (x + 1) % Lx;
  nb[2] = ((y + Ly - 1) % Ly) * Lx + x;
  nb[3] = ((y + 1) % Ly) * Lx + x;
}

/* Energy change of moving (a, b) to (na, nb): sums over neighbours use the old
 * states and include the partner with its multiplicity m; the a-b bond term is
 * m * dX_a * dX_b (Sec. 3.1, distant- and neighbouring-site cases). */
void oracle_pair_delta(const uint8_t *st, int Lx, int Ly, int a, int b, int na, int nb,
                       int out[3]) {
  int ca = st[a], cb = st[b];
  int nbra[4], nbrb[4];
  neighbours(Lx, Ly, a, nbra);
  neighbours(Lx, Ly, b, nbrb);
  int sumSa = 0, sumGa = 0, sumSb = 0, sumGb = 0, m = 0;
  for (int t = 0; t < 4; ++t) {
    sumSa += CODE_S[st[nbra[t]]];
    sumGa += CODE_SIGMA[st[nbra[t]]];
    sumSb += CODE_S[st[nbrb[t]]];
    sumGb += CODE_SIGMA[st[nbrb[t]]];
    if (nbra[t] == b) ++m;
  }
  int dSa = CODE_S[na] - CODE_S[ca];
  int dSb = CODE_S[nb] - CODE_S[cb];
  int dGa = CODE_SIGMA[na] - CODE_SIGMA[ca];
  int dGb = CODE_SIGMA[nb] - CODE_SIGMA[cb];
  out[0] = CODE_S[na] * CODE_S[na] + CODE_S[nb] * CODE_S[nb] - CODE_S[ca] * CODE_S[ca] -
           CODE_S[cb] * CODE_S[cb];
  out[1] = dSa * sumSa + dSb * sumSb + m * dSa * dSb;
  out[2] = dGa * sumGa + dGb * sumGb + m * dGa * dGb;
}

/* One coupled-pair move (Sec. 3.1): q = S_a + S_b; |q| = 2 cannot change;
 * otherwise draw one configuration of the pair's q-set uniformly (the current
 * one included), then apply the Metropolis test to dE.  The pair's random
 * field v has 16 bits (the low half of F); s0, s1 are words 0 and 1 of its
 * SLOW Philox block.
 *   v < 65532 = 12 x 5461: the choice is v mod |set| (|set| = 4 or 6 divides
 *           12) and w = floor(v / 12), uniform on [0, 5461) and independent of
 *           v mod 12, is the acceptance word's top part: accept iff thr ==
 *           0xFFFFFFFF or w 2^32 + s0 < 5461 thr (64-bit integers), which
 *           happens with probability thr / 2^32.
 *   v >= 65532: the choice is s1 mod |set| when s1 < 4294967292 (a multiple
 *           of 12), else the current configuration; accept iff thr ==
 *           0xFFFFFFFF or s0 < thr. */
int oracle_pair_move(uint8_t *st, int Lx, int Ly, int a, int b, uint32_t F,
                     const uint32_t key[2], const uint32_t slow_ctr[4], const uint32_t *table) {
  int ca = st[a], cb = st[b];
  int q = CODE_S[ca] + CODE_S[cb];
  if (q == 2 || q == -2) return 0;
  uint32_t v = F & 0xFFFFu;
  uint32_t slow[4];
  int have_slow = 0;
  const uint8_t(*set)[2] = (q == 1) ? SET_QP1 : (q == -1) ? SET_QM1 : SET_Q0;
  uint32_t nset = (q == 0) ? 6u : 4u;
  uint32_t idx;
  if (v < 65532u) {
    idx = v % nset;
  } else {
    oracle_philox4x32_10(slow_ctr, key, slow);
    have_slow = 1;
    if (slow[1] < 4294967292u) {
      idx = slow[1] % nset;
    } else {
      idx = 0;
      for (uint32_t t = 0; t < nset; ++t)
        if (set[t][0] == ca && set[t][1] == cb) idx = t;
    }
  }
  int na = set[idx][0];
  int nb = set[idx][1];
  if (na == ca && nb == cb) return 0;
  int d[3];
  oracle_pair_delta(st, Lx, Ly, a, b, na, nb, d);
  uint32_t thr = table[oracle_table_index(d[0], d[1], d[2])];
  int accept;
  if (thr == 0xFFFFFFFFu) {
    accept = 1;
  } else {
    if (!have_slow) {
      oracle_philox4x32_10(slow_ctr, key, slow);
      have_slow = 1;
    }
    if (v < 65532u) {
      uint64_t w = v / 12u;
      accept = (w << 32) + (uint64_t)slow[0] < (uint64_t)5461u * (uint64_t)thr;
    } else {
      accept = slow[0] < thr;
    }
  }
  if (!accept) return 0;
  st[a] = (uint8_t)na;
  st[b] = (uint8_t)nb;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Observables by direct definition (Eq. 3 and the charge sum of Eq. 2). */
void oracle_recount(const uint8_t *st, int Lx, int Ly, int64_t out[7]) {
  int64_t Nc = 0, BV = 0, BJ = 0, M = 0, Ms = 0, Ssum = 0, Ss = 0;
  for (int y = 0; y < Ly; ++y) {
    for (int x = 0; x < Lx; ++x) {
      int c = st[y * Lx + x];
      int cr = st[y * Lx + (x + 1) % Lx];
      int cd = st[((y + 1) % Ly) * Lx + x];
      int sign = ((x + y) % 2 == 0) ? 1 : -1;
      Nc += CODE_S[c] * CODE_S[c];
      BV += CODE_S[c] * CODE_S[cr] + CODE_S[c] * CODE_S[cd];
      BJ += CODE_SIGMA[c] * CODE_SIGMA[cr] + CODE_SIGMA[c] * CODE_SIGMA[cd];
      M += CODE_SIGMA[c];
      Ms += sign * CODE_SIGMA[c];
      Ssum += CODE_S[c];
      Ss += sign * CODE_S[c];
    }
  }
  out[0] = Nc;
  out[1] = BV;
  out[2] = BJ;
  out[3] = M;
  out[4] = Ms;
  out[5] = Ssum;
  out[6] = Ss;
}

static void write_record(const uint8_t *st, int Lx, int Ly, int64_t sweeps_done, int64_t *rec) {
  int64_t c[7];
  oracle_recount(st, Lx, Ly, c);
  rec[0] = sweeps_done;
  for (int t = 0; t < 7; ++t) rec[1 + t] = c[t];
}

/* ------------------------------------------------------------------------ */
/* One colour phase: every pair (a, a + r), a = (4i + a0x, 4j + a0y), with pair
 * index k = j * (Lx/4) + i inside the class.  A class row is cut into blocks
 * of 16 consecutive i, each served by two MOVE calls: pair (i, j) takes half
 * (i mod 2) of word (i / 4) mod 4 of Philox(seed, (j * 2 ceil(Lx/64) +
 * 2 floor(i/16) + (i / 2) mod 2, P_lo, P_hi, MOVE)) as its 16-bit field, so
 * that one call serves the eight pairs with i mod 4 in {0, 1} (or {2, 3}) of a
 * block; its slow words come from Philox(seed, (k, P_lo, P_hi, SLOW)). */
void oracle_phase(uint8_t *st, int Lx, int Ly, uint64_t seed, uint64_t P, const uint32_t *table) {
  uint32_t key[2];
  seed_key(seed, key);
  int a0x, a0y, rx, ry;
  oracle_schedule(Lx, Ly, seed, P, &a0x, &a0y, &rx, &ry);
  int Cx = Lx / 4, Cy = Ly / 4;
  uint32_t Plo = (uint32_t)P, Phi = (uint32_t)(P >> 32);
  for (int j = 0; j < Cy; ++j) {
    for (int i = 0; i < Cx; ++i) {
      int64_t k = (int64_t)j * Cx + i;
      int ax = 4 * i + a0x, ay = 4 * j + a0y;
      int bx = (ax + rx) % Lx, by = (ay + ry) % Ly;
      int64_t call = (int64_t)j * 2 * ((Cx + 15) / 16) + 2 * (i / 16) + ((i / 2) % 2);
      uint32_t mctr[4] = {(uint32_t)call, Plo, Phi, ORACLE_TAG_MOVE};
      uint32_t mw[4];
      oracle_philox4x32_10(mctr, key, mw);
      uint32_t R = (mw[(i / 4) % 4] >> (16 * (i % 2))) & 0xFFFFu;
      uint32_t sctr[4] = {(uint32_t)k, Plo, Phi, ORACLE_TAG_SLOW};
      oracle_pair_move(st, Lx, Ly, ay * Lx + ax, by * Lx + bx, R, key, sctr, table);
    }
  }
}

int64_t oracle_sweeps(uint8_t *st, int Lx, int Ly, uint64_t seed, int64_t sweep0,
                      int64_t nsweeps, double beta, double Delta, double V, double J,
                      int obs_every, int64_t *records) {
  uint32_t *table = (uint32_t *)malloc(sizeof(uint32_t) * ORACLE_TABLE_SIZE);
  if (!table) return -1;
  oracle_threshold_table(beta, Delta, V, J, table);
  int64_t nrec = 0;
  for (int64_t s = 0; s < nsweeps; ++s) {
    int64_t sweep = sweep0 + s;
    for (int p = 0; p < 8; ++p) oracle_phase(st, Lx, Ly, seed, (uint64_t)(8 * sweep + p), table);
    if (obs_every > 0 && (sweep + 1) % obs_every == 0 && records) {
      write_record(st, Lx, Ly, sweep + 1, records + ORACLE_REC * nrec);
      ++nrec;
    }
  }
  free(table);
  return nrec;
}

/* ------------------------------------------------------------------------ */
/* Sequential random-pair mode (Sec. 3.1 as a serial algorithm): move t draws an
 * ordered pair index uniform on [0, N(N-1)) from Philox(seed, (t_lo, t_hi,
 * attempt, SEQ)) words 0-1 by multiply-high with rejection; the low half of
 * word 2 is the pair's random field. */
int64_t oracle_sequential_sweeps(uint8_t *st, int Lx, int Ly, uint64_t seed, int64_t sweep0,
                                 int64_t nsweeps, double beta, double Delta, double V, double J,
                                 int obs_every, int64_t *records) {
  uint32_t key[2];
  seed_key(seed, key);
  uint32_t *table = (uint32_t *)malloc(sizeof(uint32_t) * ORACLE_TABLE_SIZE);
  if (!table) return -1;
  oracle_threshold_table(beta, Delta, V, J, table);
  uint64_t N = (uint64_t)Lx * (uint64_t)Ly;
  uint64_t npairs = N * (N - 1);
  uint64_t reject_below = (0 - npairs) % npairs;
  int64_t moves = (int64_t)(N / 2);
  int64_t nrec = 0;
  for (int64_t s = 0; s < nsweeps; ++s) {
    int64_t sweep = sweep0 + s;
    for (int64_t mv = 0; mv < moves; ++mv) {
      uint64_t t = (uint64_t)(sweep * moves + mv);
      for (uint32_t attempt = 0; attempt < 64; ++attempt) {
        uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), attempt, ORACLE_TAG_SEQ};
        uint32_t w[4];
        oracle_philox4x32_10(ctr, key, w);
        uint64_t x = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
        unsigned __int128 m = (unsigned __int128)x * (unsigned __int128)npairs;
        if ((uint64_t)m < reject_below) continue;
        uint64_t pidx = (uint64_t)(m >> 64);
        int a = (int)(pidx / (N - 1));
        int b = (int)(pidx % (N - 1));
        if (b >= a) b += 1;
        uint32_t sctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), attempt, ORACLE_TAG_SEQSLOW};
        oracle_pair_move(st, Lx, Ly, a, b, w[2], key, sctr, table);
        break;
      }
    }
    if (obs_every > 0 && (sweep + 1) % obs_every == 0 && records) {
      write_record(st, Lx, Ly, sweep + 1, records + ORACLE_REC * nrec);
      ++nrec;
    }
  }
  free(table);
  return nrec;
}

/* Short-range pair mode: the paper's first version, abandoned because it
 * misses low-temperature results on 4 x 4 (Sec. 3.2).  Each move picks site a
 * uniformly and its partner b uniformly among a's four nearest neighbours
 * (right, left, down, up), then makes the coupled-pair move of Sec. 3.1; N/2
 * moves per sweep.  Random words: Philox(seed, (t_lo, t_hi, attempt, NN)) with
 * t the global move index; words 0-1 give (a, direction) by Lemire's
 * multiply-high over 4N with rejection, the low half of word 2 is the pair's
 * random field. */
int64_t oracle_neighbour_sweeps(uint8_t *st, int Lx, int Ly, uint64_t seed, int64_t sweep0,
                                int64_t nsweeps, double beta, double Delta, double V, double J,
                                int obs_every, int64_t *records) {
  uint32_t key[2];
  seed_key(seed, key);
  uint32_t *table = (uint32_t *)malloc(sizeof(uint32_t) * ORACLE_TABLE_SIZE);
  if (!table) return -1;
  oracle_threshold_table(beta, Delta, V, J, table);
  uint64_t N = (uint64_t)Lx * (uint64_t)Ly;
  uint64_t nchoices = 4 * N;
  uint64_t reject_below = (0 - nchoices) % nchoices;
  int64_t moves = (int64_t)(N / 2);
  int64_t nrec = 0;
  for (int64_t s = 0; s < nsweeps; ++s) {
    int64_t sweep = sweep0 + s;
    for (int64_t mv = 0; mv < moves; ++mv) {
      uint64_t t = (uint64_t)(sweep * moves + mv);
      for (uint32_t attempt = 0; attempt < 64; ++attempt) {
        uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), attempt, ORACLE_TAG_NN};
        uint32_t w[4];
        oracle_philox4x32_10(ctr, key, w);
        uint64_t x = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
        unsigned __int128 m = (unsigned __int128)x * (unsigned __int128)nchoices;
        if ((uint64_t)m < reject_below) continue;
        uint64_t pidx = (uint64_t)(m >> 64);
        int a = (int)(pidx / 4), dir = (int)(pidx % 4);
        int ax = a % Lx, ay = a / Lx;
        int bx = ax, by = ay;
        if (dir == 0) bx = (ax + 1) % Lx;
        else if (dir == 1) bx = (ax + Lx - 1) % Lx;
        else if (dir == 2) by = (ay + 1) % Ly;
        else by = (ay + Ly - 1) % Ly;
        int b = by * Lx + bx;
        uint32_t sctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), attempt, ORACLE_TAG_NNSLOW};
        oracle_pair_move(st, Lx, Ly, a, b, w[2], key, sctr, table);
        break;
      }
    }
    if (obs_every > 0 && (sweep + 1) % obs_every == 0 && records) {
      write_record(st, Lx, Ly, sweep + 1, records + ORACLE_REC * nrec);
      ++nrec;
    }
  }
  free(table);
  return nrec;
}

/* ------------------------------------------------------------------------ */
/* Paper-faithful maps (Sec. 3.2, the algorithm for building a map).  A map is
 * a list of P = max(1, floor(N / 10)) pairs built by random marking on an
 * L x L array of flags, all clear at first: draw a site until it is unmarked,
 * mark it (site a); draw and mark site b the same way (b may be a neighbour
 * of a); add (a, b); mark the nearest neighbours of a and of b; repeat until
 * the map holds P pairs.  Later pairs never touch an earlier pair's sites or
 * their neighbours, so the pairs of a map do not interact.
 *
 * Draws of map m: draw d uses words 2(d mod 2), 2(d mod 2) + 1 of
 * Philox(seed, (d / 2, m_lo, m_hi, MAP)) as a 64-bit x; the site is the high
 * word of x * N unless the low word is below 2^64 mod N (rejected: next d).
 * Moves: pair p of map m takes the low half of word 0 of Philox(seed, (p,
 * m_lo, m_hi, MAPMOVE)) as its random field and (p, m_lo, m_hi, MAPSLOW) as its slow
 * counter (oracle_pair_move). */
int64_t oracle_map_size(int Lx, int Ly) {
  int64_t P = (int64_t)Lx * Ly / 10;
  return P < 1 ? 1 : P;
}

int oracle_map_build(int Lx, int Ly, uint64_t seed, int64_t m, int32_t *pairs) {
  uint32_t key[2];
  seed_key(seed, key);
  uint64_t N = (uint64_t)Lx * (uint64_t)Ly;
  int64_t P = oracle_map_size(Lx, Ly);
  uint8_t *marked = (uint8_t *)calloc((size_t)N, 1);
  if (!marked) return -1;
  uint64_t reject_below = (0 - N) % N;
  uint64_t d = 0;
  uint32_t w[4];
  for (int64_t p = 0; p < P; ++p) {
    int site[2];
    for (int k = 0; k < 2; ++k) {
      for (;;) {
        if ((d & 1) == 0) {
          uint32_t ctr[4] = {(uint32_t)(d >> 1), (uint32_t)m, (uint32_t)((uint64_t)m >> 32),
                             ORACLE_TAG_MAP};
          oracle_philox4x32_10(ctr, key, w);
        }
        int h = (int)(d & 1);
        ++d;
        uint64_t x = ((uint64_t)w[2 * h + 1] << 32) | (uint64_t)w[2 * h];
        unsigned __int128 prod = (unsigned __int128)x * (unsigned __int128)N;
        if ((uint64_t)prod < reject_below) continue;
        int cand = (int)(uint64_t)(prod >> 64);
        if (marked[cand]) continue;
        marked[cand] = 1;
        site[k] = cand;
        break;
      }
    }
    pairs[2 * p] = site[0];
    pairs[2 * p + 1] = site[1];
    for (int k = 0; k < 2; ++k) {
      int nb[4];
      neighbours(Lx, Ly, site[k], nb);
      for (int t = 0; t < 4; ++t) marked[nb[t]] = 1;
    }
  }
  free(marked);
  return 0;
}

int64_t oracle_map_sweeps(uint8_t *st, int Lx, int Ly, uint64_t seed, int64_t map0, int64_t nmaps,
                          double beta, double Delta, double V, double J, int obs_every,
                          int64_t *records) {
  uint32_t key[2];
  seed_key(seed, key);
  int64_t P = oracle_map_size(Lx, Ly);
  uint32_t *table = (uint32_t *)malloc(sizeof(uint32_t) * ORACLE_TABLE_SIZE);
  int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)P);
  if (!table || !pairs) {
    free(table);
    free(pairs);
    return -1;
  }
  oracle_threshold_table(beta, Delta, V, J, table);
  int64_t nrec = 0;
  for (int64_t k = 0; k < nmaps; ++k) {
    int64_t m = map0 + k;
    if (oracle_map_build(Lx, Ly, seed, m, pairs) != 0) {
      nrec = -1;
      break;
    }
    for (int64_t p = 0; p < P; ++p) {
      uint32_t ctr[4] = {(uint32_t)p, (uint32_t)m, (uint32_t)((uint64_t)m >> 32),
                         ORACLE_TAG_MAPMOVE};
      uint32_t w[4];
      oracle_philox4x32_10(ctr, key, w);
      uint32_t sctr[4] = {(uint32_t)p, (uint32_t)m, (uint32_t)((uint64_t)m >> 32),
                          ORACLE_TAG_MAPSLOW};
      oracle_pair_move(st, Lx, Ly, pairs[2 * p], pairs[2 * p + 1], w[0], key, sctr, table);
    }
    if (obs_every > 0 && (m + 1) % obs_every == 0 && records) {
      write_record(st, Lx, Ly, m + 1, records + ORACLE_REC * nrec);
      ++nrec;
    }
  }
  free(pairs);
  free(table);
  return nrec;
}

/* ------------------------------------------------------------------------ */
/* Single-site energy change (Eq. 3): only the terms of site a change; each of
 * its bonds contributes the change of a's value times the neighbour's (old)
 * value. */
void oracle_site_delta(const uint8_t *st, int Lx, int Ly, int a, int nc, int out[3]) {
  int c = st[a];
  int nbr[4];
  neighbours(Lx, Ly, a, nbr);
  int sumS = 0, sumG = 0;
  for (int k = 0; k < 4; ++k) {
    sumS += CODE_S[st[nbr[k]]];
    sumG += CODE_SIGMA[st[nbr[k]]];
  }
  int dS = CODE_S[nc] - CODE_S[c];
  int dG = CODE_SIGMA[nc] - CODE_SIGMA[c];
  out[0] = CODE_S[nc] * CODE_S[nc] - CODE_S[c] * CODE_S[c];
  out[1] = dS * sumS;
  out[2] = dG * sumG;
}

/* ------------------------------------------------------------------------ */
/* Penalty-function baseline (Sec. 2.2): the charge is held near nN not by the
 * move but by a chemical-potential term -mu sum_i S_i added to the energy, with
 * mu adjusted as the run goes.  Single-site Metropolis: a uniformly chosen site
 * takes one of its three other states, uniformly, accepted with probability
 * min(1, exp(-beta (dE - mu dS))), N proposals per sweep.  The paper gives no
 * rule for adjusting mu; reading: after every sweep
 *   mu <- mu + kappa (n N - sum_i S_i) / N.
 * Random words: Philox(seed, (t_lo, t_hi, 0, PENALTY)) for proposal t: words
 * 0-1 the site (Lemire over N, rejection), word 2 mod 3 the new state (word 2
 * below 4294967295, a multiple of 3; else the proposal is skipped), word 3 the
 * acceptance test (u / 2^32 < p).  Records as in the other modes; mu_trace
 * (if not NULL) receives mu after every sweep. */
int64_t oracle_penalty_sweeps(uint8_t *st, int Lx, int Ly, uint64_t seed, int64_t sweep0,
                              int64_t nsweeps, double beta, double Delta, double V, double J,
                              double n, double *mu, double kappa, int obs_every,
                              int64_t *records, double *mu_trace) {
  uint32_t key[2];
  seed_key(seed, key);
  uint64_t N = (uint64_t)Lx * (uint64_t)Ly;
  uint64_t reject_below = (0 - N) % N;
  int64_t Ssum = 0;
  for (uint64_t i = 0; i < N; ++i) Ssum += CODE_S[st[i]];
  int64_t nrec = 0;
  for (int64_t s = 0; s < nsweeps; ++s) {
    int64_t sweep = sweep0 + s;
    for (uint64_t mv = 0; mv < N; ++mv) {
      uint64_t t = (uint64_t)sweep * N + mv;
      uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), 0u, ORACLE_TAG_PENALTY};
      uint32_t w[4];
      oracle_philox4x32_10(ctr, key, w);
      uint64_t x = ((uint64_t)w[1] << 32) | (uint64_t)w[0];
      unsigned __int128 prod = (unsigned __int128)x * (unsigned __int128)N;
      if ((uint64_t)prod < reject_below || w[2] == 0xFFFFFFFFu) continue;
      int a = (int)(uint64_t)(prod >> 64);
      int c = st[a];
      int nc = (c + 1 + (int)(w[2] % 3u)) & 3;
      int d[3];
      oracle_site_delta(st, Lx, Ly, a, nc, d);
      int dS = CODE_S[nc] - CODE_S[c];
      double dE = Delta * d[0] + V * (double)d[1] + 0.25 * J * (double)d[2];
      double dEp = dE - *mu * (double)dS;
      int accept = dEp <= 0.0 || ((double)w[3] * 0x1p-32) < exp(-beta * dEp);
      if (accept) {
        st[a] = (uint8_t)nc;
        Ssum += dS;
      }
    }
    *mu += kappa * (n * (double)N - (double)Ssum) / (double)N;
    if (mu_trace) mu_trace[s] = *mu;
    if (obs_every > 0 && (sweep + 1) % obs_every == 0 && records) {
      write_record(st, Lx, Ly, sweep + 1, records + ORACLE_REC * nrec);
      ++nrec;
    }
  }
  return nrec;
}
