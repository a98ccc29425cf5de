/*
 * exact_enum.c -- exact enumeration of the constrained ensemble on tiny
 * lattices, the check the paper ran against its 4x4 exact solution (Sec. 3.3).
 *
 * TEST INFRASTRUCTURE (part of the oracle; see ccmc_oracle.h).
 *
 * Every state of an Lx x Ly torus (Lx <= 4, N <= 16) whose charge sum equals Q
 * is visited once; its integer energy terms (Nc, BV, BJ) of Eq. (3) and its
 * magnetisations are computed from the definition, row by row, and the state
 * is counted in a histogram over (Nc, BV, BJ).  Canonical averages at any
 * (beta, Delta, V, J) then follow from the histogram exactly.
 */
#include <stdlib.h>
#include <string.h>

#include "ccmc_oracle.h"

static const int ES[4] = {0, 0, 1, -1};
static const int EG[4] = {1, -1, 0, 0};

typedef struct {
  int Lx, Ly, N, nrow, Q;
  int rq[256], rnc[256], rbv[256], rbj[256], rm[256], rms[256];
  int vbv[256][256], vbj[256][256];
  int bucket_n[9];
  int bucket[9][256];
} enum_ctx;

typedef struct {
  int64_t *count, *m2, *mabs, *mstag2;
} hist;

static int code_at(int r, int x) { return (r >> (2 * x)) & 3; }

static void leaf(const enum_ctx *c, const int *rows, hist *h) {
  int Nc = 0, BV = 0, BJ = 0, M = 0, Ms = 0;
  for (int y = 0; y < c->Ly; ++y) {
    int r = rows[y], rn = rows[(y + 1) % c->Ly];
    int sgn = (y % 2 == 0) ? 1 : -1;
    Nc += c->rnc[r];
    BV += c->rbv[r] + c->vbv[r][rn];
    BJ += c->rbj[r] + c->vbj[r][rn];
    M += c->rm[r];
    Ms += sgn * c->rms[r];
  }
  int nb = 4 * c->N + 1;
  int64_t bin = ((int64_t)Nc * nb + (BV + 2 * c->N)) * nb + (BJ + 2 * c->N);
  h->count[bin] += 1;
  h->m2[bin] += (int64_t)M * M;
  h->mabs[bin] += M < 0 ? -M : M;
  h->mstag2[bin] += (int64_t)Ms * Ms;
}

static int64_t descend(const enum_ctx *c, int *rows, int depth, int qsum, hist *h) {
  if (depth == c->Ly - 1) {
    int need = c->Q - qsum;
    if (need < -4 || need > 4) return 0;
    int64_t n = 0;
    for (int t = 0; t < c->bucket_n[need + 4]; ++t) {
      rows[depth] = c->bucket[need + 4][t];
      leaf(c, rows, h);
      ++n;
    }
    return n;
  }
  int64_t n = 0;
  for (int r = 0; r < c->nrow; ++r) {
    rows[depth] = r;
    n += descend(c, rows, depth + 1, qsum + c->rq[r], h);
  }
  return n;
}

int64_t oracle_enumerate(int Lx, int Ly, int Q, int64_t *count, int64_t *m2, int64_t *mabs,
                         int64_t *mstag2) {
  if (Lx < 2 || Lx > 4 || Ly < 2 || Lx * Ly > 16) return -1;
  enum_ctx *c = (enum_ctx *)calloc(1, sizeof(enum_ctx));
  if (!c) return -1;
  c->Lx = Lx;
  c->Ly = Ly;
  c->N = Lx * Ly;
  c->nrow = 1 << (2 * Lx);
  c->Q = Q;
  for (int r = 0; r < c->nrow; ++r) {
    int q = 0, nc = 0, bv = 0, bj = 0, m = 0, ms = 0;
    for (int x = 0; x < Lx; ++x) {
      int a = code_at(r, x), b = code_at(r, (x + 1) % Lx);
      q += ES[a];
      nc += ES[a] * ES[a];
      bv += ES[a] * ES[b];
      bj += EG[a] * EG[b];
      m += EG[a];
      ms += (x % 2 == 0 ? 1 : -1) * EG[a];
    }
    c->rq[r] = q;
    c->rnc[r] = nc;
    c->rbv[r] = bv;
    c->rbj[r] = bj;
    c->rm[r] = m;
    c->rms[r] = ms;
    c->bucket[q + 4][c->bucket_n[q + 4]++] = r;
    for (int r2 = 0; r2 < c->nrow; ++r2) {
      int vv = 0, vj = 0;
      for (int x = 0; x < Lx; ++x) {
        vv += ES[code_at(r, x)] * ES[code_at(r2, x)];
        vj += EG[code_at(r, x)] * EG[code_at(r2, x)];
      }
      c->vbv[r][r2] = vv;
      c->vbj[r][r2] = vj;
    }
  }
  int nb = 4 * c->N + 1;
  int64_t nbins = (int64_t)(c->N + 1) * nb * nb;
  memset(count, 0, sizeof(int64_t) * nbins);
  memset(m2, 0, sizeof(int64_t) * nbins);
  memset(mabs, 0, sizeof(int64_t) * nbins);
  memset(mstag2, 0, sizeof(int64_t) * nbins);
  int64_t total = 0;
  int nrow = c->nrow;
#pragma omp parallel reduction(+ : total)
  {
    hist h;
    h.count = (int64_t *)calloc(nbins, sizeof(int64_t));
    h.m2 = (int64_t *)calloc(nbins, sizeof(int64_t));
    h.mabs = (int64_t *)calloc(nbins, sizeof(int64_t));
    h.mstag2 = (int64_t *)calloc(nbins, sizeof(int64_t));
    int rows[4];
#pragma omp for schedule(dynamic, 1)
    for (int r0 = 0; r0 < nrow; ++r0) {
      rows[0] = r0;
      total += descend(c, rows, 1, c->rq[r0], &h);
    }
#pragma omp critical
    {
      for (int64_t t = 0; t < nbins; ++t) {
        count[t] += h.count[t];
        m2[t] += h.m2[t];
        mabs[t] += h.mabs[t];
        mstag2[t] += h.mstag2[t];
      }
    }
    free(h.count);
    free(h.m2);
    free(h.mabs);
    free(h.mstag2);
  }
  free(c);
  return total;
}
