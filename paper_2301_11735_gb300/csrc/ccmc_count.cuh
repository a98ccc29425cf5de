// ccmc_count.cuh -- observables of a packed lattice by definition (Eq. 3 and
// Eq. 2): popcounts of the charge and sign bit planes of each class word
// against its right and down neighbour windows.  Used by the recount kernel
// and by the resident batch kernel.
#pragma once

#include <cstdint>

#include "ccmc_device.cuh"
#include "ccmc_internal.h"

namespace ccmc {

__device__ __forceinline__ int64_t warp_sum(int64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Bit planes of a class word X against its right and down neighbour windows
// Yr, Yd, with every site's type bit (1 = charged) left in place at the odd
// bit and its sign bit (1 = minus) at the even bit below it.  `vo` holds the
// odd bits of the valid sites.  Bonds are laid out two to a site: the right
// bond at the odd bit, the down bond at the even bit (the down masks shifted
// down one place, which adds to the right ones without carries).
struct WordPlanes {
  uint32_t k, kg, ug;  // charged, charged with S = -1, magnetic with sigma = -1
  uint32_t kk, uu;     // charged-charged and magnetic-magnetic bonds
  uint32_t f;          // bonds whose two signs differ
};

__device__ __forceinline__ WordPlanes word_planes(uint32_t X, uint32_t Yr, uint32_t Yd,
                                                  uint32_t vo) {
  constexpr uint32_t kEven = 0x55555555u, kOdd = 0xAAAAAAAAu;
  WordPlanes p;
  const uint32_t Xs = X << 1;  // sign bits moved up to the type bits
  p.k = X & vo;
  p.kg = X & Xs & vo;
  p.ug = ~X & Xs & vo;
  p.kk = (X & Yr & vo) + ((X & Yd & vo) >> 1);
  p.uu = (~(X | Yr) & vo) + ((~(X | Yd) & vo) >> 1);
  p.f = (((X ^ Yr) << 1) & kOdd) | ((X ^ Yd) & kEven);
  return p;
}

// Popcount sums of one class: the sites' planes and the bonds' planes, and
// the number of sites counted.  fold() turns them into c[7] (Nc, BV, BJ, M,
// M_stag, S_sum, S_stag); the staggered sign is uniform over a class.
struct ClassCounts {
  int sites = 0, nK = 0, nKG = 0, nUG = 0, nKK = 0, nKKd = 0, nUU = 0, nUUd = 0;

  __device__ __forceinline__ void bonds(const WordPlanes &p) {
    nKK += __popc(p.kk);
    nKKd += __popc(p.kk & p.f);
    nUU += __popc(p.uu);
    nUUd += __popc(p.uu & p.f);
  }
  __device__ __forceinline__ void fold(int cls, int c[7]) const {
    const int sgn = (((cls & 3) + (cls >> 2)) & 1) ? -1 : 1;
    const int M = sites - nK - 2 * nUG, S = nK - 2 * nKG;
    c[0] += nK;
    c[1] += nKK - 2 * nKKd;
    c[2] += nUU - 2 * nUUd;
    c[3] += M;
    c[4] += sgn * M;
    c[5] += S;
    c[6] += sgn * S;
  }
};

// Adds the observables of words tid, tid + nthreads, ... of class `cls` to
// c[7] (Nc, BV, BJ, M, M_stag, S_sum, S_stag), any row width.
__device__ __forceinline__ void count_class(const Geo &g, int cls, int tid, int nthreads,
                                            int c[7]) {
  const int W = g.W, nw = g.Cy * W;
  const int cx = cls & 3, cy = cls >> 2;
  const uint32_t *X0 = g.words + (int64_t)cls * g.cstride;
  const uint32_t *R0 = g.words + (int64_t)(cy * 4 + ((cx + 1) & 3)) * g.cstride;
  const uint32_t *D0 = g.words + (int64_t)(((cy + 1) & 3) * 4 + cx) * g.cstride;
  ClassCounts n;
  int wid = tid;
  int j = wid / W, w = wid - j * W;
  const int sj = nthreads / W, sw = nthreads - sj * W;
  for (; wid < nw; wid += nthreads) {
    const int s0 = w << 4;
    const int ns = min(16, g.Cx - s0);
    const uint32_t vo = ns == 16 ? 0xAAAAAAAAu : (((1u << (2 * ns)) - 1u) & 0xAAAAAAAAu);
    const uint32_t X = X0[wid];
    const uint32_t Xr = fetch_window(R0 + j * W, W, g.Cx,
                                     cx == 3 ? (s0 + 1 == g.Cx ? 0 : s0 + 1) : s0, ns);
    const int jd = cy == 3 ? (j + 1 == g.Cy ? 0 : j + 1) : j;
    const uint32_t Xd = D0[jd * W + w];
    const WordPlanes p = word_planes(X, Xr, Xd, vo);
    n.sites += ns;
    n.nK += __popc(p.k);
    n.nKG += __popc(p.kg);
    n.nUG += __popc(p.ug);
    n.bonds(p);
    w += sw;
    j += sj;
    if (w >= W) {
      w -= W;
      ++j;
    }
  }
  n.fold(cls, c);
}

// The quad path: rows of whole words (Cx a multiple of 16) with W a multiple
// of 4, four consecutive words of a class row per step with 16-byte loads.
// Every site's type bit (odd) and sign bit (even) are first copied into both
// bits of its pair, one plane per word for the word and one for its two
// neighbour windows (right window at the odd bits, down window at the even
// bits); then one AND is the charged-charged bonds of both directions, and an
// XOR of the sign planes marks the bonds whose signs differ.  The count of
// magnetic-magnetic bonds is not formed: over the whole lattice it follows
// from the others (below).  Sites of two words share one popcount (types of
// the first at the odd bits, of the second at the even bits).
struct QuadCounts {
  int nK = 0, nKG = 0, nUG = 0, nKK = 0, nKKd = 0, nUUd = 0, quads = 0;
};

// One three-input logic instruction: kLut is the function's truth table on
// the canonical inputs a = 0xF0, b = 0xCC, c = 0xAA.
template <uint32_t kLut>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(kLut));
  return d;
}
constexpr uint32_t kLutMux = 0xE4;      // c ? a : b, bit by bit
constexpr uint32_t kLutAnd3 = 0x80;     // a & b & c
constexpr uint32_t kLutNorAnd = 0x02;   // ~(a | b) & c
constexpr uint32_t kLutAndNot = 0x0C;   // ~a & b

template <bool kColR, bool kRowD>
__device__ __forceinline__ void count_quads(const uint32_t *__restrict__ X0,
                                            const uint32_t *__restrict__ R0,
                                            const uint32_t *__restrict__ D0, int W, int Cy,
                                            int q, int nthreads, QuadCounts &n) {
  constexpr uint32_t kOdd = 0xAAAAAAAAu;
  const int Wq = W >> 2, nq = Cy * Wq, last_row = (Cy - 1) * Wq;
  int wq = q % Wq;
  const int sw = nthreads % Wq;
#pragma unroll 2
  for (; q < nq; q += nthreads) {
    const int o = 4 * q;  // word offset of the quad: row j, column 4 wq
    // the down neighbours of class row Cy-1 of the last class row wrap to row 0
    const int od = kRowD ? (q < last_row ? o + W : o - last_row * 4) : o;
    const uint4 x = *reinterpret_cast<const uint4 *>(X0 + o);
    const uint4 r = *reinterpret_cast<const uint4 *>(R0 + o);
    const uint4 d = *reinterpret_cast<const uint4 *>(D0 + od);
    // right neighbours of class column 3 are one column further on: the
    // windows start one site later (the last one wraps to the row's start)
    uint32_t rn = 0u;
    if (kColR) {
      rn = R0[wq == Wq - 1 ? o + 4 - W : o + 4];
      wq += sw;
      if (wq >= Wq) wq -= Wq;
    }
    const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
    const uint32_t ds[4] = {d.x, d.y, d.z, d.w};
    const uint32_t rs[5] = {r.x, r.y, r.z, r.w, rn};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t X = xs[k], Yd = ds[k];
      const uint32_t Yr = kColR ? __funnelshift_r(rs[k], rs[k + 1], 2) : rs[k];
      const uint32_t tX = lop3<kLutMux>(X, X >> 1, kOdd);  // type in both bits
      const uint32_t gX = lop3<kLutMux>(X << 1, X, kOdd);  // sign in both bits
      const uint32_t tY = lop3<kLutMux>(Yr, Yd >> 1, kOdd);
      const uint32_t gY = lop3<kLutMux>(Yr << 1, Yd, kOdd);
      const uint32_t f = gX ^ gY;
      n.nKK += __popc(tX & tY);
      n.nKKd += __popc(lop3<kLutAnd3>(tX, tY, f));
      n.nUUd += __popc(lop3<kLutNorAnd>(tX, tY, f));
    }
#pragma unroll
    for (int k = 0; k < 4; k += 2) {
      const uint32_t T = lop3<kLutMux>(xs[k], xs[k + 1] >> 1, kOdd);
      const uint32_t S = lop3<kLutMux>(xs[k] << 1, xs[k + 1], kOdd);
      n.nK += __popc(T);
      n.nKG += __popc(T & S);
      n.nUG += __popc(lop3<kLutAndNot>(T, S, 0u));
    }
    ++n.quads;
  }
}

// Adds the quad path's counts of class `cls` to c[7].  c[2] receives
// nKK - 2 nUUd only: with nUU the magnetic-magnetic bonds, every site having
// two bonds (2N in all) and every charged site four bond ends
// (4 Nc = 2 nKK + n_mixed), the lattice total is nUU = 2N - 4 Nc + nKK, so
// BJ = nUU - 2 nUUd lacks the term 2N - 4 Nc, which bj_completion() gives
// once for the whole lattice.
__device__ __forceinline__ void count_class_quads(const Geo &g, int cls, int tid, int nthreads,
                                                  int c[7]) {
  const int cx = cls & 3, cy = cls >> 2;
  const uint32_t *X0 = g.words + (int64_t)cls * g.cstride;
  const uint32_t *R0 = g.words + (int64_t)(cy * 4 + ((cx + 1) & 3)) * g.cstride;
  const uint32_t *D0 = g.words + (int64_t)(((cy + 1) & 3) * 4 + cx) * g.cstride;
  QuadCounts n;
  if (cx == 3) {
    if (cy == 3) count_quads<true, true>(X0, R0, D0, g.W, g.Cy, tid, nthreads, n);
    else count_quads<true, false>(X0, R0, D0, g.W, g.Cy, tid, nthreads, n);
  } else {
    if (cy == 3) count_quads<false, true>(X0, R0, D0, g.W, g.Cy, tid, nthreads, n);
    else count_quads<false, false>(X0, R0, D0, g.W, g.Cy, tid, nthreads, n);
  }
  const int sgn = ((cx + cy) & 1) ? -1 : 1;
  const int M = 64 * n.quads - n.nK - 2 * n.nUG, S = n.nK - 2 * n.nKG;
  c[0] += n.nK;
  c[1] += n.nKK - 2 * n.nKKd;
  c[2] += n.nKK - 2 * n.nUUd;
  c[3] += M;
  c[4] += sgn * M;
  c[5] += S;
  c[6] += sgn * S;
}

__device__ __forceinline__ bool quads_ok(const Geo &g) {
  return (g.Cx & 15) == 0 && (g.W & 3) == 0;
}

// The part of BJ that count_class_quads leaves to the lattice total, given the
// lattice's number of charged sites Nc.
__device__ __forceinline__ int64_t bj_completion(const Geo &g, int64_t Nc) {
  return quads_ok(g) ? 2 * (int64_t)g.Lx * g.Ly - 4 * Nc : 0;
}

}  // namespace ccmc
