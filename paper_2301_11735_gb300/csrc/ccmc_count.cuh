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

// Adds the observables of words tid, tid + nthreads, ... of class `cls` to
// c[7] (Nc, BV, BJ, M, M_stag, S_sum, S_stag): popcounts of the charge and
// sign bit planes against the right and down neighbour windows.
__device__ __forceinline__ void count_class(const Geo &g, int cls, int tid, int nthreads,
                                            int c[7]) {
  const int W = g.W, nw = g.Cy * W;
  const int cx = cls & 3, cy = cls >> 2;
  const int sgn = ((cx + cy) & 1) ? -1 : 1;
  const uint32_t *X0 = g.words + (int64_t)cls * g.cstride;
  const uint32_t *R0 = g.words + (int64_t)(cy * 4 + ((cx + 1) & 3)) * g.cstride;
  const uint32_t *D0 = g.words + (int64_t)(((cy + 1) & 3) * 4 + cx) * g.cstride;
  int wid = tid;
  int j = wid / W, w = wid - j * W;
  const int sj = nthreads / W, sw = nthreads - sj * W;
  for (; wid < nw; wid += nthreads) {
    const int s0 = w << 4;
    const int n = min(16, g.Cx - s0);
    const uint32_t valid = n == 16 ? 0x55555555u : (((1u << (2 * n)) - 1u) & 0x55555555u);
    const uint32_t X = X0[wid];
    const uint32_t Xr = fetch_window(R0 + j * W, W, g.Cx,
                                     cx == 3 ? (s0 + 1 == g.Cx ? 0 : s0 + 1) : s0, n);
    const int jd = cy == 3 ? (j + 1 == g.Cy ? 0 : j + 1) : j;
    const uint32_t Xd = D0[jd * W + w];
    const uint32_t K = (X >> 1) & valid, G = X & valid;
    const uint32_t U = ~K & valid;  // magnetic
    const int chg = __popc(K & ~G) - __popc(K & G);
    const int mag = __popc(U & ~G) - __popc(U & G);
    c[0] += __popc(K);
    c[3] += mag;
    c[4] += sgn * mag;
    c[5] += chg;
    c[6] += sgn * chg;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const uint32_t Y = d ? Xd : Xr;
      const uint32_t KY = (Y >> 1) & valid, GY = Y & valid;
      const uint32_t diff = G ^ GY;
      const uint32_t KK = K & KY;
      const uint32_t UU = U & ~KY & valid;
      c[1] += __popc(KK & ~diff) - __popc(KK & diff);
      c[2] += __popc(UU & ~diff) - __popc(UU & diff);
    }
    w += sw;
    j += sj;
    if (w >= W) {
      w -= W;
      ++j;
    }
  }
}

// The same counts for rows of whole words (Cx a multiple of 16) with W a
// multiple of 4: each step takes four consecutive words of a class row with
// 16-byte loads.  Signed counts are formed as popc(P) - 2 popc(P & minus) and
// the staggered sign (uniform over a class) is applied once at the end.
__device__ __forceinline__ void count_class_quads(const Geo &g, int cls, int tid, int nthreads,
                                                  int c[7]) {
  const int W = g.W, Wq = W >> 2, nq = g.Cy * Wq;
  const int cx = cls & 3, cy = cls >> 2;
  const uint32_t *X0 = g.words + (int64_t)cls * g.cstride;
  const uint32_t *R0 = g.words + (int64_t)(cy * 4 + ((cx + 1) & 3)) * g.cstride;
  const uint32_t *D0 = g.words + (int64_t)(((cy + 1) & 3) * 4 + cx) * g.cstride;
  constexpr uint32_t kEven = 0x55555555u;
  // K: charged, K&G: S = -1, U&G: sigma = -1; KK/UU: charged-charged and
  // magnetic-magnetic bonds, *d: those whose two signs differ
  int nK = 0, nKG = 0, nUG = 0, nKK = 0, nKKd = 0, nUU = 0, nUUd = 0, words = 0;
  int q = tid;
  int j = q / Wq, wq = q - j * Wq;
  const int sj = nthreads / Wq, sw = nthreads - sj * Wq;
#pragma unroll 2
  for (; q < nq; q += nthreads) {
    const int w0 = 4 * wq;
    const int jd = cy == 3 ? (j + 1 == g.Cy ? 0 : j + 1) : j;
    const uint4 x = *reinterpret_cast<const uint4 *>(X0 + j * W + w0);
    const uint4 r = *reinterpret_cast<const uint4 *>(R0 + j * W + w0);
    const uint4 d = *reinterpret_cast<const uint4 *>(D0 + jd * W + w0);
    // right neighbours of class column 3 are one column further on: the
    // windows start one site later (the last one wraps to the row's start)
    const uint32_t rn = cx == 3 ? R0[j * W + (w0 + 4 == W ? 0 : w0 + 4)] : 0u;
    const uint32_t xs[4] = {x.x, x.y, x.z, x.w};
    const uint32_t ds[4] = {d.x, d.y, d.z, d.w};
    const uint32_t rs[5] = {r.x, r.y, r.z, r.w, rn};
    // every mask below has even bits only, so two of them add without carries
    // into one word whose popcount is the sum of theirs (halves the popcounts)
    uint32_t mK[4], mKG[4], mUG[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t X = xs[k];
      const uint32_t K = (X >> 1) & kEven, G = X & kEven, U = ~K & kEven;
      mK[k] = K;
      mKG[k] = K & G;
      mUG[k] = U & G;
      const uint32_t Xr = cx == 3 ? __funnelshift_r(rs[k], rs[k + 1], 2) : rs[k];
      const uint32_t Xd = ds[k];
      const uint32_t KR = (Xr >> 1) & kEven, KD = (Xd >> 1) & kEven;
      const uint32_t fR = G ^ Xr, fD = G ^ Xd;  // sign bits differ (even bits)
      const uint32_t KKR = K & KR, KKD = K & KD, UUR = U & ~KR, UUD = U & ~KD;
      nKK += __popc(KKR + (KKD << 1));
      nKKd += __popc((KKR & fR) + ((KKD & fD) << 1));
      nUU += __popc(UUR + (UUD << 1));
      nUUd += __popc((UUR & fR) + ((UUD & fD) << 1));
    }
    nK += __popc(mK[0] + (mK[1] << 1)) + __popc(mK[2] + (mK[3] << 1));
    nKG += __popc(mKG[0] + (mKG[1] << 1)) + __popc(mKG[2] + (mKG[3] << 1));
    nUG += __popc(mUG[0] + (mUG[1] << 1)) + __popc(mUG[2] + (mUG[3] << 1));
    words += 4;
    wq += sw;
    j += sj;
    if (wq >= Wq) {
      wq -= Wq;
      ++j;
    }
  }
  const int sgn = ((cx + cy) & 1) ? -1 : 1;
  const int M = 16 * words - nK - 2 * nUG, S = nK - 2 * nKG;
  c[0] += nK;
  c[1] += nKK - 2 * nKKd;
  c[2] += nUU - 2 * nUUd;
  c[3] += M;
  c[4] += sgn * M;
  c[5] += S;
  c[6] += sgn * S;
}

__device__ __forceinline__ bool quads_ok(const Geo &g) {
  return (g.Cx & 15) == 0 && (g.W & 3) == 0;
}

}  // namespace ccmc
