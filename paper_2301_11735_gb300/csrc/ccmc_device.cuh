// ccmc_device.cuh -- device building blocks of the coupled-pair Metropolis
// sweep (Budrin et al., Sec. 3): counter-based random numbers, the packed
// lattice layout, the colour schedule and the per-pair move.
//
// Packed layout.  Site (x, y) belongs to residue class (x mod 4, y mod 4) and
// sits at column i = x / 4, row j = y / 4 of that class's Cy x Cx grid
// (Cx = Lx / 4, Cy = Ly / 4).  Each class row is stored as W = ceil(Cx / 16)
// 32-bit words, 16 sites per word, site i at bits 2 (i mod 16) .. +1 of word
// i / 16; the 16 classes are stored one after another (class c = 4 (y mod 4) +
// (x mod 4)).  A colour phase updates all pairs (a, a + r) with a in one class:
// the a-sites of one word are 16 pairs whose partners, and all their
// neighbours, are 16 consecutive sites of other class rows -- fetched as one
// shifted word ("window").
#pragma once

#include <cstdint>

#include "ccmc_internal.h"

namespace ccmc {

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies whose halves are cross-mixed with the key, the key advancing by
// the two Weyl constants between rounds.
struct U4 {
  uint32_t x, y, z, w;
};

// The 64-bit product of two 32-bit words as its low and high halves (one wide
// multiply instead of a low and a high one).
__device__ __forceinline__ void mul_wide(uint32_t a, uint32_t b, uint32_t &lo, uint32_t &hi) {
  uint64_t p;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(b));
  lo = (uint32_t)p;
  hi = (uint32_t)(p >> 32);
}

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    c0 = hi1 ^ c1 ^ k0;
    c2 = hi0 ^ c3 ^ k1;
    c1 = lo1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// The round keys of a seed, precomputed: round r uses (k0 + r 0x9E3779B9,
// k1 + r 0xBB67AE85).  Passed as a kernel parameter, each key is a constant
// operand of its round's XOR instead of an addition per call.
struct RoundKeys {
  uint32_t k0[10], k1[10];
};

inline RoundKeys round_keys(uint32_t k0, uint32_t k1) {
  RoundKeys rk;
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0 + (uint32_t)r * 0x9E3779B9u;
    rk.k1[r] = k1 + (uint32_t)r * 0xBB67AE85u;
  }
  return rk;
}

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     const RoundKeys &rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0, hi0, lo1, hi1;
    mul_wide(0xD2511F53u, c0, lo0, hi0);
    mul_wide(0xCD9E8D57u, c2, lo1, hi1);
    c0 = hi1 ^ c1 ^ rk.k0[r];
    c2 = hi0 ^ c3 ^ rk.k1[r];
    c1 = lo1;
    c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

// Where a kernel's Philox keys come from: the seed (keys added per round) or
// precomputed round keys.
struct SeedKeys {
  uint32_t k0, k1;
  __device__ __forceinline__ U4 operator()(uint32_t c0, uint32_t c1, uint32_t c2,
                                           uint32_t c3) const {
    return philox(c0, c1, c2, c3, k0, k1);
  }
};
struct TableKeys {
  const RoundKeys *rk;
  __device__ __forceinline__ U4 operator()(uint32_t c0, uint32_t c1, uint32_t c2,
                                           uint32_t c3) const {
    return philox(c0, c1, c2, c3, *rk);
  }
};

__device__ __forceinline__ uint32_t *row_ptr(const Geo &g, int cls, int row) {
  return g.words + (int64_t)cls * g.cstride + (int64_t)row * g.W;
}

// n (<= 16) consecutive sites of a class row starting at column `start`
// (periodic in the row), site t at bits 2t .. 2t+1.  Bits beyond 2n are
// unspecified.
__device__ __forceinline__ uint32_t fetch_window(const uint32_t *row, int W, int Cx, int start,
                                                 int n) {
  const int wi = start >> 4, o = start & 15;
  const uint32_t lo = row[wi];
  const uint32_t hi = row[(wi + 1 < W) ? wi + 1 : 0];
  uint32_t v = __funnelshift_r(lo, hi, 2 * o);
  const int n1 = Cx - start;  // sites left before the row wraps
  if (n1 < n) v = (v & ((1u << (2 * n1)) - 1u)) | (row[0] << (2 * n1));
  return v;
}

// XOR the first n sites of D into the class row at column `start` (periodic).
// Only bits of the caller's own sites are nonzero, so concurrent XORs from other
// threads into the same words commute.
__device__ __forceinline__ void scatter_xor(uint32_t *row, int Cx, int start, int n, uint32_t D) {
  if (D == 0u) return;
  const int n1 = min(n, Cx - start);
  const uint32_t d1 = (n1 < 16) ? (D & ((1u << (2 * n1)) - 1u)) : D;
  const int wi = start >> 4, o = start & 15;
  if (d1) {
    atomicXor(row + wi, d1 << (2 * o));
    if (o) {
      const uint32_t h = d1 >> (32 - 2 * o);
      if (h) atomicXor(row + wi + 1, h);
    }
  }
  if (n1 < n) {
    const uint32_t d2 = D >> (2 * n1);
    if (d2) atomicXor(row, d2);
  }
}

// ----------------------------------------------------------------------------
// Colour schedule of global phase P (Sec. 3.2, a "map" of non-interacting
// pairs): attempt t draws Philox(seed, (t, P_lo, P_hi, SCHED)); class a0 from
// the low 4 bits of word 0 and the offset index from words 1-2 by Lemire's
// multiply-high with rejection; the first attempt whose offset is allowed wins.
struct Sched {
  int a0x, a0y, rx, ry;
  int near;  // r is an exact nearest-neighbour offset: the pair shares a bond
};

__device__ __forceinline__ bool offset_allowed(int Lx, int Ly, int rx, int ry) {
  if (rx == 0 && ry == 0) return false;
  if (ry == 0 && (rx == 1 || rx == Lx - 1)) return true;
  if (rx == 0 && (ry == 1 || ry == Ly - 1)) return true;
  const int mx = rx & 3, my = ry & 3;
  if (mx == 0 && my == 0) return false;
  if (my == 0 && (mx & 1)) return false;
  if (mx == 0 && (my & 1)) return false;
  return true;
}

// Executed by one full warp; every lane returns the same schedule.
__device__ __forceinline__ Sched draw_schedule(const Geo &g, uint64_t P) {
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t N = (uint64_t)g.Lx * (uint64_t)g.Ly;
  Sched s{0, 0, 2, 2, 0};
  for (uint32_t base = 0; base < 64; base += 32) {
    const U4 w = philox(base + lane, (uint32_t)P, (uint32_t)(P >> 32), TAG_SCHED, g.k0, g.k1);
    const uint64_t x = ((uint64_t)w.z << 32) | (uint64_t)w.y;
    const uint64_t lo = x * N;
    const uint64_t idx = __umul64hi(x, N);
    const int rx = (int)(idx % (uint64_t)g.Lx);
    const int ry = (int)(idx / (uint64_t)g.Lx);
    const bool ok = (lo >= g.rej) && offset_allowed(g.Lx, g.Ly, rx, ry);
    const unsigned ballot = __ballot_sync(0xFFFFFFFFu, ok);
    if (ballot) {
      const int src = __ffs(ballot) - 1;
      s.a0x = __shfl_sync(0xFFFFFFFFu, (int)(w.x & 3u), src);
      s.a0y = __shfl_sync(0xFFFFFFFFu, (int)((w.x >> 2) & 3u), src);
      s.rx = __shfl_sync(0xFFFFFFFFu, rx, src);
      s.ry = __shfl_sync(0xFFFFFFFFu, ry, src);
      break;
    }
  }
  s.near = (s.ry == 0 && (s.rx == 1 || s.rx == g.Lx - 1)) ||
           (s.rx == 0 && (s.ry == 1 || s.ry == g.Ly - 1));
  return s;
}

// ----------------------------------------------------------------------------
// Byte permute (PTX prmt, generic mode): result byte n is source byte
// sel[4n..4n+2] of the 8 bytes {a, b}; when sel bit 4n+3 is set the byte is
// filled with the sign bit of that source byte instead.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

// Neighbour sums of 16 sites held in four neighbour windows, in 4-bit lanes:
// lane u of *_e is site 2u, of *_o site 2u + 1; value = sum over the four
// neighbours of (S + 1) (s*) or (sigma + 1) (g*), in [0, 8].
struct Sums {
  uint32_t se, so, ge, go;
};

// Each window is first rewritten in the linear code (bit 1 = charged XOR
// sign, bit 0 = sign), in which S = b1 - b0 and sigma = 1 - b1 - b0 hold for all
// four states.  Two lane sums over the neighbours, c = sum (2 b1 + b0) and
// n1 = sum b1, then give sum (S + 1) = 3 n1 - c + 4 and sum (sigma + 1) =
// n1 - c + 8.  (Lane values may overflow in between; the 32-bit results are
// exact because every final lane value lies in [0, 8].)
__device__ __forceinline__ uint32_t linear_code(uint32_t X) {
  return X ^ ((X << 1) & 0xAAAAAAAAu);
}

__device__ __forceinline__ Sums neighbour_sums(uint32_t X0, uint32_t X1, uint32_t X2,
                                               uint32_t X3) {
  const uint32_t Y0 = linear_code(X0), Y1 = linear_code(X1), Y2 = linear_code(X2),
                 Y3 = linear_code(X3);
  const uint32_t E0 = Y0 & 0x33333333u, E1 = Y1 & 0x33333333u, E2 = Y2 & 0x33333333u,
                 E3 = Y3 & 0x33333333u;
  const uint32_t O0 = (Y0 >> 2) & 0x33333333u, O1 = (Y1 >> 2) & 0x33333333u,
                 O2 = (Y2 >> 2) & 0x33333333u, O3 = (Y3 >> 2) & 0x33333333u;
  const uint32_t ce = E0 + E1 + E2 + E3, co = O0 + O1 + O2 + O3;
  const uint32_t ne = ((E0 & 0x22222222u) + (E1 & 0x22222222u) + (E2 & 0x22222222u) +
                       (E3 & 0x22222222u)) >> 1;
  const uint32_t no = ((O0 & 0x22222222u) + (O1 & 0x22222222u) + (O2 & 0x22222222u) +
                       (O3 & 0x22222222u)) >> 1;
  Sums s;
  s.se = 3u * ne + 0x44444444u - ce;
  s.so = 3u * no + 0x44444444u - co;
  s.ge = ne + 0x88888888u - ce;
  s.go = no + 0x88888888u - co;
  return s;
}

// Byte lanes of group k (sites k, k + 4, k + 8, k + 12) from 4-bit lanes.
__device__ __forceinline__ uint32_t group_bytes(uint32_t e, uint32_t o, int k) {
  const uint32_t src = (k & 1) ? o : e;
  return ((k & 2) ? (src >> 4) : src) & 0x0F0F0F0Fu;
}

}  // namespace ccmc
