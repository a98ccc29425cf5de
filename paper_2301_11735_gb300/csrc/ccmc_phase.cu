// ccmc_phase.cu -- the colour-phase kernels of the coupled-pair Metropolis
// sweep for sm_103a (one lattice per launch: direct and tile-staged; several
// lattices in lock step; the resident batch kernel) and their launchers
// (declared in ccmc_internal.h).
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "ccmc_count.cuh"
#include "ccmc_device.cuh"
#include "ccmc_internal.h"
#include "ccmc_launch.cuh"

namespace ccmc {

// ============================================================================
// One colour phase (Sec. 3.1-3.2).  A word of the a-class holds 16 pairs
// (a, a + r), site t of the word at bits 2t..2t+1.  Its pairs are read as the
// a word, the four neighbour windows of a, the b window and the four neighbour
// windows of b; every pair's move is evaluated; the a word is stored and the
// changed b sites are XORed back.
//
// Random fields: pair t takes the 16-bit half (t mod 2) of word (t / 4) mod 4
// of MOVE call c = (t / 2) mod 2 of its word, i.e. call c serves the pair
// groups k = 2c (low halves) and k = 2c + 1 (high halves), group k being the
// sites k, k + 4, k + 8, k + 12 (lane q = site / 4).  Per pair, with pc =
// 4 code_a + code_b and its field v:
//   w      = floor(v / 12), the choice class v - 12 w (v < 65532 = 12 x 5461)
//   entry  = trans[v - 12 w][near][pc] -> base, byte coefficients, pc XOR npc
//   index  = dp4a(coefficients, (D8, GA, GB, 0), base)  (threshold index)
//   accept = w < T[index], with T = floor(5461 thr / 2^32) (5461 when thr is
//            0xFFFFFFFF): w < T implies w 2^32 + s < 5461 thr for every 32-bit
//            s, w > T the opposite
// The fast decision is always applied.  A tie (w == T) or a field v >= 65532
// sends the call's pairs through the exact path, which decides each truly rare
// pair (the fast path rejected it) with its SLOW random words (about one pair
// in 4000).
struct PhaseSmem {
  uint2 trans[kMoveN];
  uint16_t thrT[kThrT];
  Sched sched;
};

// Uniform per phase: where the ten windows of a word come from.  Column offsets
// are in sites, normalised to [0, Cx).
struct PhaseU {
  const uint32_t *cA, *cAL, *cAR, *cAU, *cAD, *cB, *cBL, *cBR, *cBU, *cBD;
  int offAL, offAR, offB, offBL, offBR;
  int dyAU, dyAD, qy, dyBU, dyBD;
  int wmask;  // W - 1 (rows of power-of-two width only)
};

// How the word code reads its windows: rows of any width (kRowGeneral), rows
// of whole words (kRowAligned), or rows of whole words and power-of-two width
// W, staged as bands whose first row is the tile's first row (kRowTile: column
// wraps are masks and every row offset dy is 0).
enum RowMode { kRowGeneral = 0, kRowAligned = 1, kRowTile = 2 };

__device__ __forceinline__ int wrap(int v, int n) { return v >= n ? v - n : (v < 0 ? v + n : v); }

__device__ __forceinline__ PhaseU phase_uniform(const Geo &g, const Sched &sc) {
  PhaseU u;
  const int ax = sc.a0x, ay = sc.a0y;
  const int bxx = ax + sc.rx, byy = ay + sc.ry;
  const int cbx = bxx & 3, cby = byy & 3;
  auto cls = [&](int cx, int cy) { return g.words + (int64_t)(cy * 4 + cx) * g.cstride; };
  u.cA = cls(ax, ay);
  u.cAL = cls((ax + 3) & 3, ay);
  u.cAR = cls((ax + 1) & 3, ay);
  u.cAU = cls(ax, (ay + 3) & 3);
  u.cAD = cls(ax, (ay + 1) & 3);
  u.cB = cls(cbx, cby);
  u.cBL = cls((cbx + 3) & 3, cby);
  u.cBR = cls((cbx + 1) & 3, cby);
  u.cBU = cls(cbx, (cby + 3) & 3);
  u.cBD = cls(cbx, (cby + 1) & 3);
  const int qx = (bxx >> 2) % g.Cx;
  u.offAL = ax == 0 ? g.Cx - 1 : 0;
  u.offAR = ax == 3 ? (g.Cx == 1 ? 0 : 1) : 0;
  u.offB = qx;
  u.offBL = cbx == 0 ? wrap(qx - 1, g.Cx) : qx;
  u.offBR = cbx == 3 ? wrap(qx + 1, g.Cx) : qx;
  u.dyAU = ay == 0 ? -1 : 0;
  u.dyAD = ay == 3 ? 1 : 0;
  u.qy = (byy >> 2) % g.Cy;
  u.dyBU = cby == 0 ? -1 : 0;
  u.dyBD = cby == 3 ? 1 : 0;
  u.wmask = g.W - 1;
  return u;
}

// Window of n sites at column 16 w + off (mod Cx) of one class row.
template <int kMode>
__device__ __forceinline__ uint32_t window(const uint32_t *cls, const Geo &g, const PhaseU &u,
                                           int row, int w, int off, int n) {
  const uint32_t *r = cls + row * g.W;
  if constexpr (kMode == kRowTile) {
    const int wl = (w + (off >> 4)) & u.wmask;
    return __funnelshift_r(r[wl], r[(wl + 1) & u.wmask], 2 * (off & 15));
  } else if constexpr (kMode == kRowAligned) {  // the window straddles at most two words
    const int wl = wrap(w + (off >> 4), g.W);
    const int sh = 2 * (off & 15);
    if (sh == 0) return r[wl];
    const int wh = wl + 1 == g.W ? 0 : wl + 1;
    return __funnelshift_r(r[wl], r[wh], sh);
  } else {
    return fetch_window(r, g.W, g.Cx, wrap(16 * w + off, g.Cx), n);
  }
}

// Move entry of choice class r (v mod 12) and pc8 = 8 pc + 128 near: entry
// (2 r + near) 16 + (pc XOR r) of the move table, at byte offset
// 256 r + 128 near + 8 (pc XOR r) = (264 r) XOR pc8.  The XOR spreads a warp's
// lookups over the banks: with entry (2 r + near) 16 + pc the bank pair of a
// lookup was its pair state alone, and the few common states (both sites
// magnetic) piled onto four of sixteen bank pairs.  Word 0: the threshold
// index's base; word 1: the signed byte coefficients of (D8, GA, GB) and, at
// bits 24-27 (the byte dp4a multiplies by zero), the move pc XOR npc.
__device__ __forceinline__ uint2 move_entry(const uint2 *trans, uint32_t r, uint32_t pc8) {
  return *reinterpret_cast<const uint2 *>(reinterpret_cast<const char *>(trans) +
                                          ((r * 264u) ^ pc8));
}

// floor(v / 12) for v < 2^16 by a multiply-high: floor(v m / 2^32) with
// m = ceil(2^32 / 12) is exact there.
__device__ __forceinline__ uint32_t div12(uint32_t v) { return __umulhi(v, 357913942u); }

// The pair's move nibble (a bits 2-3, b bits 0-1) in an entry's word 1.
__device__ __forceinline__ uint32_t move_nibble(uint32_t ey) { return (ey >> 24) & 15u; }

// Byte lanes of one pair group (sites k, k + 4, k + 8, k + 12): x01/x23 hold
// (D8, GA) of lanes 0, 1 / 2, 3, gb the GB of its four lanes, pc8 the
// move-table offsets 8 pc + near128.
struct Group {
  uint32_t x01, x23, gb, pc8;
};

__device__ __forceinline__ Group group_env(const Sums &sa, const Sums &sb, uint32_t pcE,
                                           uint32_t pcO, uint32_t near128, int k) {
  const uint32_t d8 = group_bytes(sa.se, sa.so, k) + 0x08080808u - group_bytes(sb.se, sb.so, k);
  const uint32_t ga = group_bytes(sa.ge, sa.go, k);
  Group gr;
  gr.gb = group_bytes(sb.ge, sb.go, k);
  gr.x01 = prmt(d8, ga, 0x5140u);
  gr.x23 = prmt(d8, ga, 0x7362u);
  gr.pc8 = group_bytes(pcE, pcO, k) * 8u + near128 * 0x01010101u;
  return gr;
}

// dp4a operand (D8, GA, GB, 0) of lane q of a group (q a compile-time constant
// in the unrolled loops).
__device__ __forceinline__ uint32_t lane_env(const Group &gr, int q) {
  return q == 0 ? prmt(gr.x01, gr.gb, 0x8410u)
       : q == 1 ? prmt(gr.x01, gr.gb, 0x8532u)
       : q == 2 ? prmt(gr.x23, gr.gb, 0x8610u)
                : prmt(gr.x23, gr.gb, 0x8732u);
}

// The inputs of a word's pairs: its a word, its b window and the neighbour
// sums of both sides.
struct WordIn {
  uint32_t A, B;
  Sums sa, sb;
};

// Row jr + dy of a class (periodic in Cy); staged bands start at the right row.
template <int kMode>
__device__ __forceinline__ int band_row(const Geo &g, int r0, int dy) {
  return kMode == kRowTile ? r0 : wrap(r0 + dy, g.Cy);
}

// n: the word's sites inside its row (16 unless the row ends in it).
template <int kMode>
__device__ __forceinline__ WordIn gather(const Geo &g, const PhaseU &u, int jr, int w, int n) {
  WordIn in;
  in.A = u.cA[jr * g.W + w];
  const int jb = band_row<kMode>(g, jr, u.qy);
  in.B = window<kMode>(u.cB, g, u, jb, w, u.offB, n);
  in.sa = neighbour_sums(window<kMode>(u.cAL, g, u, jr, w, u.offAL, n),
                         window<kMode>(u.cAR, g, u, jr, w, u.offAR, n),
                         u.cAU[band_row<kMode>(g, jr, u.dyAU) * g.W + w],
                         u.cAD[band_row<kMode>(g, jr, u.dyAD) * g.W + w]);
  in.sb = neighbour_sums(window<kMode>(u.cBL, g, u, jb, w, u.offBL, n),
                         window<kMode>(u.cBR, g, u, jb, w, u.offBR, n),
                         window<kMode>(u.cBU, g, u, band_row<kMode>(g, jb, u.dyBU), w, u.offB, n),
                         window<kMode>(u.cBD, g, u, band_row<kMode>(g, jb, u.dyBD), w, u.offB, n));
  return in;
}

__device__ __forceinline__ uint32_t pcE_of(const WordIn &in) {
  return ((in.A & 0x33333333u) << 2) | (in.B & 0x33333333u);
}
__device__ __forceinline__ uint32_t pcO_of(const WordIn &in) {
  return (in.A & 0xCCCCCCCCu) | ((in.B >> 2) & 0x33333333u);
}

// The fast path of the pairs of a word one thread evaluates: kTPW threads
// share a word (1, 2 or 4), thread `sub` of them takes MOVE call(s) and
// half(s):
//   kTPW 1: both calls, both halves (all 16 pairs);
//   kTPW 2: call sub, both halves (8 pairs);
//   kTPW 4: call sub / 2, half sub mod 2 (4 pairs: group k = sub).
// Returns the (dA, dB) of the fast decisions and, in z, bit c for every call
// c with a rare pair (a tie or a field >= 65532; the fast path rejected it).
template <int kTPW, class Keys>
__device__ __forceinline__ uint3 fast_moves(const Geo &g, const uint2 *trans,
                                            const uint16_t *thrT, int j, int w, int sub,
                                            const WordIn &in, uint64_t P, uint32_t near128,
                                            const Keys &keys) {
  static_assert(kTPW == 1 || kTPW == 2 || kTPW == 4, "one, two or four threads a word");
  constexpr int kCalls = kTPW == 1 ? 2 : 1;
  constexpr int kHalves = kTPW == 4 ? 1 : 2;
  const int c0 = kTPW == 1 ? 0 : (kTPW == 2 ? sub : sub >> 1);
  const int h0 = kTPW == 4 ? (sub & 1) : 0;
  const uint32_t pcE = pcE_of(in), pcO = pcO_of(in);
  const uint32_t gbase = (uint32_t)j * (uint32_t)(2 * g.W) + (uint32_t)(2 * w);
  uint32_t dA = 0u, dB = 0u, slow = 0u;
#pragma unroll
  for (int ci = 0; ci < kCalls; ++ci) {
    const int c = c0 + ci;
    const U4 r = keys(gbase + (uint32_t)c, (uint32_t)P, (uint32_t)(P >> 32), TAG_MOVE);
    uint32_t mn = 0xFFFFFFFFu, mx = 0u;  // smallest w - T, largest v of the call
#pragma unroll
    for (int hi = 0; hi < kHalves; ++hi) {
      const int h = h0 + hi;
      const int k = 2 * c + h;
      const Group gr = group_env(in.sa, in.sb, pcE, pcO, near128, k);
      uint32_t acc = 0u;  // byte q: the accepted move of lane q
      uint32_t d0 = 0xFFFFFFFFu, v0 = 0u;
#pragma unroll
      for (int q = 3; q >= 0; --q) {
        const uint32_t X = q == 0 ? r.x : q == 1 ? r.y : q == 2 ? r.z : r.w;
        const uint32_t v = h ? X >> 16 : X & 0xFFFFu;
        const uint32_t wq = div12(v);
        const uint2 e = move_entry(trans, v - 12u * wq, prmt(gr.pc8, 0u, 0x4440u + (uint32_t)q));
        const uint32_t T = thrT[__dp4a((int)e.y, (int)lane_env(gr, q), (int)e.x)];
        const uint32_t d = wq - T;  // negative: accept; zero: a tie
        if (q & 1) {
          d0 = d;
          v0 = v;
        } else {
          mn = __vimin3_u32(mn, d0, d);
          mx = __vimax3_u32(mx, v0, v);
        }
        acc = __funnelshift_l((int)d < 0 ? e.y : 0u, acc, 8);
      }
      // byte q of acc -> site k + 4 q: b bits to 2 (k + 4 q) of dB, a bits of dA
      dB |= (acc & 0x03030303u) << (2 * k);
      dA |= ((acc >> 2) & 0x03030303u) << (2 * k);
    }
    if (mn == 0u || mx >= 65532u) slow |= 1u << c;
  }
  return make_uint3(dA, dB, slow);
}

// Apply the moves (dA, dB) of word w (row jr of u's arrays, n sites): the a
// word by a plain read-modify-write when this thread owns it (kOwnA), else by
// atomic XOR; the b sites by atomic XOR (their words are shared with the
// partners of neighbouring words).
template <int kMode, bool kOwnA>
__device__ __forceinline__ void apply_moves(const Geo &g, const PhaseU &u, int jr, int w, int n,
                                            uint32_t dA, uint32_t dB) {
  if constexpr (kMode == kRowGeneral) {
    if (n < 16) {  // pairs past the end of the row do not exist
      const uint32_t valid = (1u << (2 * n)) - 1u;
      dA &= valid;
      dB &= valid;
    }
  }
  if (dA) {
    uint32_t *pa = const_cast<uint32_t *>(u.cA) + jr * g.W + w;
    if constexpr (kOwnA)
      *pa ^= dA;
    else
      atomicXor(pa, dA);
  }
  if (dB) {
    uint32_t *rb = const_cast<uint32_t *>(u.cB) + band_row<kMode>(g, jr, u.qy) * g.W;
    if constexpr (kMode == kRowTile) {
      const int wl = (w + (u.offB >> 4)) & u.wmask;
      const int sh = 2 * (u.offB & 15);
      atomicXor(rb + wl, dB << sh);
      if (sh) {
        const uint32_t hi = dB >> (32 - sh);
        if (hi) atomicXor(rb + ((wl + 1) & u.wmask), hi);
      }
    } else if constexpr (kMode == kRowAligned) {
      const int wl = wrap(w + (u.offB >> 4), g.W);
      const int sh = 2 * (u.offB & 15);
      atomicXor(rb + wl, dB << sh);
      if (sh) {
        const uint32_t hi = dB >> (32 - sh);
        if (hi) atomicXor(rb + (wl + 1 == g.W ? 0 : wl + 1), hi);
      }
    } else {
      scatter_xor(rb, g.Cx, wrap((w << 4) + u.offB, g.Cx), n, dB);
    }
  }
}

// The exact path of one pair, by one lane of a warp that takes the rare calls
// of a word together: pair t = k + 4 q (group k = 2 c + h, lane q of the
// group) of MOVE call c of word w (inputs `in`, n sites in the row), decided
// with its SLOW words if it is rare (the fast path rejected it), and applied
// to the word's a and b sites by atomic XOR.
template <int kMode>
__device__ __forceinline__ void exact_pair(const Geo &g, const PhaseU &u, const uint2 *trans,
                                           const uint16_t *thrT, const uint32_t *thr32, int j,
                                           int jr, int w, int n, int c, int h, int q,
                                           const WordIn &in, uint64_t P, uint32_t near128) {
  const int k = 2 * c + h;
  const int t = k + 4 * q;
  if (t >= n) return;  // past the end of the row: no pair
  const uint32_t gbase = (uint32_t)j * (uint32_t)(2 * g.W) + (uint32_t)(2 * w);
  const U4 r = philox(gbase + (uint32_t)c, (uint32_t)P, (uint32_t)(P >> 32), TAG_MOVE, g.k0, g.k1);
  const uint32_t X = q == 0 ? r.x : q == 1 ? r.y : q == 2 ? r.z : r.w;
  const uint32_t v = h ? X >> 16 : X & 0xFFFFu;
  const uint32_t wq = div12(v);
  const Group gr = group_env(in.sa, in.sb, pcE_of(in), pcO_of(in), near128, k);
  const uint32_t pc8 = prmt(gr.pc8, 0u, 0x4440u + (uint32_t)q);
  const uint32_t env = prmt(q < 2 ? gr.x01 : gr.x23, gr.gb,
                            0x8410u + ((q & 1) ? 0x0122u : 0u) + ((q & 2) ? 0x0200u : 0u));
  uint2 e = move_entry(trans, v - 12u * wq, pc8);
  if (v < 65532u && wq != thrT[__dp4a((int)e.y, (int)env, (int)e.x)]) return;  // not rare
  const uint32_t slow0 = (uint32_t)((uint64_t)j * g.Cx + (uint32_t)(w << 4));
  const U4 sl = philox(slow0 + (uint32_t)t, (uint32_t)P, (uint32_t)(P >> 32), TAG_SLOW, g.k0, g.k1);
  if (v >= 65532u) {
    if (sl.y >= 4294967292u) return;  // keep the current configuration
    e = move_entry(trans, sl.y % 12u, pc8);
  }
  const uint32_t thr = thr32[__dp4a((int)e.y, (int)env, (int)e.x)];
  const bool accept = thr == 0xFFFFFFFFu ||
                      (v < 65532u ? ((uint64_t)wq << 32) + sl.x < 5461ull * thr : sl.x < thr);
  if (accept) {
    const uint32_t x = move_nibble(e.y);
    apply_moves<kMode, false>(g, u, jr, w, n, (x >> 2) << (2 * t), (x & 3u) << (2 * t));
  }
}

// One word's pairs by one lane, with all 32 lanes of the warp calling
// together (inactive lanes: active false): the fast decisions are applied;
// then, for every lane with rare calls (about one word in 250), the warp
// decides that word's rare pairs together, one pair a lane, from the owner's
// inputs.  The rare pairs were rejected by the fast path, and no other pair of
// the phase touches their sites or neighbours, so the order does not matter.
// j: the a word's row in the class (keys the random streams); jr: its row in
// u's arrays (j itself for a lattice in global memory, the row inside a
// staged tile otherwise); near128: 128 if the phase's partners are nearest
// neighbours, else 0; keys: the source of the Philox keys (SeedKeys or
// TableKeys of the lattice's seed); kTPW threads share the word, this lane is
// thread `sub` of them (see fast_moves).
template <int kMode, int kTPW = 1, class Keys = SeedKeys>
__device__ __forceinline__ void warp_word(const Geo &g, const PhaseU &u, const uint2 *trans,
                                          const uint16_t *thrT, const uint32_t *thr32, int j,
                                          int jr, int w, uint64_t P, uint32_t near128,
                                          const Keys &keys, int sub = 0, bool active = true) {
  const int n = active ? (kMode == kRowGeneral ? min(16, g.Cx - (w << 4)) : 16) : 0;
  WordIn in{};
  uint32_t rz = 0u;
  if (active) {
    in = gather<kMode>(g, u, jr, w, n);
    const uint3 d = fast_moves<kTPW>(g, trans, thrT, j, w, sub, in, P, near128, keys);
    apply_moves<kMode, kTPW == 1>(g, u, jr, w, n, d.x, d.y);
    rz = d.z;
  }
  unsigned ball = __ballot_sync(0xFFFFFFFFu, rz != 0u);
  if (ball) {
    const int lane = threadIdx.x & 31;
    __syncwarp();  // the fast moves of every lane are in memory
#pragma unroll 1
    while (ball) {
      const int src = __ffs(ball) - 1;
      ball &= ball - 1u;
      const uint32_t orz = __shfl_sync(0xFFFFFFFFu, rz, src);
      WordIn o;
      o.A = __shfl_sync(0xFFFFFFFFu, in.A, src);
      o.B = __shfl_sync(0xFFFFFFFFu, in.B, src);
      o.sa.se = __shfl_sync(0xFFFFFFFFu, in.sa.se, src);
      o.sa.so = __shfl_sync(0xFFFFFFFFu, in.sa.so, src);
      o.sa.ge = __shfl_sync(0xFFFFFFFFu, in.sa.ge, src);
      o.sa.go = __shfl_sync(0xFFFFFFFFu, in.sa.go, src);
      o.sb.se = __shfl_sync(0xFFFFFFFFu, in.sb.se, src);
      o.sb.so = __shfl_sync(0xFFFFFFFFu, in.sb.so, src);
      o.sb.ge = __shfl_sync(0xFFFFFFFFu, in.sb.ge, src);
      o.sb.go = __shfl_sync(0xFFFFFFFFu, in.sb.go, src);
      const int oj = __shfl_sync(0xFFFFFFFFu, j, src), ojr = __shfl_sync(0xFFFFFFFFu, jr, src),
                ow = __shfl_sync(0xFFFFFFFFu, w, src), on = __shfl_sync(0xFFFFFFFFu, n, src);
      // the owner's pairs, one a lane: 16 (both calls), 8 (one call) or 4
      int c, h;
      if constexpr (kTPW == 1) {
        c = (lane >> 3) & 1;
        h = (lane >> 2) & 1;
      } else {
        const int osub = __shfl_sync(0xFFFFFFFFu, sub, src);
        c = kTPW == 2 ? osub : osub >> 1;
        h = kTPW == 2 ? (lane >> 2) & 1 : osub & 1;
      }
      if (lane < 16 / kTPW && ((orz >> c) & 1u))
        exact_pair<kMode>(g, u, trans, thrT, thr32, oj, ojr, ow, on, c, h, lane & 3, o, P,
                          near128);
    }
  }
}

template <bool kAligned>
__global__ void __launch_bounds__(256, 4) phase_kernel(Geo g, const uint16_t *thrT,
                                                    const uint32_t *thr32, const uint32_t *trans,
                                                    int64_t p_off) {
  __shared__ PhaseSmem sm;
  // The tables come from host uploads that precede the whole launch chain, so
  // they are loaded before waiting for the previous kernel of the stream (which
  // lets this prologue overlap its tail under programmatic dependent launch).
  for (int t = threadIdx.x; t < kThrT / 2; t += blockDim.x)
    reinterpret_cast<uint32_t *>(sm.thrT)[t] = reinterpret_cast<const uint32_t *>(thrT)[t];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // The next kernel may launch now: with one resident wave its blocks only take
  // the slots of blocks that finish, and it waits for this whole grid before
  // touching the lattice.
  asm volatile("griddepcontrol.launch_dependents;");
  const uint64_t P = (uint64_t)(g.ctl[kCtlPhaseBase] + p_off);
  if (threadIdx.x < 32) {
    const Sched s = draw_schedule(g, P);
    if (threadIdx.x == 0) sm.sched = s;
  }
  __syncthreads();
  const Sched sc = sm.sched;
  for (int t = threadIdx.x; t < kMoveN; t += blockDim.x)
    sm.trans[t] = make_uint2(trans[2 * t], trans[2 * t + 1]);
  __syncthreads();
  const PhaseU u = phase_uniform(g, sc);
  const uint32_t near128 = sc.near ? 128u : 0u;
  const int nw = g.Cy * g.W;
  const int stride = gridDim.x * blockDim.x;
  // a trip count uniform across the block, so that every warp's lanes stay
  // together for the cooperative exact path
  for (int base = blockIdx.x * blockDim.x; base < nw; base += stride) {
    const int wid = base + threadIdx.x;
    const bool act = wid < nw;
    const int j = act ? wid / g.W : 0, w = act ? wid - j * g.W : 0;
    warp_word<kAligned ? kRowAligned : kRowGeneral>(g, u, sm.trans, sm.thrT, thr32, j, j, w, P,
                                                     near128, SeedKeys{g.k0, g.k1}, 0, act);
  }
}

// ----------------------------------------------------------------------------
// Tile-staged phase (lattices whose class rows are W words with W dividing 256
// and a multiple of 4, and Cy a multiple of R = 256 / W).  A tile is R
// consecutive rows of the a-class (256 words, one per thread).  CTA c takes
// tiles c, c + grid, ... c + (kBufs - 1) grid first, then claims tiles beyond
// kBufs grid one at a time from a counter in the lattice's control block, so
// that CTAs which start late (placed on an SM whose previous CTA finished
// last) take fewer tiles instead of ending the phase late.  The claim for a
// buffer is made when the buffer is refilled, kBufs - 1 tiles ahead of its
// use, so its latency is hidden.  Phase P claims from slot P mod 2; its kernel
// tags slot (P + 1) mod 2 for phase P + 1 (with P + 1 in the high word) once
// phase P - 1 is done with it; a slot whose tag is not the phase's own (the
// previous phase ran on another path, or the phase counter was just set: that
// zeroes both slots) makes every CTA of the phase keep to the fixed order c +
// t grid.  A tile's ten row bands -- the a rows,
// the b rows and the rows of all eight neighbour classes, each band R full
// rows -- arrive in shared memory by bulk asynchronous copies (one band per
// lane of the staging warp) that complete on the buffer's `full` mbarrier.
// The threads evaluate their words from shared memory.  The last warp to
// finish a tile (counted on the buffer's arrival counter) sends its a and b
// bands back to global memory with plain vector stores and stages the tile
// kBufs later into the same buffer, so every buffer is refilled as soon as it
// is free, kBufs - 1 tiles ahead of its use, and no warp waits for another
// warp except on a tile's data.  (A fixed staging thread that first evaluated
// its own word trailed the slowest warp every tile; the other warps' polls
// then starved it of issue slots: first tiles landed 2.6 to 19 us after a
// phase started.)  Waits suspend in hardware (try_wait with a time hint)
// instead of spinning.  No two tiles of a phase write the same rows (each b
// row is the partner row of exactly one a row), and no tile reads a row
// another tile writes (the pairs of a phase do not interact), so global memory
// sees no atomics and staging may run ahead of the write-back.
constexpr int kTileWords = 256;
constexpr int kBands = 10;
constexpr int kTileBufs = 3;
constexpr uint32_t kTileBytes = kBands * kTileWords * 4;
constexpr uint32_t kWaitSpins = 1u << 24;              // bounded mbarrier waits:
constexpr unsigned long long kWaitNs = 1000000000ull;  // at most 2^24 polls or 1 s
constexpr uint32_t kSuspendNs = 20000;                 // suspend-time hint of a poll

// The lattice's threshold levels and the move table, contiguous in device
// memory (thrT, trans), staged with one bulk copy.
constexpr uint32_t kStagedTableBytes = 2u * kThrT + 8u * kMoveN;
static_assert(kStagedTableBytes % 16 == 0, "bulk copies move multiples of 16 bytes");

// Row band: R rows of one class starting at row j0 + dy of the tile's first a
// row j0 (periodic in Cy).
struct Band {
  const uint32_t *cls;
  int dy;
};

// kBufs: band buffers (three for the pipelined tile loop, one for a CTA that
// takes a single tile).
template <int kBufs = kTileBufs>
struct TileSmem {
  alignas(128) uint16_t thrT[kThrT];
  uint2 trans[kMoveN];  // directly after thrT, as in device memory
  alignas(128) uint32_t band[kBufs][kBands][kTileWords];
  alignas(8) unsigned long long full[kBufs];  // bands landed (transaction count)
  alignas(8) unsigned long long tables;       // the tables landed
  int done[kBufs];     // warps finished with the buffer's tile
  int armed[kBufs];    // times the buffer's `full` barrier was armed
  int tile[kBufs];     // the tile staged in the buffer, -1: no more tiles
  Band bands[kBands];
  Sched sched;
  int err;
  int busy0, busy1;  // classes the previous phase writes (early staging waits for them)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of parity `parity` of the mbarrier at `bar` to complete:
// true when it did, false after kWaitSpins polls or kWaitNs nanoseconds.  Each
// poll may suspend the thread (up to kSuspendNs) until the phase completes.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (uint32_t i = 0; i < kWaitSpins; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kSuspendNs)
        : "memory");
    if (ok) return true;
    if ((i & 63u) == 0) {
      const unsigned long long t = global_ns();
      if (i == 0)
        t0 = t;
      else if (t - t0 > kWaitNs)
        return false;
    }
  }
  return false;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      :
      : "r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// One tile-staged phase of lattice g by CTA `cta` of the `ncta` CTAs that
// work on it; keys: the source of its Philox keys.
// kSingle: every CTA takes at most one tile (ncta == tiles): one band buffer.
// kTPW: threads a word (the CTA has kTileWords kTPW threads; see fast_moves).
template <bool kSingle, int kTPW, class Keys>
__device__ __forceinline__ void tile_phase(const Geo &g, const uint16_t *thrT,
                                           const uint32_t *thr32, int64_t p_off, int cta,
                                           int ncta, const Keys &keys) {
  extern __shared__ __align__(128) unsigned char tile_smem[];
  constexpr int kBufs = kSingle ? 1 : kTileBufs;
  constexpr int kWarps = kTileWords * kTPW / 32;
  using Smem = TileSmem<kBufs>;
  Smem &sm = *reinterpret_cast<Smem *>(tile_smem);
  static_assert(offsetof(Smem, trans) == 2 * kThrT, "tables staged as one block");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    sm.err = 0;
    for (int b = 0; b < kBufs; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.full[b])));
      sm.done[b] = 0;
      sm.armed[b] = 0;
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.tables)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // The tables come from host uploads that precede the whole launch chain:
    // their copy may start before the previous kernel of the stream finishes.
    const uint32_t bar = smem_u32(&sm.tables);
    mbar_expect(bar, kStagedTableBytes);
    bulk_load(smem_u32(sm.thrT), thrT, kStagedTableBytes, bar);
  }
  // The phase index.  A launch after the first of a chain (p_off > 0) reads the
  // counter base, draws its schedule and places its bands before it waits for
  // its predecessor: the base was written by a kernel at least two launches
  // back (the chain's counter advance), which the predecessor's
  // griddepcontrol.wait has already waited for.  With several tiles a CTA it
  // then stages the bands of its first tiles that lie in classes the
  // predecessor (phase P - 1, whose schedule it draws too) does not write,
  // while that phase is still finishing, and the other bands once it has
  // finished.  Only lattices whose phases give every CTA several tiles do
  // this: for smaller ones it measured slower when several lattices share the
  // GPU on their own streams.
  const bool pre = p_off > 0;
  const bool early = !kSingle && pre && g.Cy / (kTileWords / g.W) > ncta;
  if (!pre) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
  }
  const uint64_t P = (uint64_t)(g.ctl[kCtlPhaseBase] + p_off);
  if (warp == 0) {
    const Sched sc = draw_schedule(g, P);
    if (early) {
      const Sched pv = draw_schedule(g, P - 1u);
      if (lane == 0) {
        sm.busy0 = pv.a0y * 4 + pv.a0x;
        sm.busy1 = ((pv.a0y + pv.ry) & 3) * 4 + ((pv.a0x + pv.rx) & 3);
      }
    }
    if (lane == 0) {
      sm.sched = sc;
      const PhaseU u0 = phase_uniform(g, sc);
      const Band bs[kBands] = {{u0.cA, 0},       {u0.cAL, 0},       {u0.cAR, 0},
                               {u0.cAU, u0.dyAU}, {u0.cAD, u0.dyAD}, {u0.cB, u0.qy},
                               {u0.cBL, u0.qy},   {u0.cBR, u0.qy},   {u0.cBU, u0.qy + u0.dyBU},
                               {u0.cBD, u0.qy + u0.dyBD}};
      for (int k = 0; k < kBands; ++k) sm.bands[k] = bs[k];
    }
  }
  __syncthreads();
  const Sched sc = sm.sched;
  const uint32_t near128 = sc.near ? 128u : 0u;
  const PhaseU u = phase_uniform(g, sc);
  const int W = g.W, R = kTileWords / W, Cy = g.Cy;
  const int ntiles = Cy / R;
  const uint32_t row_bytes = (uint32_t)W * 4u;

  // lane `lane` (< kBands) of the calling warp: the bulk loads of band `lane`
  // of tile `tile` into buffer b, if `mask` selects it
  auto stage_band = [&](int tile, int b, unsigned mask) {
    if (lane < kBands && ((mask >> lane) & 1u)) {
      const Band bd = sm.bands[lane];
      const int j0 = tile * R;
      int r0 = j0 + bd.dy;  // in [-Cy, 2 Cy)
      r0 = r0 < 0 ? r0 + Cy : (r0 >= Cy ? r0 - Cy : r0);
      const int n1 = min(R, Cy - r0);
      const uint32_t bar = smem_u32(&sm.full[b]);
      const uint32_t dst = smem_u32(&sm.band[b][lane][0]);
      bulk_load(dst, bd.cls + (int64_t)r0 * W, (uint32_t)n1 * row_bytes, bar);
      if (n1 < R)
        bulk_load(dst + (uint32_t)n1 * row_bytes, bd.cls, (uint32_t)(R - n1) * row_bytes, bar);
    }
  };
  // lane 0 of the calling warp arms buffer b for tile `tile` (its ten bands'
  // bytes), or marks it empty (tile < 0: the barrier completes at once)
  auto arm = [&](int tile, int b) {
    if (lane == 0) {
      ++sm.armed[b];
      sm.tile[b] = tile;
      if (tile >= 0)
        mbar_expect(smem_u32(&sm.full[b]), kTileBytes);
      else
        mbar_arrive(smem_u32(&sm.full[b]));
    }
    __syncwarp();
  };
  // the first kBufs tiles are fixed (cta + i ncta), staged by warp 0
  auto first_tile = [&](int i) { return cta + i * ncta < ntiles ? cta + i * ncta : -1; };
  if (early) {
    unsigned busy = 0u;  // bands in the classes the previous phase writes
    for (int k = 0; k < kBands; ++k)
      if (sm.bands[k].cls == g.words + (int64_t)sm.busy0 * g.cstride ||
          sm.bands[k].cls == g.words + (int64_t)sm.busy1 * g.cstride)
        busy |= 1u << k;
    if (warp == 0) {
      for (int i = 0; i < kBufs; ++i) {
        arm(first_tile(i), i);
        if (first_tile(i) >= 0) stage_band(first_tile(i), i, ~busy & ((1u << kBands) - 1u));
      }
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    if (warp == 0)
      for (int i = 0; i < kBufs; ++i)
        if (first_tile(i) >= 0) stage_band(first_tile(i), i, busy);
  } else {
    if (pre) {
      asm volatile("griddepcontrol.wait;" ::: "memory");
      asm volatile("griddepcontrol.launch_dependents;");
    }
    if (warp == 0)
      for (int i = 0; i < kBufs; ++i) {
        arm(first_tile(i), i);
        if (first_tile(i) >= 0) stage_band(first_tile(i), i, (1u << kBands) - 1u);
      }
  }
  // phase P - 1 is done (griddepcontrol.wait): tag the claim slot of phase P + 1
  if (!kSingle && cta == 0 && threadIdx.x == 0)
    *reinterpret_cast<volatile unsigned long long *>(g.ctl + kCtlTileClaim + ((P + 1u) & 1u)) =
        (unsigned long long)(uint32_t)(P + 1u) << 32;
  if (!mbar_wait(smem_u32(&sm.tables), 0u)) sm.err = 1;

  const int lw = __ffs(W) - 1;  // W is a power of two
  const int wi = (int)threadIdx.x / kTPW, sub = (int)threadIdx.x % kTPW;  // word of the tile
  const int jr = wi >> lw, w = wi & (W - 1);
  // a tile's bands in buffer b as the windows' sources
  auto local_u = [&](int b) {
    const uint32_t *base = sm.band[b][0];
    PhaseU lu = u;
    lu.cA = base;
    lu.cAL = base + 1 * kTileWords;
    lu.cAR = base + 2 * kTileWords;
    lu.cAU = base + 3 * kTileWords;
    lu.cAD = base + 4 * kTileWords;
    lu.cB = base + 5 * kTileWords;
    lu.cBL = base + 6 * kTileWords;
    lu.cBR = base + 7 * kTileWords;
    lu.cBU = base + 8 * kTileWords;
    lu.cBD = base + 9 * kTileWords;
    return lu;
  };
  int b = 0;
  for (int t = 0;; ++t) {
    // (1) evaluate this thread's word of the tile in buffer b, if any
    if (!mbar_wait(smem_u32(&sm.full[b]), (uint32_t)(t / kBufs) & 1u)) {
      sm.err = 1;
      break;
    }
    const int tile = sm.tile[b];
    if (tile < 0) break;
    warp_word<kRowTile, kTPW>(g, local_u(b), sm.trans, sm.thrT, thr32, tile * R + jr, jr, w, P,
                              near128, keys, sub);
    // (2) this warp is done with the tile: its shared-memory writes are ordered
    // before the async copies that will refill the buffer, and before the
    // last warp's reads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    int last = 0;
    if (lane == 0) {
      __threadfence_block();
      last = atomicAdd(&sm.done[b], 1) == kWarps - 1;
      if (last) __threadfence_block();
    }
    last = __shfl_sync(0xFFFFFFFFu, last, 0);
    __syncwarp();
    if (last) {
      // (3) the last warp: write the a and b bands back, then refill the buffer
      if (*(volatile int *)&sm.err == 0) {
        const int j0 = tile * R;
        const uint4 *sa = reinterpret_cast<const uint4 *>(sm.band[b][0]);
        const uint4 *sb = reinterpret_cast<const uint4 *>(sm.band[b][5]);
        uint4 *ga = reinterpret_cast<uint4 *>(const_cast<uint32_t *>(u.cA) + (int64_t)j0 * W);
        int rb = j0 + u.qy;
        rb = rb >= Cy ? rb - Cy : rb;
        const int split = min(R, Cy - rb) * W / 4;  // uint4 before the band wraps
        uint4 *gb = reinterpret_cast<uint4 *>(const_cast<uint32_t *>(u.cB));
        const int64_t gb1 = (int64_t)rb * W / 4;  // in uint4
#pragma unroll
        for (int q = lane; q < kTileWords / 4; q += 32) {
          ga[q] = sa[q];
          gb[q < split ? gb1 + q : (int64_t)(q - split)] = sb[q];
        }
      }
      __syncwarp();
      if constexpr (!kSingle) {
        // the buffer's next tile: claimed, or in the fixed order when the
        // claim slot is not this phase's
        int next = 0;
        if (lane == 0) {
          sm.done[b] = 0;
          const unsigned long long old = atomicAdd(
              reinterpret_cast<unsigned long long *>(g.ctl + kCtlTileClaim + (P & 1u)), 1ull);
          next = (uint32_t)(old >> 32) == (uint32_t)P ? kBufs * ncta + (int)(uint32_t)old
                                                      : cta + (t + kBufs) * ncta;
          if (next >= ntiles || *(volatile int *)&sm.err != 0) next = -1;
        }
        next = __shfl_sync(0xFFFFFFFFu, next, 0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        arm(next, b);
        if (next >= 0) stage_band(next, b, (1u << kBands) - 1u);
      }
    }
    if constexpr (kSingle) break;  // one tile per CTA
    b = b == kBufs - 1 ? 0 : b + 1;
    // leave together: the warp's lanes meet in __syncwarp every tile
    if (__any_sync(0xFFFFFFFFu, *(volatile int *)&sm.err != 0)) break;
  }
  __syncthreads();
  if (threadIdx.x == 0 && sm.err) {
    // give loads still in flight a bounded chance to land before exiting: the
    // last staging of every buffer (phases complete in order)
    mbar_wait(smem_u32(&sm.tables), 0u);
    for (int q = 0; q < kBufs; ++q)
      if (sm.armed[q] > 0) mbar_wait(smem_u32(&sm.full[q]), (uint32_t)(sm.armed[q] - 1) & 1u);
    g.ctl[kCtlStatus] = 1;
  }
}

// kMinBlocks, kSingle: four CTAs per SM with the pipelined tile loop (the
// large-lattice kernel), or five CTAs per SM, one tile per CTA and one band
// buffer (the compact kernel for lattices whose phase fits one wave: more CTAs
// resident for several lattices on their own streams, at 48 registers).
template <int kMinBlocks, bool kSingle, int kTPW = 1>
__global__ void __launch_bounds__(256 * kTPW, kMinBlocks) phase_tile_kernel(
    Geo g, const uint16_t *thrT, const uint32_t *thr32, int64_t p_off,
    const __grid_constant__ RoundKeys rk) {
  tile_phase<kSingle, kTPW>(g, thrT, thr32, p_off, (int)blockIdx.x, (int)gridDim.x,
                            TableKeys{&rk});
}

// Lock-step tile-staged phase of several lattices in one launch: CTAs
// [cta_begin, cta_begin + cta_count) of the grid work on job j, each lattice
// with its own tables, phase counter and schedule.
__global__ void __launch_bounds__(256, 4) phase_tile_multi_kernel(const MultiJob *__restrict__ jobs,
                                                                  int njobs, int64_t p_off) {
  int j = 0;
  while (j + 1 < njobs && (int)blockIdx.x >= jobs[j + 1].cta_begin) ++j;
  const MultiJob &J = jobs[j];
  const Geo g = J.g;
  tile_phase<false, 1>(g, J.thrT, J.thr32, p_off, (int)blockIdx.x - J.cta_begin, J.cta_count,
                       SeedKeys{g.k0, g.k1});
}

// Lock-step phase of several lattices in one launch: each CTA works on one
// lattice (its share of the grid is proportional to the lattice's words), with
// that lattice's tables, phase counter and schedule.
template <bool kAligned>
__global__ void __launch_bounds__(256, 4) phase_multi_kernel(const MultiJob *__restrict__ jobs,
                                                             int njobs, int64_t p_off) {
  __shared__ PhaseSmem sm;
  __shared__ int s_job;
  if (threadIdx.x == 0) {
    int j = 0;
    while (j + 1 < njobs && (int)blockIdx.x >= jobs[j + 1].cta_begin) ++j;
    s_job = j;
  }
  __syncthreads();
  const MultiJob &J = jobs[s_job];
  const Geo g = J.g;
  for (int t = threadIdx.x; t < kThrT / 2; t += blockDim.x)
    reinterpret_cast<uint32_t *>(sm.thrT)[t] = reinterpret_cast<const uint32_t *>(J.thrT)[t];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  const uint64_t P = (uint64_t)(g.ctl[kCtlPhaseBase] + p_off);
  if (threadIdx.x < 32) {
    const Sched sc = draw_schedule(g, P);
    if (threadIdx.x == 0) sm.sched = sc;
  }
  __syncthreads();
  const Sched sc = sm.sched;
  for (int t = threadIdx.x; t < kMoveN; t += blockDim.x)
    sm.trans[t] = make_uint2(J.trans[2 * t], J.trans[2 * t + 1]);
  __syncthreads();
  const PhaseU u = phase_uniform(g, sc);
  const uint32_t near128 = sc.near ? 128u : 0u;
  const int nw = g.Cy * g.W;
  const int stride = J.cta_count * blockDim.x;
  for (int base = ((int)blockIdx.x - J.cta_begin) * blockDim.x; base < nw; base += stride) {
    const int wid = base + threadIdx.x;
    const bool act = wid < nw;
    const int j = act ? wid / g.W : 0, w = act ? wid - j * g.W : 0;
    warp_word<kAligned ? kRowAligned : kRowGeneral>(g, u, sm.trans, sm.thrT, J.thr32, j, j, w, P,
                                                     near128, SeedKeys{g.k0, g.k1}, 0, act);
  }
}

// One lattice run by one warp of a resident CTA (JobDesc.warp): its words in
// the warp's share of the shared memory, its tables read through L1 from
// global memory, the warp's own barrier between phases.  The same per-word
// code as the CTA path, so results are identical.
template <int kMode, int kTPW>
__device__ __forceinline__ void warp_job_phase(const Geo &gs, const PhaseU &u, const uint2 *trans,
                                               const uint16_t *thrT, const uint32_t *thr32,
                                               int nwa, uint64_t P, uint32_t near128) {
  const int lane = threadIdx.x & 31;
  const SeedKeys keys{gs.k0, gs.k1};
  for (int base = 0; base < kTPW * nwa; base += 32) {  // uniform trip count
    const int i = base + lane;
    const bool act = i < kTPW * nwa;
    const int wid = !act ? 0 : (kTPW == 1 ? i : (kTPW == 2 ? i >> 1 : i >> 2));
    const int sub = act ? i - kTPW * wid : 0;
    const int j = wid / gs.W, w = wid - j * gs.W;
    warp_word<kMode, kTPW>(gs, u, trans, thrT, thr32, j, j, w, P, near128, keys, sub, act);
  }
}

__device__ __forceinline__ void warp_job(const JobDesc &J, uint32_t *region, PhaseU &su) {
  const int lane = threadIdx.x & 31;
  const Geo g = J.g;
  const int64_t nw = 16 * g.cstride;
  for (int64_t t = lane; t < nw; t += 32) region[t] = g.words[t];
  const int64_t P0 = g.ctl[kCtlPhaseBase];
  const int64_t nsweeps = J.nsweeps;
  const int obs_every = J.obs_every;
  Geo gs = g;
  gs.words = region;
  const bool aligned = (g.Cx & 15) == 0;
  const int nwa = g.Cy * g.W;  // a-words per phase
  const int tpw = J.max_tpw >= 4 && 4 * nwa <= 32 ? 4 : J.max_tpw >= 2 && 2 * nwa <= 32 ? 2 : 1;
  const uint2 *trans = reinterpret_cast<const uint2 *>(J.trans);
  int64_t obs_cnt = 0, obs_slot = 0;
  if (lane == 0 && obs_every > 0) {
    obs_cnt = g.ctl[kCtlObsCount];
    obs_slot = obs_cnt % J.ring_cap;
  }
  __syncwarp();
  for (int64_t s = 0; s < nsweeps; ++s) {
    for (int p = 0; p < 8; ++p) {
      const uint64_t P = (uint64_t)(P0 + 8 * s + p);
      const Sched sc = draw_schedule(gs, P);
      if (lane == 0) su = phase_uniform(gs, sc);
      __syncwarp();
      const PhaseU &u = su;  // read from shared memory where used
      const uint32_t near128 = sc.near ? 128u : 0u;
      if (aligned) {
        if (tpw == 1)
          warp_job_phase<kRowAligned, 1>(gs, u, trans, J.thrT, J.thr32, nwa, P, near128);
        else if (tpw == 2)
          warp_job_phase<kRowAligned, 2>(gs, u, trans, J.thrT, J.thr32, nwa, P, near128);
        else
          warp_job_phase<kRowAligned, 4>(gs, u, trans, J.thrT, J.thr32, nwa, P, near128);
      } else {
        if (tpw == 1)
          warp_job_phase<kRowGeneral, 1>(gs, u, trans, J.thrT, J.thr32, nwa, P, near128);
        else if (tpw == 2)
          warp_job_phase<kRowGeneral, 2>(gs, u, trans, J.thrT, J.thr32, nwa, P, near128);
        else
          warp_job_phase<kRowGeneral, 4>(gs, u, trans, J.thrT, J.thr32, nwa, P, near128);
      }
      __syncwarp();  // the phase's writes before the next phase's reads
    }
    const int64_t done = P0 / 8 + s + 1;
    if (obs_every > 0 && done % obs_every == 0) {
      // the 16 classes side by side, two lanes a class
      int c[7] = {0, 0, 0, 0, 0, 0, 0};
      count_class(gs, lane >> 1, lane & 1, 2, c);
      int64_t rec[8];
      rec[0] = done;
#pragma unroll
      for (int k = 0; k < 7; ++k) rec[1 + k] = warp_sum((int64_t)c[k]);
      if (lane == 0) {
        for (int k = 0; k < 8; ++k) g.ctl[kCtlLatest + k] = rec[k];
        int64_t *dst = J.ring + obs_slot * 8;
        for (int k = 0; k < 8; ++k) dst[k] = rec[k];
        g.ctl[kCtlObsCount] = ++obs_cnt;
        if (++obs_slot == J.ring_cap) obs_slot = 0;
        if (J.hist) {
          const int64_t N = (int64_t)g.Lx * g.Ly;
          const int64_t vals[3] = {rec[4], rec[5], rec[7]};
          for (int h = 0; h < 3; ++h)
            atomicAdd(reinterpret_cast<unsigned long long *>(
                          J.hist + h * J.nbins + (vals[h] + N) * J.nbins / (2 * N + 1)),
                      1ull);
        }
      }
      __syncwarp();
    }
  }
  for (int64_t t = lane; t < nw; t += 32) g.words[t] = region[t];
  if (lane == 0) g.ctl[kCtlPhaseBase] = P0 + 8 * nsweeps;
  __syncwarp();
}

// ============================================================================
// Resident batch kernel (many lattices of uneven size, one persistent launch).
// Each CTA takes lattices from a work queue, largest first; it holds the whole
// packed lattice and its tables in shared memory and runs all of that lattice's
// sweeps with block barriers between phases, recounting into the lattice's ring
// when due; then it writes the lattice back and takes the next one.  The same
// per-word code as phase_kernel runs against shared memory, so results are
// identical to the per-phase launches.
__global__ void __launch_bounds__(512, 1) resident_kernel(const JobDesc *__restrict__ jobs, int njobs,
                                                       int *queue, int warp_words) {
  extern __shared__ __align__(16) uint32_t dyn[];
  uint16_t *s_thrT = reinterpret_cast<uint16_t *>(dyn);
  uint2 *s_trans = reinterpret_cast<uint2 *>(dyn + kThrT / 2);
  uint32_t *s_words = dyn + kResTableWords;
  __shared__ Sched s_sched[8];  // the schedules of the current sweep's phases
  __shared__ PhaseU s_u[8];     // and their class pointers and offsets
  __shared__ int s_job;
  __shared__ int64_t s_red[32][7];
  __shared__ PhaseU s_wu[16];  // one-warp jobs: each warp's current phase
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) s_job = atomicAdd(queue, 1);
    __syncthreads();
    const int job = s_job;
    if (job >= njobs) break;
    if (jobs[job].warp) {
      // the rest of the queue is one-warp jobs (the planner orders them
      // last): every warp takes its own from here on, warp 0 this one
      uint32_t *region = dyn + (int64_t)warp * warp_words;
      for (int jw = warp == 0 ? job : -1;;) {
        if (jw < 0) {
          int x = 0;
          if (lane == 0) x = atomicAdd(queue, 1);
          jw = __shfl_sync(0xFFFFFFFFu, x, 0);
        }
        if (jw >= njobs) return;
        if (jobs[jw].warp && 16 * jobs[jw].g.cstride <= warp_words)
          warp_job(jobs[jw], region, s_wu[warp]);
        else if (lane == 0)
          jobs[jw].g.ctl[kCtlStatus] = 1;  // not a one-warp job: the planner's order broke
        jw = -1;
      }
    }
    const JobDesc &J = jobs[job];
    const Geo g = J.g;
    const int64_t nw = 16 * g.cstride;
    for (int t = threadIdx.x; t < kThrT / 2; t += blockDim.x)
      dyn[t] = reinterpret_cast<const uint32_t *>(J.thrT)[t];
    for (int t = threadIdx.x; t < kMoveN; t += blockDim.x)
      s_trans[t] = make_uint2(J.trans[2 * t], J.trans[2 * t + 1]);
    for (int64_t t = threadIdx.x; t < nw; t += blockDim.x) s_words[t] = g.words[t];
    const int64_t P0 = g.ctl[kCtlPhaseBase];
    const int64_t nsweeps = J.nsweeps;
    const int obs_every = J.obs_every;
    Geo gs = g;
    gs.words = s_words;
    const bool aligned = (g.Cx & 15) == 0;
    const int nwa = g.Cy * g.W;  // a-words per phase
    // threads a word: the most (four, two; at most J.max_tpw) that still take
    // a phase's words in one pass of the CTA, else one
    const int tpw = J.max_tpw >= 4 && 4 * nwa <= (int)blockDim.x ? 4
                  : J.max_tpw >= 2 && 2 * nwa <= (int)blockDim.x ? 2 : 1;
    // thread 0's copies of the record count and its ring slot: read once per
    // job, so that a record costs no global load on the sweep's critical path
    int64_t obs_cnt = 0, obs_slot = 0;
    if (threadIdx.x == 0 && obs_every > 0) {
      obs_cnt = g.ctl[kCtlObsCount];
      obs_slot = obs_cnt % J.ring_cap;
    }
    __syncthreads();
    const int nwarps = blockDim.x >> 5;
    for (int64_t s = 0; s < nsweeps; ++s) {
      // the eight schedules of the sweep depend on nothing but the phase
      // index: the warps draw them (and derive each phase's class pointers)
      // together, then every phase needs only the barrier that orders it
      // after the previous one
      for (int q = warp; q < 8; q += nwarps) {
        const Sched sc = draw_schedule(gs, (uint64_t)(P0 + 8 * s + q));
        if (lane == 0) {
          s_sched[q] = sc;
          s_u[q] = phase_uniform(gs, sc);
        }
      }
      __syncthreads();
      for (int p = 0; p < 8; ++p) {
        const uint64_t P = (uint64_t)(P0 + 8 * s + p);
        const PhaseU &u = s_u[p];  // read from shared memory where used
        const uint32_t near128 = s_sched[p].near ? 128u : 0u;
        for (int base = 0; base < tpw * nwa; base += blockDim.x) {  // uniform trip count
          const int i = base + threadIdx.x;
          const bool act = i < tpw * nwa;
          const int wid = !act ? 0 : tpw == 1 ? i : (tpw == 2 ? i >> 1 : i >> 2);
          const int sub = act ? i - tpw * wid : 0;
          const int j = wid / g.W, w = wid - j * g.W;
          const SeedKeys keys{gs.k0, gs.k1};
          if (aligned) {
            if (tpw == 1)
              warp_word<kRowAligned, 1>(gs, u, s_trans, s_thrT, J.thr32, j, j, w, P, near128, keys,
                                        sub, act);
            else if (tpw == 2)
              warp_word<kRowAligned, 2>(gs, u, s_trans, s_thrT, J.thr32, j, j, w, P, near128, keys,
                                        sub, act);
            else
              warp_word<kRowAligned, 4>(gs, u, s_trans, s_thrT, J.thr32, j, j, w, P, near128, keys,
                                        sub, act);
          } else {
            if (tpw == 1)
              warp_word<kRowGeneral, 1>(gs, u, s_trans, s_thrT, J.thr32, j, j, w, P, near128, keys,
                                        sub, act);
            else if (tpw == 2)
              warp_word<kRowGeneral, 2>(gs, u, s_trans, s_thrT, J.thr32, j, j, w, P, near128, keys,
                                        sub, act);
            else
              warp_word<kRowGeneral, 4>(gs, u, s_trans, s_thrT, J.thr32, j, j, w, P, near128, keys,
                                        sub, act);
          }
        }
        __syncthreads();
      }
      const int64_t done = P0 / 8 + s + 1;
      if (obs_every > 0 && done % obs_every == 0) {
        // the 16 classes side by side: thread t takes words t mod (blockDim / 16),
        // ... of class 16 t / blockDim (blockDim a multiple of 16)
        int c[7] = {0, 0, 0, 0, 0, 0, 0};
        const int per_cls = (int)blockDim.x >> 4;
        count_class(gs, (int)threadIdx.x / per_cls, (int)threadIdx.x % per_cls, per_cls, c);
#pragma unroll
        for (int k = 0; k < 7; ++k) {
          const int64_t v = warp_sum((int64_t)c[k]);
          if (lane == 0) s_red[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          int64_t rec[8];
          rec[0] = done;
          for (int k = 0; k < 7; ++k) {
            int64_t v = 0;
            for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) v += s_red[wv][k];
            rec[1 + k] = v;
          }
          for (int k = 0; k < 8; ++k) g.ctl[kCtlLatest + k] = rec[k];
          int64_t *dst = J.ring + obs_slot * 8;
          for (int k = 0; k < 8; ++k) dst[k] = rec[k];
          g.ctl[kCtlObsCount] = ++obs_cnt;
          if (++obs_slot == J.ring_cap) obs_slot = 0;
          if (J.hist) {  // reductions: no load to wait for
            const int64_t N = (int64_t)g.Lx * g.Ly;
            const int64_t vals[3] = {rec[4], rec[5], rec[7]};
            for (int h = 0; h < 3; ++h)
              atomicAdd(reinterpret_cast<unsigned long long *>(
                            J.hist + h * J.nbins + (vals[h] + N) * J.nbins / (2 * N + 1)),
                        1ull);
          }
        }
        __syncthreads();
      }
    }
    for (int64_t t = threadIdx.x; t < nw; t += blockDim.x) g.words[t] = s_words[t];
    if (threadIdx.x == 0) g.ctl[kCtlPhaseBase] = P0 + 8 * nsweeps;
    __syncthreads();
  }
}

int64_t resident_smem_bytes(int64_t max_words) {
  return (int64_t)sizeof(uint32_t) * (kResTableWords + max_words);
}

int resident_ctas_per_sm(int threads, int64_t max_words) {
  const int smem = (int)resident_smem_bytes(max_words);
  int per_sm = 0;
  if (cudaFuncSetAttribute(resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resident_kernel, threads, smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return per_sm < 1 ? 1 : per_sm;
}

int64_t resident_warp_words(int threads, int64_t max_words) {
  return ((kResTableWords + max_words) / (threads / 32)) & ~(int64_t)3;
}

cudaError_t launch_resident(const JobDesc *d_jobs, int njobs, int *d_queue, int grid, int threads,
                            int64_t max_words, cudaStream_t s) {
  const int64_t smem = resident_smem_bytes(max_words);
  cudaError_t e = cudaFuncSetAttribute(resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  resident_kernel<<<grid, threads, (size_t)smem, s>>>(
      d_jobs, njobs, d_queue, (int)resident_warp_words(threads, max_words));
  return cudaGetLastError();
}

// ============================================================================
// Launchers.
int phase_resident_grid(bool aligned) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cudaError_t e =
      aligned ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, phase_kernel<true>, 256, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, phase_kernel<false>, 256, 0);
  if (e != cudaSuccess || per_sm < 1 || sms < 1) return 152 * 3;
  return per_sm * sms;
}

int tile_count(const Geo &g) { return g.Cy / (kTileWords / g.W); }

bool tile_path_ok(const Geo &g) {
  return (g.Cx & 15) == 0 && (g.W & 3) == 0 && g.W <= kTileWords && kTileWords % g.W == 0 &&
         g.Cy % (kTileWords / g.W) == 0;
}

// Also raises the tile kernel's dynamic shared memory limit on the current
// device (outside any stream capture: called when a lattice is created).  0
// when that fails: the lattice then takes the direct path.
int tile_resident_grid() {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  constexpr int bytes = (int)sizeof(TileSmem<>);
  if (cudaFuncSetAttribute(phase_tile_kernel<4, false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
      cudaFuncSetAttribute(phase_tile_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           bytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, phase_tile_kernel<4, false>, 256,
                                                    bytes) != cudaSuccess ||
      per_sm < 1 || sms < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sms;
}

// The single-tile kernel: one thread a word, five CTAs per SM (48 registers;
// six at 40 registers spilled more and measured slower).  Two threads a word
// (512-thread CTAs, two per SM) measured 5.6 us a 4096^2 phase against 5.4,
// and half the throughput for four such lattices on their own streams: the
// phase is bound by the issue rate of the SMs that hold two tiles, not by the
// chain of one thread.
constexpr int kSmallTPW = 1;
constexpr int kSmallMinB = 5;

int tile_resident_grid_small() {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  constexpr int bytes = (int)sizeof(TileSmem<1>);
  if (cudaFuncSetAttribute(phase_tile_kernel<kSmallMinB, true, kSmallTPW>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, phase_tile_kernel<kSmallMinB, true, kSmallTPW>, 256 * kSmallTPW, bytes) !=
          cudaSuccess ||
      per_sm < 1 || sms < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sms;
}

cudaError_t launch_phase(const Geo &g, const DevTables &t, int64_t p_off, const LaunchCfg &cfg,
                         cudaStream_t s) {
  const int64_t nw = (int64_t)g.Cy * g.W;
  if (cfg.tile_grid > 0) {
    const int64_t tiles = nw / kTileWords;
    if (reinterpret_cast<const char *>(t.trans) !=
            reinterpret_cast<const char *>(t.thrT) + 2 * kThrT ||
        (reinterpret_cast<uintptr_t>(t.thrT) & 15u))
      return cudaErrorInvalidValue;  // the tables must be one staged block
    // A phase that fits one wave of the compact kernel (one tile per CTA)
    // takes it: measured faster for several such lattices on their own streams.
    if (cfg.tile_grid_small > 0 && tiles <= cfg.tile_grid_small)
      return launch_pdl_smem(phase_tile_kernel<kSmallMinB, true, kSmallTPW>, (int)tiles,
                             256 * kSmallTPW, sizeof(TileSmem<1>), s, g,
                             (const uint16_t *)t.thrT, t.thr32, p_off, round_keys(g.k0, g.k1));
    const int grid = (int)(tiles < cfg.tile_grid ? tiles : cfg.tile_grid);
    return launch_pdl_smem(phase_tile_kernel<4, false>, grid, 256, sizeof(TileSmem<>),
                           s, g, (const uint16_t *)t.thrT, t.thr32, p_off,
                           round_keys(g.k0, g.k1));
  }
  const int grid = grid_for(nw, 256, cfg.phase_grid_cap);
  const uint16_t *thrT = t.thrT;
  const uint32_t *thr32 = t.thr32, *tr = t.trans;
  if ((g.Cx & 15) == 0)
    return launch_pdl(phase_kernel<true>, grid, 256, s, g, thrT, thr32, tr, p_off);
  return launch_pdl(phase_kernel<false>, grid, 256, s, g, thrT, thr32, tr, p_off);
}

cudaError_t launch_phase_tile_multi(const MultiJob *d_jobs, int njobs, int grid, int64_t p_off,
                                    cudaStream_t s) {
  return launch_pdl_smem(phase_tile_multi_kernel, grid, 256, sizeof(TileSmem<>), s,
                         d_jobs, njobs, p_off);
}

cudaError_t launch_phase_multi(const MultiJob *d_jobs, int njobs, int grid, bool aligned,
                               int64_t p_off, cudaStream_t s) {
  if (aligned) return launch_pdl(phase_multi_kernel<true>, grid, 256, s, d_jobs, njobs, p_off);
  return launch_pdl(phase_multi_kernel<false>, grid, 256, s, d_jobs, njobs, p_off);
}

}  // namespace ccmc
