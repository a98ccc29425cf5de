// ccmc_kernels.cu -- CUDA kernels of the coupled-pair Metropolis sweep for
// sm_103a, and their launchers (declared in ccmc_internal.h).
#include <cuda_runtime.h>

#include <cstdint>

#include "ccmc_device.cuh"
#include "ccmc_internal.h"

namespace ccmc {

// ============================================================================
// Initial state (Sec. 3.1, stage 1): exactly N+ sites S=+1 and N- sites S=-1.
// Site index i = y Lx + x gets rank pi(i) under a seeded four-round Feistel
// permutation of [0, 4^h) with cycle-walking into [0, N); rank < N+ -> S=+1,
// rank < N+ + N- -> S=-1, else magnetic with sign bit i of the SIGN stream.
__device__ __forceinline__ uint64_t feistel_round_trip(uint32_t k0, uint32_t k1, int h,
                                                       uint64_t x) {
  const uint64_t mask = ((uint64_t)1 << h) - 1;
  uint64_t L = x >> h, R = x & mask;
#pragma unroll
  for (uint32_t round = 0; round < 4; ++round) {
    const U4 w = philox((uint32_t)R, round, 0u, TAG_FEISTEL, k0, k1);
    const uint64_t nR = L ^ ((uint64_t)w.x & mask);
    L = R;
    R = nR;
  }
  return (L << h) | R;
}

__global__ void init_kernel(Geo g, int h, int64_t n_plus, int64_t n_minus) {
  const int64_t nwords = 16 * g.cstride;
  const uint64_t N = (uint64_t)g.Lx * (uint64_t)g.Ly;
  for (int64_t wid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; wid < nwords;
       wid += (int64_t)gridDim.x * blockDim.x) {
    const int cls = (int)(wid / g.cstride);
    const int64_t rem = wid - (int64_t)cls * g.cstride;
    const int j = (int)(rem / g.W), w = (int)(rem - (int64_t)j * g.W);
    const int cx = cls & 3, cy = cls >> 2;
    const int s0 = w << 4;
    const int n = min(16, g.Cx - s0);
    uint32_t word = 0;
    for (int t = 0; t < n; ++t) {
      const int x = 4 * (s0 + t) + cx, y = 4 * j + cy;
      const uint64_t site = (uint64_t)y * g.Lx + x;
      uint64_t r = feistel_round_trip(g.k0, g.k1, h, site);
      while (r >= N) r = feistel_round_trip(g.k0, g.k1, h, r);
      uint32_t code;
      if ((int64_t)r < n_plus) {
        code = 2u;
      } else if ((int64_t)r < n_plus + n_minus) {
        code = 3u;
      } else {
        const U4 sw = philox((uint32_t)(site >> 7), 0u, 0u, TAG_SIGN, g.k0, g.k1);
        const uint32_t q = (uint32_t)(site >> 5) & 3u;
        const uint32_t bits = q == 0 ? sw.x : q == 1 ? sw.y : q == 2 ? sw.z : sw.w;
        code = (bits >> (site & 31u)) & 1u;
      }
      word |= code << (2 * t);
    }
    g.words[wid] = word;
  }
}

// ============================================================================
// One colour phase (Sec. 3.1-3.2).  Each thread owns one word of the a-class:
// up to 16 pairs (a, a + r).  It reads the a word, the four neighbour windows
// of a, the b window and the four neighbour windows of b; evaluates every
// pair's move; stores the a word and XORs the changed b sites back.
struct PhaseSmem {
  uint16_t thr[kTableN + 128];  // high halves of the thresholds, 64 entries of slack each side
  int32_t trans[256];
  Sched sched;
};

// Full evaluation of pair t when the fast path cannot decide it: the q = 0
// choice needs the SLOW stream (v >= 65532), or the 16-bit comparison tied.
__device__ __noinline__ void pair_slow(const Geo &g, const uint32_t *thr32, const int32_t *trans,
                                       uint32_t A, uint32_t B, const Sums &sa, const Sums &sb,
                                       uint32_t group, int t, uint64_t k, uint64_t P,
                                       uint32_t &dA, uint32_t &dB) {
  const U4 mv = philox(group, (uint32_t)P, (uint32_t)(P >> 32), TAG_MOVE, g.k0, g.k1);
  const int q = t & 3;
  const uint32_t R = q == 0 ? mv.x : q == 1 ? mv.y : q == 2 ? mv.z : mv.w;
  const uint32_t ca = (A >> (2 * t)) & 3u, cb = (B >> (2 * t)) & 3u;
  const uint32_t pc = (ca << 2) | cb;
  const uint32_t qc = (kQClass >> (2 * pc)) & 3u;
  if (qc == 0u) return;
  const U4 sl = philox((uint32_t)k, (uint32_t)P, (uint32_t)(P >> 32), TAG_SLOW, g.k0, g.k1);
  const uint32_t v = R & 0xFFFFu;
  uint32_t npc;
  if (qc == 2u) {
    uint32_t idx;
    if (v < 65532u) {
      idx = v % 6u;
    } else if (sl.y < 4294967292u) {
      idx = sl.y % 6u;
    } else {
      idx = 0xFFu;  // keep the current configuration
    }
    npc = idx == 0xFFu ? pc : (kSet0 >> (4 * idx)) & 15u;
  } else {
    npc = ((qc == 1u ? kSetP : kSetM) >> (4 * (v & 3u))) & 15u;
  }
  if (npc == pc) return;
  const int idx = trans_index(trans[pc * 16 + npc], lane4(sa.se, sa.so, t),
                              lane4(sb.se, sb.so, t), lane4(sa.ge, sa.go, t),
                              lane4(sb.ge, sb.go, t));
  const uint32_t thr = thr32[min(max(idx, 0), kTableN - 1)];
  const uint32_t u = (R & 0xFFFF0000u) | (sl.x & 0xFFFFu);
  if (thr == 0xFFFFFFFFu || u < thr) {
    const uint32_t x = pc ^ npc;
    dA |= (x >> 2) << (2 * t);
    dB |= (x & 3u) << (2 * t);
  }
}

__device__ __forceinline__ void phase_word(const Geo &g, const Sched &sc, const PhaseSmem &sm,
                                           const uint32_t *thr32, int j, int w, uint64_t P) {
  const int s0 = w << 4;
  const int n = min(16, g.Cx - s0);
  const int ax = sc.a0x, ay = sc.a0y;
  const int Cx = g.Cx, Cy = g.Cy, W = g.W;
  const int jm = j == 0 ? Cy - 1 : j - 1;
  const int jp = j + 1 == Cy ? 0 : j + 1;

  uint32_t *rowA = row_ptr(g, ay * 4 + ax, j);
  const uint32_t A = rowA[w];
  Sums sa{0u, 0u, 0u, 0u};
  add_neighbour(sa, fetch_window(row_ptr(g, ay * 4 + ((ax + 3) & 3), j), W, Cx,
                                 ax == 0 ? (s0 == 0 ? Cx - 1 : s0 - 1) : s0, n));
  add_neighbour(sa, fetch_window(row_ptr(g, ay * 4 + ((ax + 1) & 3), j), W, Cx,
                                 ax == 3 ? (s0 + 1 == Cx ? 0 : s0 + 1) : s0, n));
  add_neighbour(sa, row_ptr(g, ((ay + 3) & 3) * 4 + ax, ay == 0 ? jm : j)[w]);
  add_neighbour(sa, row_ptr(g, ((ay + 1) & 3) * 4 + ax, ay == 3 ? jp : j)[w]);

  const int bxx = ax + sc.rx, byy = ay + sc.ry;
  const int cbx = bxx & 3, cby = byy & 3;
  int jb = j + (byy >> 2);
  if (jb >= Cy) jb -= Cy;
  int sbb = s0 + (bxx >> 2);
  if (sbb >= Cx) sbb -= Cx;
  const int jbm = jb == 0 ? Cy - 1 : jb - 1;
  const int jbp = jb + 1 == Cy ? 0 : jb + 1;
  uint32_t *rowB = row_ptr(g, cby * 4 + cbx, jb);
  const uint32_t B = fetch_window(rowB, W, Cx, sbb, n);
  Sums sb{0u, 0u, 0u, 0u};
  add_neighbour(sb, fetch_window(row_ptr(g, cby * 4 + ((cbx + 3) & 3), jb), W, Cx,
                                 cbx == 0 ? (sbb == 0 ? Cx - 1 : sbb - 1) : sbb, n));
  add_neighbour(sb, fetch_window(row_ptr(g, cby * 4 + ((cbx + 1) & 3), jb), W, Cx,
                                 cbx == 3 ? (sbb + 1 == Cx ? 0 : sbb + 1) : sbb, n));
  add_neighbour(sb, fetch_window(row_ptr(g, ((cby + 3) & 3) * 4 + cbx, cby == 0 ? jbm : jb), W,
                                 Cx, sbb, n));
  add_neighbour(sb, fetch_window(row_ptr(g, ((cby + 1) & 3) * 4 + cbx, cby == 3 ? jbp : jb), W,
                                 Cx, sbb, n));

  // Random words: pair (i, j) of the class takes word i mod 4 of
  // Philox(seed, (j Cx4 + i / 4, P_lo, P_hi, MOVE)).
  uint32_t Rw[16];
  const uint32_t gbase = (uint32_t)j * (uint32_t)g.Cx4 + (uint32_t)(s0 >> 2);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (4 * q < n) {
      const U4 r = philox(gbase + q, (uint32_t)P, (uint32_t)(P >> 32), TAG_MOVE, g.k0, g.k1);
      Rw[4 * q + 0] = r.x;
      Rw[4 * q + 1] = r.y;
      Rw[4 * q + 2] = r.z;
      Rw[4 * q + 3] = r.w;
    } else {
      Rw[4 * q + 0] = Rw[4 * q + 1] = Rw[4 * q + 2] = Rw[4 * q + 3] = 0u;
    }
  }

  uint32_t dA = 0u, dB = 0u, slow = 0u;
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    if (t < n) {
      const uint32_t ca = (A >> (2 * t)) & 3u, cb = (B >> (2 * t)) & 3u;
      const uint32_t pc = (ca << 2) | cb;
      const uint32_t qc = (kQClass >> (2 * pc)) & 3u;
      const uint32_t R = Rw[t];
      const uint32_t v = R & 0xFFFFu;
      uint32_t npc;
      if (qc == 2u) {
        const uint32_t idx = v - 6u * ((v * 43691u) >> 18);  // v mod 6 for v < 2^16
        npc = (kSet0 >> (4 * idx)) & 15u;
        if (v >= 65532u) slow |= 1u << t;
      } else {
        npc = ((qc == 1u ? kSetP : kSetM) >> (4 * (v & 3u))) & 15u;
      }
      if (qc != 0u && npc != pc && !((slow >> t) & 1u)) {
        const int idx = trans_index(sm.trans[pc * 16 + npc], lane4(sa.se, sa.so, t),
                                    lane4(sb.se, sb.so, t), lane4(sa.ge, sa.go, t),
                                    lane4(sb.ge, sb.go, t));
        const uint32_t th = sm.thr[64 + idx];
        const uint32_t uhi = R >> 16;
        if (uhi < th) {
          const uint32_t x = pc ^ npc;
          dA |= (x >> 2) << (2 * t);
          dB |= (x & 3u) << (2 * t);
        } else if (uhi == th) {
          slow |= 1u << t;
        }
      }
    }
  }
  while (slow) {
    const int t = __ffs(slow) - 1;
    slow &= slow - 1u;
    pair_slow(g, thr32, sm.trans, A, B, sa, sb, gbase + (uint32_t)(t >> 2), t,
              (uint64_t)j * Cx + s0 + t, P, dA, dB);
  }
  if (dA) rowA[w] = A ^ dA;
  scatter_xor(rowB, Cx, sbb, n, dB);
}

__global__ void __launch_bounds__(256) phase_kernel(Geo g, const uint16_t *thr16,
                                                    const uint32_t *thr32,
                                                    const int32_t *trans_far,
                                                    const int32_t *trans_near, int64_t p_off) {
  __shared__ PhaseSmem sm;
  const uint64_t P = (uint64_t)(g.ctl[kCtlPhaseBase] + p_off);
  if (threadIdx.x < 32) {
    const Sched s = draw_schedule(g, P);
    if (threadIdx.x == 0) sm.sched = s;
  }
  for (int t = threadIdx.x; t < kTableN + 128; t += blockDim.x) {
    const int src = t - 64;
    sm.thr[t] = (src >= 0 && src < kTableN) ? thr16[src] : (uint16_t)0;
  }
  __syncthreads();
  const Sched sc = sm.sched;
  const int32_t *trans = sc.near ? trans_near : trans_far;
  for (int t = threadIdx.x; t < 256; t += blockDim.x) sm.trans[t] = trans[t];
  __syncthreads();
  const int64_t nw = (int64_t)g.Cy * g.W;
  for (int64_t wid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; wid < nw;
       wid += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(wid / g.W), w = (int)(wid - (int64_t)j * g.W);
    phase_word(g, sc, sm, thr32, j, w, P);
  }
}

// ============================================================================
// Recount (Eq. 3 and Eq. 2 by definition): per class word, popcounts of the
// charge/sign bit planes against the right and down neighbour windows.  Block
// partials go to scratch; the last block to arrive sums them into a record,
// appends it to the ring and the histograms, and re-arms the ticket.
struct RecountArgs {
  int64_t *partials;    // gridDim.x x 7 scratch
  int64_t *ring;        // cap x 8 records (nullptr: latest only)
  int64_t ring_cap;
  int64_t *hist;        // 3 x nbins (nullptr: none)
  int nbins;
  int64_t sweep_off;    // sweeps_done = phase_base / 8 + sweep_off
};

__device__ __forceinline__ int64_t warp_sum(int64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) recount_kernel(Geo g, RecountArgs a) {
  int c[7] = {0, 0, 0, 0, 0, 0, 0};  // Nc, BV, BJ, M, Ms, S, Ss
  const int64_t nwords = 16 * g.cstride;
  for (int64_t wid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; wid < nwords;
       wid += (int64_t)gridDim.x * blockDim.x) {
    const int cls = (int)(wid / g.cstride);
    const int64_t rem = wid - (int64_t)cls * g.cstride;
    const int j = (int)(rem / g.W), w = (int)(rem - (int64_t)j * g.W);
    const int cx = cls & 3, cy = cls >> 2;
    const int s0 = w << 4;
    const int n = min(16, g.Cx - s0);
    const uint32_t valid = n == 16 ? 0x55555555u : (((1u << (2 * n)) - 1u) & 0x55555555u);
    const uint32_t X = g.words[wid];
    const uint32_t Xr = fetch_window(row_ptr(g, cy * 4 + ((cx + 1) & 3), j), g.W, g.Cx,
                                     cx == 3 ? (s0 + 1 == g.Cx ? 0 : s0 + 1) : s0, n);
    const int jd = cy == 3 ? (j + 1 == g.Cy ? 0 : j + 1) : j;
    const uint32_t Xd = row_ptr(g, ((cy + 1) & 3) * 4 + cx, jd)[w];
    const uint32_t K = (X >> 1) & valid, G = X & valid;
    const uint32_t U = ~K & valid;  // magnetic
    const int chg = __popc(K & ~G) - __popc(K & G);
    const int mag = __popc(U & ~G) - __popc(U & G);
    const int sgn = ((cx + cy) & 1) ? -1 : 1;
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
  }
  __shared__ int64_t red[8][7];
  __shared__ bool last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const int64_t v = warp_sum((int64_t)c[k]);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    int64_t v = 0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) v += red[wv][threadIdx.x];
    a.partials[blockIdx.x * 7 + threadIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long prev =
        atomicAdd(reinterpret_cast<unsigned long long *>(g.ctl + kCtlTicket), 1ull);
    last = (prev == (unsigned long long)(gridDim.x - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ int64_t rec[8];
  if (threadIdx.x < 7) {
    int64_t v = 0;
    for (unsigned b = 0; b < gridDim.x; ++b)
      v += *(volatile int64_t *)(a.partials + (int64_t)b * 7 + threadIdx.x);
    rec[1 + threadIdx.x] = v;
  }
  if (threadIdx.x == 0) rec[0] = g.ctl[kCtlPhaseBase] / 8 + a.sweep_off;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 8; ++k) g.ctl[kCtlLatest + k] = rec[k];
    if (a.ring) {
      const int64_t cnt = g.ctl[kCtlObsCount];
      int64_t *dst = a.ring + (cnt % a.ring_cap) * 8;
      for (int k = 0; k < 8; ++k) dst[k] = rec[k];
      g.ctl[kCtlObsCount] = cnt + 1;
      if (a.hist) {
        const int64_t N = (int64_t)g.Lx * g.Ly;
        const int64_t vals[3] = {rec[4], rec[5], rec[7]};
        for (int h = 0; h < 3; ++h) {
          const int64_t bin = (vals[h] + N) * a.nbins / (2 * N + 1);
          a.hist[h * a.nbins + bin] += 1;
        }
      }
    }
    g.ctl[kCtlTicket] = 0;
  }
}

// ============================================================================
__global__ void advance_kernel(int64_t *ctl, int64_t phases) { ctl[kCtlPhaseBase] += phases; }

__global__ void set_ctl_kernel(int64_t *ctl, int64_t phase_base) {
  for (int k = threadIdx.x; k < kCtlWords; k += blockDim.x) ctl[k] = 0;
  __syncthreads();
  if (threadIdx.x == 0) ctl[kCtlPhaseBase] = phase_base;
}

// Logical bytes (site y Lx + x) <-> packed class words.
__global__ void unpack_kernel(Geo g, uint8_t *out) {
  const int64_t nwords = 16 * g.cstride;
  for (int64_t wid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; wid < nwords;
       wid += (int64_t)gridDim.x * blockDim.x) {
    const int cls = (int)(wid / g.cstride);
    const int64_t rem = wid - (int64_t)cls * g.cstride;
    const int j = (int)(rem / g.W), w = (int)(rem - (int64_t)j * g.W);
    const int s0 = w << 4, n = min(16, g.Cx - s0);
    const uint32_t X = g.words[wid];
    for (int t = 0; t < n; ++t) {
      const int64_t x = 4 * (s0 + t) + (cls & 3), y = 4 * j + (cls >> 2);
      out[y * g.Lx + x] = (uint8_t)((X >> (2 * t)) & 3u);
    }
  }
}

__global__ void pack_kernel(Geo g, const uint8_t *in, int *bad) {
  const int64_t nwords = 16 * g.cstride;
  for (int64_t wid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; wid < nwords;
       wid += (int64_t)gridDim.x * blockDim.x) {
    const int cls = (int)(wid / g.cstride);
    const int64_t rem = wid - (int64_t)cls * g.cstride;
    const int j = (int)(rem / g.W), w = (int)(rem - (int64_t)j * g.W);
    const int s0 = w << 4, n = min(16, g.Cx - s0);
    uint32_t X = 0u;
    for (int t = 0; t < n; ++t) {
      const int64_t x = 4 * (s0 + t) + (cls & 3), y = 4 * j + (cls >> 2);
      const uint32_t c = in[y * g.Lx + x];
      if (c > 3u) *bad = 1;
      X |= (c & 3u) << (2 * t);
    }
    g.words[wid] = X;
  }
}

__global__ void philox_kernel(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                              uint32_t k1, int64_t count, uint32_t *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const U4 r = philox(c0 + (uint32_t)i, c1, c2, c3, k0, k1);
    out[4 * i + 0] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
  }
}

// ============================================================================
// Launchers.
static int grid_for(int64_t items, int block, int cap) {
  int64_t b = (items + block - 1) / block;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_init(const Geo &g, int h, int64_t n_plus, int64_t n_minus, cudaStream_t s) {
  init_kernel<<<grid_for(16 * g.cstride, 256, 152 * 16), 256, 0, s>>>(g, h, n_plus, n_minus);
  return cudaGetLastError();
}

cudaError_t launch_phase(const Geo &g, const DevTables &t, int64_t p_off, const LaunchCfg &cfg,
                         cudaStream_t s) {
  const int64_t nw = (int64_t)g.Cy * g.W;
  phase_kernel<<<grid_for(nw, 256, cfg.phase_grid_cap), 256, 0, s>>>(
      g, t.thr16, t.thr32, t.trans_far, t.trans_near, p_off);
  return cudaGetLastError();
}

int recount_grid(const Geo &g) { return grid_for(16 * g.cstride, 256, 152 * 4); }

cudaError_t launch_recount(const Geo &g, int64_t *partials, int64_t *ring, int64_t ring_cap,
                           int64_t *hist, int nbins, int64_t sweep_off, cudaStream_t s) {
  RecountArgs a{partials, ring, ring_cap, hist, nbins, sweep_off};
  recount_kernel<<<recount_grid(g), 256, 0, s>>>(g, a);
  return cudaGetLastError();
}

cudaError_t launch_advance(int64_t *ctl, int64_t phases, cudaStream_t s) {
  advance_kernel<<<1, 1, 0, s>>>(ctl, phases);
  return cudaGetLastError();
}

cudaError_t launch_set_ctl(int64_t *ctl, int64_t phase_base, cudaStream_t s) {
  set_ctl_kernel<<<1, 32, 0, s>>>(ctl, phase_base);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const Geo &g, uint8_t *out, cudaStream_t s) {
  unpack_kernel<<<grid_for(16 * g.cstride, 256, 152 * 16), 256, 0, s>>>(g, out);
  return cudaGetLastError();
}

cudaError_t launch_pack(const Geo &g, const uint8_t *in, int *bad, cudaStream_t s) {
  pack_kernel<<<grid_for(16 * g.cstride, 256, 152 * 16), 256, 0, s>>>(g, in, bad);
  return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                          uint32_t k1, int64_t count, uint32_t *out, cudaStream_t s) {
  philox_kernel<<<grid_for(count, 256, 152 * 8), 256, 0, s>>>(c0, c1, c2, c3, k0, k1, count, out);
  return cudaGetLastError();
}

}  // namespace ccmc
