// ccmc_kernels.cu -- the CUDA kernels around the colour phases for sm_103a
// (initial state, observables recount, phase counter, state packing, Philox
// export) and their launchers (declared in ccmc_internal.h).  The phase
// kernels are in ccmc_phase.cu.
#include <cuda_runtime.h>

#include <cstdint>

#include "ccmc_count.cuh"
#include "ccmc_device.cuh"
#include "ccmc_fault.h"
#include "ccmc_internal.h"
#include "ccmc_launch.cuh"
#include "ccmc_state.h"

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
// Recount (Eq. 3 and Eq. 2 by definition): per class word, popcounts of the
// charge/sign bit planes against the right and down neighbour windows.  Block
// partials go to scratch; the last block to arrive sums them into a record,
// appends it to the ring and the histograms, and re-arms the ticket.
struct RecountArgs {
  int64_t *partials;    // (gridDim.x * gridDim.y) x 7 scratch
  int64_t *ring;        // cap x 8 records (nullptr: latest only)
  int64_t ring_cap;
  int64_t *hist;        // 3 x nbins (nullptr: none)
  int nbins;
  int64_t sweep_off;    // sweeps_done = phase_base / 8 + sweep_off
};

// Grid (gx, 16): grid row y counts class y.
__global__ void __launch_bounds__(256, 5) recount_kernel(Geo g, RecountArgs a) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  int c[7] = {0, 0, 0, 0, 0, 0, 0};  // Nc, BV, BJ, M, Ms, S, Ss
  if (quads_ok(g))
    count_class_quads(g, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x,
                      gridDim.x * blockDim.x, c);
  else
    count_class(g, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, c);
  const unsigned nblocks = gridDim.x * gridDim.y;
  const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
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
    a.partials[bid * 7 + threadIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long prev =
        atomicAdd(reinterpret_cast<unsigned long long *>(g.ctl + kCtlTicket), 1ull);
    last = (prev == (unsigned long long)(nblocks - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block sums the partials with all its threads (L2 loads: the
  // partials were written by other blocks)
  __shared__ int64_t rec[8];
  int64_t v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] += __ldcg(a.partials + (int64_t)b * 7 + k);
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const int64_t x = warp_sum(v[k]);
    if (lane == 0) red[warp][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    int64_t x = 0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) x += red[wv][threadIdx.x];
    rec[1 + threadIdx.x] = x;
  }
  if (threadIdx.x == 0) rec[0] = g.ctl[kCtlPhaseBase] / 8 + a.sweep_off;
  __syncthreads();
  if (threadIdx.x == 0) {
    rec[3] += bj_completion(g, rec[1]);
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
__global__ void advance_kernel(int64_t *ctl, int64_t phases) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  ctl[kCtlPhaseBase] += phases;
}

// Self-test of the bounded device waits: one CTA waits on an mbarrier that
// nothing completes, polling at most `polls` times, then records the timeout in
// *status and returns -- as the phase kernels' waits do on a bulk copy or an
// arrival that never comes, so that the context stays usable.
__global__ void wait_selftest_kernel(uint32_t polls, int *status) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool done = false;
  for (uint32_t i = 0; i < polls && !done; ++i) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"(a)
        : "memory");
    done = r != 0;
  }
  if (!done && threadIdx.x == 0) *status = 1;
}

cudaError_t launch_wait_selftest(uint32_t polls, int *status, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(polls, status);
  return cudaGetLastError();
}

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

// Compact row-major state, 2 bits a site: site i = y Lx + x at bits 2 (i mod
// 4) of byte i / 4.  As Lx is a multiple of 4, byte i of row y holds column i of
// the four classes (cx = 0..3) of class row y / 4, y mod 4: one thread builds
// (or splits) the four class words of column block w from 16 consecutive bytes.
__device__ __forceinline__ uint32_t gather_field(uint32_t q, int cx) {
  // the cx-th 2-bit field of each of q's four bytes, packed into 8 bits
  uint32_t x = (q >> (2 * cx)) & 0x03030303u;
  x = (x | (x >> 6)) & 0x000F000Fu;
  return (x | (x >> 12)) & 0xFFu;
}

__device__ __forceinline__ uint32_t scatter_field(uint32_t f, int cx) {
  // inverse of gather_field: 8 bits -> the cx-th field of four bytes
  uint32_t x = (f | (f << 12)) & 0x000F000Fu;
  x = (x | (x << 6)) & 0x03030303u;
  return x << (2 * cx);
}

__global__ void pack2_kernel(Geo g, const uint8_t *in) {
  const int64_t nthr = 4 * (int64_t)g.Cy * g.W;
  const int64_t row_bytes = g.Lx / 4;
  const bool vec = (row_bytes & 15) == 0;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < nthr;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int w = (int)(id % g.W);
    const int64_t r = id / g.W;  // r = cy Cy + j
    const int cy = (int)(r / g.Cy), j = (int)(r - (int64_t)cy * g.Cy);
    const uint8_t *src = in + (int64_t)(4 * j + cy) * row_bytes + 16 * w;
    const int n = min(16, g.Cx - 16 * w);
    uint32_t q[4] = {0u, 0u, 0u, 0u};
    if (vec) {
      const uint4 v = *reinterpret_cast<const uint4 *>(src);
      q[0] = v.x;
      q[1] = v.y;
      q[2] = v.z;
      q[3] = v.w;
    } else {
      for (int t = 0; t < n; ++t) q[t >> 2] |= (uint32_t)src[t] << (8 * (t & 3));
    }
#pragma unroll
    for (int cx = 0; cx < 4; ++cx) {
      uint32_t word = 0u;
#pragma unroll
      for (int k = 0; k < 4; ++k) word |= gather_field(q[k], cx) << (8 * k);
      g.words[(int64_t)(cy * 4 + cx) * g.cstride + (int64_t)j * g.W + w] = word;
    }
  }
}

__global__ void unpack2_kernel(Geo g, uint8_t *out) {
  const int64_t nthr = 4 * (int64_t)g.Cy * g.W;
  const int64_t row_bytes = g.Lx / 4;
  const bool vec = (row_bytes & 15) == 0;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < nthr;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int w = (int)(id % g.W);
    const int64_t r = id / g.W;
    const int cy = (int)(r / g.Cy), j = (int)(r - (int64_t)cy * g.Cy);
    uint8_t *dst = out + (int64_t)(4 * j + cy) * row_bytes + 16 * w;
    const int n = min(16, g.Cx - 16 * w);
    uint32_t q[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int cx = 0; cx < 4; ++cx) {
      const uint32_t word = g.words[(int64_t)(cy * 4 + cx) * g.cstride + (int64_t)j * g.W + w];
#pragma unroll
      for (int k = 0; k < 4; ++k) q[k] |= scatter_field((word >> (8 * k)) & 0xFFu, cx);
    }
    if (vec) {
      *reinterpret_cast<uint4 *>(dst) = make_uint4(q[0], q[1], q[2], q[3]);
    } else {
      for (int t = 0; t < n; ++t) dst[t] = (uint8_t)(q[t >> 2] >> (8 * (t & 3)));
    }
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
cudaError_t launch_init(const Geo &g, int h, int64_t n_plus, int64_t n_minus, cudaStream_t s) {
  init_kernel<<<grid_for(16 * g.cstride, 256, 152 * 16), 256, 0, s>>>(g, h, n_plus, n_minus);
  return cudaGetLastError();
}

// Grid x-extent of recount_kernel (its y-extent is the 16 classes): at most
// 16 x 47 = 752 blocks, one wave at five blocks per SM (48 registers).  A
// thread's unit is a word, or four words on rows that allow 16-byte loads.
static int recount_gx(const Geo &g) {
  const int64_t units = (int64_t)g.Cy * g.W / (((g.Cx & 15) == 0 && (g.W & 3) == 0) ? 4 : 1);
  return grid_for(units, 256, 47);
}

int recount_grid(const Geo &g) { return 16 * recount_gx(g); }

cudaError_t launch_recount(const Geo &g, int64_t *partials, int64_t *ring, int64_t ring_cap,
                           int64_t *hist, int nbins, int64_t sweep_off, cudaStream_t s) {
  RecountArgs a{partials, ring, ring_cap, hist, nbins, sweep_off};
  return launch_pdl(recount_kernel, dim3((unsigned)recount_gx(g), 16u), 256, s, g, a);
}

cudaError_t launch_advance(int64_t *ctl, int64_t phases, cudaStream_t s) {
  return launch_pdl(advance_kernel, 1, 1, s, ctl, phases);
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

cudaError_t launch_pack2(const Geo &g, const uint8_t *in, cudaStream_t s) {
  pack2_kernel<<<grid_for(4 * (int64_t)g.Cy * g.W, 256, 152 * 16), 256, 0, s>>>(g, in);
  return cudaGetLastError();
}

cudaError_t launch_unpack2(const Geo &g, uint8_t *out, cudaStream_t s) {
  unpack2_kernel<<<grid_for(4 * (int64_t)g.Cy * g.W, 256, 152 * 16), 256, 0, s>>>(g, out);
  return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                          uint32_t k1, int64_t count, uint32_t *out, cudaStream_t s) {
  philox_kernel<<<grid_for(count, 256, 152 * 8), 256, 0, s>>>(c0, c1, c2, c3, k0, k1, count, out);
  return cudaGetLastError();
}

}  // namespace ccmc
