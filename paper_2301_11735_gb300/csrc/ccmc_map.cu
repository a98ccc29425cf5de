// ccmc_map.cu -- device side of the paper-faithful map mode (Sec. 3.2): one
// thread per pair of a host-built map, each making the coupled-pair move of
// Sec. 3.1 on the packed lattice.  The pairs of a map do not interact (none
// is inside another's covering), so all of them move at once; the only words
// two threads may share are the packed words of their own sites, which they
// change with atomic XORs of their own bits.
//
// The move uses the library's own tables: the 64-bit move entry of the pair's
// state, choice and kind (partner a nearest neighbour of a or not), the dp4a threshold index from (sum_a (S+1) - sum_b (S+1) + 8,
// sum_a (sigma+1), sum_b (sigma+1)) and the full 32-bit threshold.  Random
// words of pair p of map m: the 16-bit field v = the low half of word 0 of
// Philox(seed, (p, m_lo, m_hi, 11)) and, when v >= 65532 or its level w =
// v / 12 ties the threshold's level, the slow words of Philox(seed, (p, m_lo,
// m_hi, 12)) -- the same rules as the colour phases' exact path.
#include <cuda_runtime.h>

#include <cstdint>

#include "ccmc_device.cuh"
#include "ccmc_internal.h"
#include "ccmc_map.h"

namespace ccmc {

namespace {

constexpr uint32_t kTagMapMove = 11u;
constexpr uint32_t kTagMapSlow = 12u;

struct SiteRef {
  uint32_t *word;
  int shift;
};

__device__ __forceinline__ SiteRef site_ref(const Geo &g, int x, int y) {
  const int cls = (y & 3) * 4 + (x & 3), i = x >> 2, j = y >> 2;
  return SiteRef{g.words + (int64_t)cls * g.cstride + (int64_t)j * g.W + (i >> 4), 2 * (i & 15)};
}

__device__ __forceinline__ uint32_t code_at(const Geo &g, int x, int y) {
  const SiteRef r = site_ref(g, x, y);
  return (*r.word >> r.shift) & 3u;
}

// S + 1 and sigma + 1 of a site code (0: s=+1/2, 1: s=-1/2, 2: S=+1, 3: S=-1)
__device__ __forceinline__ uint32_t s_plus1(uint32_t c) { return (0x0211u >> (4 * c)) & 3u; }
__device__ __forceinline__ uint32_t g_plus1(uint32_t c) { return (0x1102u >> (4 * c)) & 3u; }

__global__ void __launch_bounds__(256) map_kernel(Geo g, const int32_t *__restrict__ pairs,
                                                  int64_t npairs, uint32_t m_lo, uint32_t m_hi,
                                                  const uint32_t *__restrict__ thr32,
                                                  const uint2 *__restrict__ trans) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const int a = pairs[2 * p], b = pairs[2 * p + 1];
  const int Lx = g.Lx, Ly = g.Ly;
  const int ax = a % Lx, ay = a / Lx, bx = b % Lx, by = b / Lx;
  const SiteRef ra = site_ref(g, ax, ay), rb = site_ref(g, bx, by);
  const uint32_t ca = (*ra.word >> ra.shift) & 3u, cb = (*rb.word >> rb.shift) & 3u;
  // neighbour sums (old states, partner included)
  uint32_t SA = 0, GA = 0, SB = 0, GB = 0;
  bool near = false;
  {
    const int nx[4] = {ax == 0 ? Lx - 1 : ax - 1, ax + 1 == Lx ? 0 : ax + 1, ax, ax};
    const int ny[4] = {ay, ay, ay == 0 ? Ly - 1 : ay - 1, ay + 1 == Ly ? 0 : ay + 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t c = code_at(g, nx[k], ny[k]);
      SA += s_plus1(c);
      GA += g_plus1(c);
      near |= (nx[k] == bx && ny[k] == by);
    }
  }
  {
    const int nx[4] = {bx == 0 ? Lx - 1 : bx - 1, bx + 1 == Lx ? 0 : bx + 1, bx, bx};
    const int ny[4] = {by, by, by == 0 ? Ly - 1 : by - 1, by + 1 == Ly ? 0 : by + 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t c = code_at(g, nx[k], ny[k]);
      SB += s_plus1(c);
      GB += g_plus1(c);
    }
  }
  const U4 rw = philox((uint32_t)p, m_lo, m_hi, kTagMapMove, g.k0, g.k1);
  const uint32_t v = rw.x & 0xFFFFu, wq = v / 12u;
  U4 sl{0u, 0u, 0u, 0u};
  bool have_slow = false;
  uint32_t r;
  if (v < 65532u) {
    r = v % 12u;
  } else {
    sl = philox((uint32_t)p, m_lo, m_hi, kTagMapSlow, g.k0, g.k1);
    have_slow = true;
    if (sl.y >= 4294967292u) return;  // keep the current configuration
    r = sl.y % 12u;
  }
  const uint32_t pc = (ca << 2) | cb;
  const uint2 e = trans[(2u * r + (near ? 1u : 0u)) * 16u + (pc ^ r)];
  const uint32_t x = (e.y >> 24) & 15u;  // pc XOR the chosen configuration
  if (x == 0u) return;           // the chosen configuration is the current one
  const uint32_t env = (SA + 8u - SB) | (GA << 8) | (GB << 16);
  const uint32_t thr = thr32[__dp4a((int)e.y, (int)env, (int)e.x)];
  bool accept;
  if (thr == 0xFFFFFFFFu) {
    accept = true;
  } else if (v >= 65532u) {
    accept = sl.x < thr;  // have_slow: drawn for the choice
  } else if (wq != threshold_level(thr)) {
    accept = wq < threshold_level(thr);
  } else {
    if (!have_slow) sl = philox((uint32_t)p, m_lo, m_hi, kTagMapSlow, g.k0, g.k1);
    accept = ((uint64_t)wq << 32) + sl.x < 5461ull * thr;
  }
  if (!accept) return;
  if (x >> 2) atomicXor(ra.word, (x >> 2) << ra.shift);
  if (x & 3u) atomicXor(rb.word, (x & 3u) << rb.shift);
}

}  // namespace

cudaError_t launch_map(const Geo &g, const int32_t *d_pairs, int64_t npairs, uint64_t m,
                       const DevTables &t, cudaStream_t s) {
  if (npairs <= 0) return cudaSuccess;
  const int64_t blocks = (npairs + 255) / 256;
  map_kernel<<<(unsigned)blocks, 256, 0, s>>>(
      g, d_pairs, npairs, (uint32_t)m, (uint32_t)(m >> 32), t.thr32,
      reinterpret_cast<const uint2 *>(t.trans));
  return cudaGetLastError();
}

}  // namespace ccmc
