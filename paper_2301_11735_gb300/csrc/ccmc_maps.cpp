// ccmc_maps.cpp -- host generation of the paper's maps (Sec. 3.2, the
// algorithm for building a map).
//
// A map is a list of P = max(1, floor(N / 10)) site pairs built by random
// marking on an array of N flags, all clear at first: draw a site until one is
// unmarked and mark it (a); draw and mark b the same way (b may neighbour a);
// append (a, b); mark the four nearest neighbours of a and of b; repeat until
// P pairs are listed.  Every later pair avoids the earlier pairs' sites and
// their neighbours, so the pairs of one map do not interact and a device
// kernel may move all of them at once.  P pairs always fit: before pair p at
// most 10 p sites are marked, and N - 10 (P - 1) >= 2.
//
// Random draws (keyed by the 64-bit seed): draw d of map m takes the 64-bit
// value of words 2 (d mod 2) and 2 (d mod 2) + 1 of Philox4x32-10(counter
// (d / 2, m_lo, m_hi, 10)); the site is the high half of value * N, redrawn
// when the low half is below 2^64 mod N (exact uniformity).
//
// Maps are independent of each other, so several host threads build the maps
// of one call in parallel; the result does not depend on the thread count.
#include <cstdint>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "../../include/ccmc.h"

namespace {

constexpr uint32_t kTagMap = 10u;

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32 x 32 -> 64-bit
// multiplies whose halves are cross-mixed with the key; the key advances by
// the two Weyl constants between rounds.
void philox_host(const uint32_t ctr[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// Map m into pairs[2P]; `marked` is N bytes of scratch.
void build_one(int Lx, int Ly, uint64_t seed, int64_t m, int64_t P, uint8_t *marked,
               int32_t *pairs) {
  const uint64_t N = (uint64_t)Lx * (uint64_t)Ly;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint64_t floor_lo = (0 - N) % N;  // 2^64 mod N
  std::memset(marked, 0, (size_t)N);
  uint64_t d = 0;
  uint32_t w[4] = {0, 0, 0, 0};
  auto draw_unmarked = [&]() -> int32_t {
    for (;;) {
      const int h = (int)(d & 1u);
      if (h == 0) {
        const uint32_t ctr[4] = {(uint32_t)(d >> 1), (uint32_t)(uint64_t)m,
                                 (uint32_t)((uint64_t)m >> 32), kTagMap};
        philox_host(ctr, k0, k1, w);
      }
      ++d;
      const uint64_t x = ((uint64_t)w[2 * h + 1] << 32) | w[2 * h];
      const unsigned __int128 prod = (unsigned __int128)x * N;
      if ((uint64_t)prod < floor_lo) continue;
      const uint64_t site = (uint64_t)(prod >> 64);
      if (marked[site]) continue;
      marked[site] = 1;
      return (int32_t)site;
    }
  };
  auto mark_neighbours = [&](int32_t s) {
    const int x = s % Lx, y = s / Lx;
    marked[(size_t)y * Lx + (x + 1 == Lx ? 0 : x + 1)] = 1;
    marked[(size_t)y * Lx + (x == 0 ? Lx - 1 : x - 1)] = 1;
    marked[(size_t)(y + 1 == Ly ? 0 : y + 1) * Lx + x] = 1;
    marked[(size_t)(y == 0 ? Ly - 1 : y - 1) * Lx + x] = 1;
  };
  for (int64_t p = 0; p < P; ++p) {
    const int32_t a = draw_unmarked();
    const int32_t b = draw_unmarked();
    pairs[2 * p] = a;
    pairs[2 * p + 1] = b;
    mark_neighbours(a);
    mark_neighbours(b);
  }
}

}  // namespace

extern "C" int64_t ccmc_map_size(int Lx, int Ly) {
  if (Lx < 2 || Ly < 2) return CCMC_E_INVAL;
  const int64_t P = (int64_t)Lx * Ly / 10;
  return P < 1 ? 1 : P;
}

extern "C" int ccmc_maps_build(int Lx, int Ly, uint64_t seed, int64_t map0, int64_t nmaps,
                               int32_t *pairs_out, int nthreads) {
  if (Lx < 2 || Ly < 2 || (int64_t)Lx * Ly > (int64_t)1 << 31 || map0 < 0 || nmaps < 0 ||
      (nmaps > 0 && !pairs_out))
    return CCMC_E_INVAL;
  if (nmaps == 0) return CCMC_OK;
  const int64_t P = ccmc_map_size(Lx, Ly);
  const size_t N = (size_t)Lx * Ly;
  int threads = nthreads > 0 ? nthreads : (int)std::thread::hardware_concurrency();
  if (threads < 1) threads = 1;
  if (threads > nmaps) threads = (int)nmaps;
  if (threads > 256) threads = 256;
  std::vector<std::vector<uint8_t>> scratch;
  try {
    scratch.resize((size_t)threads);
    for (auto &v : scratch) v.resize(N);
  } catch (const std::bad_alloc &) {
    return CCMC_E_NOMEM;
  }
  auto worker = [&](int t) {
    for (int64_t k = t; k < nmaps; k += threads)
      build_one(Lx, Ly, seed, map0 + k, P, scratch[(size_t)t].data(), pairs_out + 2 * P * k);
  };
  if (threads == 1) {
    worker(0);
    return CCMC_OK;
  }
  std::vector<std::thread> pool;
  try {
    for (int t = 0; t < threads; ++t) pool.emplace_back(worker, t);
  } catch (...) {
    for (auto &th : pool) th.join();
    return CCMC_E_NOMEM;
  }
  for (auto &th : pool) th.join();
  return CCMC_OK;
}
