// ccmc_noalloc.cu -- an observables recount that allocates no memory.
//
// Some callers cannot let a library allocate device memory at the point of the
// call: a serving loop that reserved its whole memory budget up front and must
// not see a library take more, or a latency-critical path that must not pay
// for (or be serialised by) cudaMalloc/cudaFree.  ccmc_recount_noalloc serves
// them: the caller passes the lattice and the output buffer, and the scratch
// the reduction needs (one partial-sum slot per block and an arrival counter)
// lives in the fixed-size static device array below.  That array is part of
// the library's device image, so every GPU that loads the library holds it
// (kNaScratchBytes) until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/ccmc.h"

namespace {

constexpr int kNaBlocks = 1024;   // the grid never exceeds this: one slot each
constexpr int kNaThreads = 256;
constexpr int kNaSlot = 8;        // 7 partial sums per block, padded to 8
constexpr int kNaMaxDevices = 64;
constexpr int64_t kNaMaxSites = (int64_t)1 << 30;

// Scratch: kNaBlocks slots of partial sums, then the arrival counter.
static __device__ __align__(256) long long g_na_scratch[kNaBlocks * kNaSlot + kNaSlot];
constexpr size_t kNaScratchBytes = sizeof(long long) * (kNaBlocks * kNaSlot + kNaSlot);
static_assert(kNaScratchBytes <= 80 * 1024, "keep the per-device scratch modest");

std::mutex g_na_mutex;
long long *g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current (in host code the array's name is only a
// stand-in for the symbol, not an address a kernel may use).
int na_scratch(long long **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return CCMC_E_CUDA;
  if (dev < 0 || dev >= kNaMaxDevices) return CCMC_E_INVAL;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || p == nullptr) return CCMC_E_CUDA;
    g_na_ptr[dev] = static_cast<long long *>(p);
  }
  *out = g_na_ptr[dev];
  return CCMC_OK;
}

__device__ __forceinline__ long long na_warp_sum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Observables of Eq. (3) by definition, one site per loop step: the site's own
// terms and its right and down bonds.  Same reduction as the library's recount
// (block partials, last block to arrive sums them), with the partials and the
// counter in `scratch`.
__global__ void __launch_bounds__(kNaThreads) na_recount_kernel(const uint8_t *st, int Lx, int Ly,
                                                                long long *scratch,
                                                                long long *out) {
  const int kS[4] = {0, 0, 1, -1};
  const int kG[4] = {1, -1, 0, 0};
  int c[7] = {0, 0, 0, 0, 0, 0, 0};  // Nc, BV, BJ, M, M_stag, S_sum, S_stag
  const int64_t N = (int64_t)Lx * Ly;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / Lx), x = (int)(i - (int64_t)y * Lx);
    const int s = st[i] & 3;
    const int r = st[(int64_t)y * Lx + (x + 1 == Lx ? 0 : x + 1)] & 3;
    const int d = st[(int64_t)(y + 1 == Ly ? 0 : y + 1) * Lx + x] & 3;
    const int sgn = ((x + y) & 1) ? -1 : 1;
    c[0] += kS[s] * kS[s];
    c[1] += kS[s] * (kS[r] + kS[d]);
    c[2] += kG[s] * (kG[r] + kG[d]);
    c[3] += kG[s];
    c[4] += sgn * kG[s];
    c[5] += kS[s];
    c[6] += sgn * kS[s];
  }
  __shared__ long long red[kNaThreads / 32][7];
  __shared__ bool last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const long long v = na_warp_sum((long long)c[k]);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    long long v = 0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) v += red[wv][threadIdx.x];
    scratch[blockIdx.x * kNaSlot + threadIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  unsigned long long *ticket =
      reinterpret_cast<unsigned long long *>(scratch + kNaBlocks * kNaSlot);
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1ull) == (unsigned long long)(gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 7) {
    long long v = 0;
    for (unsigned b = 0; b < gridDim.x; ++b)
      v += *(volatile long long *)(scratch + (int64_t)b * kNaSlot + threadIdx.x);
    out[threadIdx.x] = v;
  }
  if (threadIdx.x == 0) *ticket = 0ull;
}

}  // namespace

extern "C" int ccmc_recount_noalloc(const uint8_t *d_state, int Lx, int Ly, int64_t *d_out,
                                    void *cuda_stream) {
  if (!d_state || !d_out || Lx < 2 || Ly < 2) return CCMC_E_INVAL;
  const int64_t N = (int64_t)Lx * Ly;
  if (N > kNaMaxSites) return CCMC_E_INVAL;  // beyond the largest lattice supported
  long long *scratch = nullptr;
  const int rc = na_scratch(&scratch);
  if (rc != CCMC_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the arrival counter must start at zero even if an earlier call was cut short
  if (cudaMemsetAsync(scratch + kNaBlocks * kNaSlot, 0, sizeof(long long), s) != cudaSuccess)
    return CCMC_E_CUDA;
  int64_t blocks = (N + (int64_t)kNaThreads * 8 - 1) / ((int64_t)kNaThreads * 8);
  if (blocks > kNaBlocks) blocks = kNaBlocks;
  if (blocks < 1) blocks = 1;
  na_recount_kernel<<<(int)blocks, kNaThreads, 0, s>>>(d_state, Lx, Ly, scratch,
                                                       reinterpret_cast<long long *>(d_out));
  return cudaGetLastError() == cudaSuccess ? CCMC_OK : CCMC_E_CUDA;
}
