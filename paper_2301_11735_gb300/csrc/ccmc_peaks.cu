// ccmc_peaks.cu -- measured on-chip bandwidth peaks of the device (diagnostics
// for the roofline of the shared-memory and L2 paths; the paper has no
// counterpart).  Each kernel streams reads that cannot be elided (the values
// feed a result that is stored only if it matches an impossible key) at the
// widest access the path offers, from every SM, and the host times a launch
// with CUDA events after a warm-up launch.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/ccmc.h"

namespace {

constexpr int kSmemThreads = 512;
constexpr int kSmemBytes = 32 * 1024;  // per CTA: static shared memory
constexpr int kSmemIters = 4096;       // 16-byte reads per thread: kSmemIters * 8

// Every thread reads kSmemIters * 8 uint4 from its CTA's shared buffer, warp
// by warp over consecutive 16-byte chunks (four conflict-free 128-byte
// wavefronts a warp-read), eight independent reads in flight.
__global__ void __launch_bounds__(kSmemThreads) smem_read_kernel(uint32_t key, uint4 *sink) {
  __shared__ uint4 buf[kSmemBytes / 16];
  for (int i = threadIdx.x; i < kSmemBytes / 16; i += blockDim.x)
    buf[i] = make_uint4(i, i * 3u, i * 5u, i * 7u);
  __syncthreads();
  uint4 acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = make_uint4(0u, 0u, 0u, 0u);
  constexpr int kN = kSmemBytes / 16;
  int idx = threadIdx.x;
#pragma unroll 1
  for (int it = 0; it < kSmemIters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint4 v = buf[(idx + k * (kN / 8)) & (kN - 1)];  // eight distinct addresses
      acc[k].x ^= v.x;
      acc[k].y ^= v.y;
      acc[k].z ^= v.z;
      acc[k].w ^= v.w;
    }
    idx = (idx + 32) & (kN - 1);
  }
  uint4 r = acc[0];
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    r.x ^= acc[k].x;
    r.y ^= acc[k].y;
    r.z ^= acc[k].z;
    r.w ^= acc[k].w;
  }
  if (r.x == key && r.y == key) sink[blockIdx.x * blockDim.x + threadIdx.x] = r;
}
static_assert((kSmemBytes / 16 & (kSmemBytes / 16 - 1)) == 0, "a power-of-two buffer");

// Reads of a buffer that L2 holds, 16 bytes a thread per step, bypassing L1
// (ld.global.cg), every thread striding over the whole buffer.
__global__ void __launch_bounds__(256) l2_read_kernel(const uint4 *__restrict__ buf, int64_t n,
                                                      int reps, uint32_t key, uint4 *sink) {
  uint4 acc = make_uint4(0u, 0u, 0u, 0u);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
      const uint4 v = __ldcg(buf + i);
      acc.x ^= v.x;
      acc.y ^= v.y;
      acc.z ^= v.z;
      acc.w ^= v.w;
    }
  if (acc.x == key && acc.y == key) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void fill_kernel(uint4 *buf, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    buf[i] = make_uint4((uint32_t)i, (uint32_t)(i >> 7), 3u, 5u);
}

int sm_count(int *sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || *sms < 1)
    return CCMC_E_CUDA;
  return CCMC_OK;
}

}  // namespace

extern "C" int ccmc_peak_smem_read(double *bytes_per_s) {
  if (!bytes_per_s) return CCMC_E_INVAL;
  int sms = 0;
  if (sm_count(&sms) != CCMC_OK) return CCMC_E_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smem_read_kernel, kSmemThreads, 0) !=
          cudaSuccess ||
      per_sm < 1)
    return CCMC_E_CUDA;
  const int grid = sms * per_sm;
  uint4 *sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = CCMC_E_CUDA;
  if (cudaMalloc(&sink, sizeof(uint4) * (size_t)grid * kSmemThreads) != cudaSuccess) {
    cudaGetLastError();
    return CCMC_E_NOMEM;
  }
  if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
    smem_read_kernel<<<grid, kSmemThreads>>>(0x9E3779B9u, sink);  // warm-up
    cudaEventRecord(a);
    smem_read_kernel<<<grid, kSmemThreads>>>(0x9E3779B9u, sink);
    cudaEventRecord(b);
    float ms = 0.f;
    if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess &&
        ms > 0.f) {
      const double bytes = (double)grid * kSmemThreads * kSmemIters * 8.0 * 16.0;
      *bytes_per_s = bytes / (ms * 1e-3);
      rc = CCMC_OK;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(sink);
  return rc;
}

extern "C" int ccmc_peak_l2_read(int64_t buffer_bytes, double *bytes_per_s) {
  if (!bytes_per_s || buffer_bytes < (1 << 20) || buffer_bytes > ((int64_t)1 << 30))
    return CCMC_E_INVAL;
  int sms = 0;
  if (sm_count(&sms) != CCMC_OK) return CCMC_E_CUDA;
  const int64_t n = buffer_bytes / 16;
  const int grid = sms * 8, reps = 8;
  uint4 *buf = nullptr, *sink = nullptr;
  if (cudaMalloc(&buf, sizeof(uint4) * (size_t)n) != cudaSuccess ||
      cudaMalloc(&sink, sizeof(uint4) * (size_t)grid * 256) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(buf);
    return CCMC_E_NOMEM;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = CCMC_E_CUDA;
  if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
    fill_kernel<<<grid, 256>>>(buf, n);
    l2_read_kernel<<<grid, 256>>>(buf, n, 1, 0x9E3779B9u, sink);  // warm-up: the buffer into L2
    cudaEventRecord(a);
    l2_read_kernel<<<grid, 256>>>(buf, n, reps, 0x9E3779B9u, sink);
    cudaEventRecord(b);
    float ms = 0.f;
    if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess &&
        ms > 0.f) {
      *bytes_per_s = (double)n * 16.0 * reps / (ms * 1e-3);
      rc = CCMC_OK;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(buf);
  cudaFree(sink);
  return rc;
}
