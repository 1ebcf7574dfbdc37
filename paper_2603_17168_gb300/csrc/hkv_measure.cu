// Random-access rate of device memory: the ceiling that a hash table's
// scattered accesses meet long before the sequential copy bandwidth. The
// probe touches uniformly random, naturally aligned units of 8, 32 or 128
// bytes in a buffer far larger than L2. A 128-byte unit is moved by 8 lanes
// with 16-byte accesses (one line per 8 lanes, as a probe group reads a
// digest line), a 32-byte unit by 2 lanes, an 8-byte unit by one lane; every
// thread keeps 8 independent accesses in flight so that the rate measured is
// the memory system's, not the probe's latency.
#include <algorithm>

#include "hkv_internal.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kInFlight = 8;

// n_units is a power of two: a mask, not a 64-bit division, keeps the
// probe's own arithmetic far below the memory system's rate.
__device__ __forceinline__ uint64_t unit_of(uint64_t a, uint64_t n_units) {
  return hkv::fmix64(a * 0x9E3779B97F4A7C15ull + 0x5851F42D4C957F2Dull) & (n_units - 1);
}

template <int UNIT, bool WRITE>
__global__ void __launch_bounds__(kProbeThreads)
    random_access_kernel(uint4* __restrict__ buf, uint64_t n_units, uint64_t accesses,
                         unsigned long long* sink) {
  constexpr int LPA = UNIT >= 16 ? UNIT / 16 : 1;  // lanes per access
  const uint64_t tid = blockIdx.x * (uint64_t)kProbeThreads + threadIdx.x;
  const uint64_t streams = (uint64_t)gridDim.x * kProbeThreads / LPA;
  const int sub = threadIdx.x % LPA;
  unsigned long long acc = 0;
  for (uint64_t a0 = tid / LPA; a0 < accesses; a0 += streams * kInFlight) {
    uint64_t unit[kInFlight];
#pragma unroll
    for (int k = 0; k < kInFlight; ++k) unit[k] = unit_of(a0 + k * streams, n_units);
    if (UNIT == 8) {
      const unsigned long long* p = reinterpret_cast<const unsigned long long*>(buf);
      unsigned long long v[kInFlight];
#pragma unroll
      for (int k = 0; k < kInFlight; ++k) {
        const bool in = a0 + k * streams < accesses;
        if (WRITE) {
          if (in) reinterpret_cast<unsigned long long*>(buf)[unit[k]] = a0;
          v[k] = 0;
        } else {
          v[k] = in ? __ldg(p + unit[k]) : 0ull;
        }
      }
#pragma unroll
      for (int k = 0; k < kInFlight; ++k) acc += v[k];
    } else {
      uint4 v[kInFlight];
#pragma unroll
      for (int k = 0; k < kInFlight; ++k) {
        const bool in = a0 + k * streams < accesses;
        uint4* q = buf + unit[k] * LPA + sub;
        if (WRITE) {
          if (in) *q = make_uint4((uint32_t)a0, (uint32_t)k, 0u, 0u);
          v[k] = make_uint4(0u, 0u, 0u, 0u);
        } else {
          v[k] = in ? __ldg(q) : make_uint4(0u, 0u, 0u, 0u);
        }
      }
#pragma unroll
      for (int k = 0; k < kInFlight; ++k) acc += v[k].x ^ v[k].w;
    }
  }
  if (acc == 0x5EEDull) *sink = acc;  // keeps the loads alive
}

template <int UNIT, bool WRITE>
void launch_probe(uint4* buf, uint64_t n_units, uint64_t accesses, unsigned long long* sink,
                  unsigned grid) {
  random_access_kernel<UNIT, WRITE><<<grid, kProbeThreads>>>(buf, n_units, accesses, sink);
}

}  // namespace

extern "C" hkv_status hkv_measure_random_access(uint32_t unit_bytes, int write,
                                                uint64_t buffer_bytes, uint64_t accesses,
                                                int repeats, double* accesses_per_s) {
  if (!accesses_per_s || (unit_bytes != 8 && unit_bytes != 32 && unit_bytes != 128) ||
      buffer_bytes < (1ull << 20) || buffer_bytes % 128 || accesses == 0 || repeats < 1) {
    hkv::set_last_error("random-access measurement arguments");
    return HKV_ERR_INVALID_ARG;
  }
  void* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, buffer_bytes + 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    hkv::set_last_error("random-access measurement buffer");
    return HKV_ERR_OOM;
  }
  uint4* buf = static_cast<uint4*>(mem);
  auto* sink = reinterpret_cast<unsigned long long*>(static_cast<char*>(mem) + buffer_bytes);
  uint64_t n_units = 1;
  while (n_units * 2 <= buffer_bytes / unit_bytes) n_units *= 2;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)sms * 4;
  auto run = [&]() {
    if (unit_bytes == 8)
      write ? launch_probe<8, true>(buf, n_units, accesses, sink, grid)
            : launch_probe<8, false>(buf, n_units, accesses, sink, grid);
    else if (unit_bytes == 32)
      write ? launch_probe<32, true>(buf, n_units, accesses, sink, grid)
            : launch_probe<32, false>(buf, n_units, accesses, sink, grid);
    else
      write ? launch_probe<128, true>(buf, n_units, accesses, sink, grid)
            : launch_probe<128, false>(buf, n_units, accesses, sink, grid);
  };
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaMemset(mem, 0x5A, buffer_bytes);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  double best = 0.0;
  if (e == cudaSuccess) {
    run();  // warm-up
    for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
      cudaEventRecord(a);
      run();
      cudaEventRecord(b);
      e = cudaEventSynchronize(b);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      if (e == cudaSuccess && ms > 0.f) best = std::max(best, accesses / (ms * 1e-3));
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(mem);
  if (e != cudaSuccess) return hkv::cuda_status(e, "random-access measurement");
  *accesses_per_s = best;
  return HKV_OK;
}
