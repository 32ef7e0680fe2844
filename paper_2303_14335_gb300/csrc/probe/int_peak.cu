// int_peak.cu -- measured throughput of the integer pipes the search uses.
//
// The search kernel's work is plain 32-bit integer arithmetic: logic ops and
// adds on bit fields, and population counts.  Its roofline denominator is
// derived from lane counts and the clock; these two kernels measure what the
// pipes actually sustain on this device, for the same mix:
//   mode 0: acc = (acc ^ x) + i        -- logic + add, 2 ops per step
//   mode 1: acc += popc(x ^ acc)        -- logic + popcount + add, 3 ops
// Each thread runs 8 independent chains; the grid fills every SM.  Built
// into a library of its own (libmpld_probe.so) for the benchmark's roofline
// context; libmpld.so does not contain it.
#include <cuda_runtime.h>

#include <stdint.h>

#include "../../../include/mpld.h"

namespace {

__global__ void __launch_bounds__(256) int_pipe_kernel(uint32_t seed, int iters, int popc,
                                                       uint32_t *sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[8], acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    x[j] = (t + 1u) * 0x9E3779B9u + (uint32_t)j * 0x85EBCA6Bu + seed;
    acc[j] = x[j] >> 3;
  }
  if (popc) {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] += (uint32_t)__popc(x[j] ^ acc[j]);
    }
  } else {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = (acc[j] ^ x[j]) + (uint32_t)i;
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s ^= acc[j];
  if (s == seed + 0x12345u) sink[t & 255u] = s;   // keeps the chains live
}

}  // namespace

// out[0]: logic + add throughput, out[1]: logic + popcount + add throughput,
// both in 10^9 integer ops per second over every SM of the current device.
extern "C" int mpld_probe_int_peak(int iters, double *out) {
  if (!out || iters < 16) return MPLD_E_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MPLD_E_CUDA;
  const int threads = 256, blocks = sms * 8;
  uint32_t *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MPLD_OK;
  if (cudaMalloc((void **)&sink, 1024) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = MPLD_E_CUDA;
  }
  for (int mode = 0; mode < 2 && rc == MPLD_OK; ++mode) {
    int_pipe_kernel<<<blocks, threads>>>(7u, iters / 8, mode, sink);   // warm-up
    cudaEventRecord(e0);
    int_pipe_kernel<<<blocks, threads>>>(11u, iters, mode, sink);
    cudaEventRecord(e1);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        ms <= 0.f) {
      rc = MPLD_E_CUDA;
      break;
    }
    const double ops = (double)blocks * threads * (double)iters * 8.0 * (mode ? 3.0 : 2.0);
    out[mode] = ops / ((double)ms * 1e-3) / 1e9;
  }
  if (rc != MPLD_OK) cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  return rc;
}
