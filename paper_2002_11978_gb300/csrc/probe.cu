// L2 read-bandwidth probe (tsfde_probe_l2_read).
//
// The level solves keep their Krylov vectors and FFT work buffers resident in
// L2, so the bandwidth they could at best draw is L2's, not HBM's.  This
// kernel measures that ceiling on the running GPU: every resident thread
// streams 16-byte loads that bypass L1 (ld.global.cg) over a buffer the caller
// sized to fit in L2, `reps` times over.  The loads feed an XOR that is stored
// only under a condition the data never meets, which keeps them alive without
// adding stores to the traffic.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "../../include/tsfde.h"

namespace {

constexpr int kProbeThreads = 512;

__global__ void __launch_bounds__(kProbeThreads) k_l2_read(const uint4* __restrict__ p, size_t n16, int reps,
                                                           unsigned* __restrict__ sink) {
  unsigned acc = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll 1
  for (int r = 0; r < reps; ++r) {
#pragma unroll 8
    for (size_t i = i0; i < n16; i += stride) {
      const uint4 v = __ldcg(p + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    acc = (acc << 1) | (acc >> 31);
  }
  if (acc == 0x9e3779b9u && sink) sink[0] = acc;
}

}  // namespace

extern "C" int tsfde_probe_l2_read(const void* buf, size_t bytes, int reps, void* stream) {
  if (!buf || bytes < 16 || (bytes & 15) || ((uintptr_t)buf & 15) || reps < 1) return TSFDE_EINVAL;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TSFDE_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TSFDE_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_l2_read, kProbeThreads, 0) != cudaSuccess ||
      per_sm < 1)
    return TSFDE_ECUDA;
  k_l2_read<<<sms * per_sm, kProbeThreads, 0, (cudaStream_t)stream>>>(
      static_cast<const uint4*>(buf), bytes / 16, reps, nullptr);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "tsfde_probe_l2_read: %s\n", cudaGetErrorString(e));
    return TSFDE_ECUDA;
  }
  return TSFDE_OK;
}
