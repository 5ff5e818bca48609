// Arithmetic-pipe probes: the measured denominators of the roofline fractions for kernels
// bound by the FP64 or FP32 SIMT pipes (no tensor cores), where no library routine gives a
// clean peak. Each thread runs kChains independent multiply-add chains for `iters` rounds,
// so the pipe, not the dependency latency, limits the rate; the result is stored so the
// compiler keeps the work. Work per launch: blocks * threads * iters * kChains * 2 flop
// (kinds 0, 1); kinds 2 and 3 run the same loop on one lane per warp, so a launch takes as
// many warp instructions with 1/32 of the lanes' work: equal times mean the pipe costs the
// same per warp instruction whatever the active lanes.
#include <cuda_runtime.h>

#include "../../include/nmc.h"

namespace {

constexpr int kChains = 8;

// active: lanes per warp that run the loop (the others skip it), so that the rate per warp
// instruction can be compared with the rate per lane
template <typename T>
__global__ void k_fma_loop(int iters, T a, T b, T* out, int active) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  if ((int)(threadIdx.x & 31) < active) {
    for (int k = 0; k < iters; ++k) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" nmc_status nmc_fma_probe(int kind, int blocks, int threads, int iters, void* d_out,
                                    void* cuda_stream) {
  if (kind < 0 || kind > 3 || blocks < 1 || threads < 32 || threads > 1024 || iters < 1 ||
      !d_out)
    return NMC_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int active = kind >= 2 ? 1 : 32;   // kinds 2, 3: one active lane per warp
  if (kind % 2 == 0)
    k_fma_loop<double><<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, (double*)d_out, active);
  else
    k_fma_loop<float><<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-5f, (float*)d_out, active);
  return cudaGetLastError() == cudaSuccess ? NMC_OK : NMC_ECUDA;
}
