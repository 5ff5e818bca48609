// Arithmetic-pipe probes: the measured denominators of the roofline fractions for kernels
// bound by the FP64 or FP32 SIMT pipes (no tensor cores), where no library routine gives a
// clean peak. Each thread runs kChains independent multiply-add chains for `iters` rounds,
// so the pipe, not the dependency latency, limits the rate; the result is stored so the
// compiler keeps the work. Work per launch: blocks * threads * iters * kChains * 2 flop.
#include <cuda_runtime.h>

#include "../../include/nmc.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void k_fma_loop(int iters, T a, T b, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" nmc_status nmc_fma_probe(int kind, int blocks, int threads, int iters, void* d_out,
                                    void* cuda_stream) {
  if ((kind != 0 && kind != 1) || blocks < 1 || threads < 32 || threads > 1024 || iters < 1 ||
      !d_out)
    return NMC_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (kind == 0)
    k_fma_loop<double><<<blocks, threads, 0, st>>>(iters, 0.999999, 1e-7, (double*)d_out);
  else
    k_fma_loop<float><<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-5f, (float*)d_out);
  return cudaGetLastError() == cudaSuccess ? NMC_OK : NMC_ECUDA;
}
