// Convolutional field generator (include/nmc_cgen.h): four periodic 3D convolutions
// (3 x 3 x 3 kernels, channels 1 -> C -> C -> C -> 1, ReLU between) mapping N(0,1) noise
// to Bernoulli logits per field entry, trained by maximum likelihood on DQMC fields.
//
// Every convolution reads BF16 operands and accumulates in FP32 (SIMT FMA): the activations
// and the gradients flowing between layers are stored as BF16, the weights are used as a
// BF16 copy of the FP32 master weights. Kernels, all over the batch [n][C][S] with
// S = L_tau * Ly * Lx (x fastest, so the last layer's entry p is field entry (i, l) at
// p = l N + i):
//   k_cg_fwd     out[n][co][p] = b[co] + sum_ci sum_k W[co][ci][k] in[n][ci][p + d_k]
//                (one thread per output entry; the CTA's output channel's weights in
//                shared memory), then ReLU and BF16, or FP32 logits for the last layer;
//   k_cg_loss    the Bernoulli negative log-likelihood and dL/dlogit = (sigmoid(l) - y) /
//                (n S), as BF16 for the backward convolutions;
//   k_cg_bwd_in  dL/din[n][ci][q] = sum_co sum_k W[co][ci][k] g[n][co][q - d_k], times the
//                ReLU mask of that input (it is the previous layer's output), as BF16;
//   k_cg_bwd_w   dL/dW[co][ci][k] = sum_{n,p} g[n][co][p] in[n][ci][p + d_k] and
//                dL/db[co] = sum g[n][co][p]: one CTA per (ci, co), 27 + 1 FP32 partial
//                sums per thread, then a block reduction;
//   k_cg_adam    Adam on the FP32 master weights, then their BF16 copy.
// Noise and Bernoulli draws are Philox4x32-10 words (counter (p, sample, stream, tag)).
#include <cuda_bf16.h>

#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "nmc_cgen.h"
#include "nmc_internal.cuh"

using nmc::philox4x32_10;

namespace {

constexpr int kLayers = 4;
constexpr int kK = 27;             // 3 x 3 x 3 kernel entries
constexpr uint32_t kTagNoise = 5u, kTagDraw = 6u, kTagInit = 7u;
constexpr int kFwdThreads = 128;
constexpr int kWThreads = 256;

struct Dims {
  int T, A, B;   // L_tau, Ly, Lx
  __host__ __device__ int S() const { return T * A * B; }
};

__device__ __forceinline__ float bf(__nv_bfloat16 v) { return __bfloat162float(v); }

// entry p + d_k (periodic), d_k = (k / 9 - 1, (k / 3) % 3 - 1, k % 3 - 1)
__device__ __forceinline__ int neighbour(const Dims& d, int t, int a, int b, int k, int sign) {
  const int dt = sign * (k / 9 - 1), da = sign * ((k / 3) % 3 - 1), db = sign * (k % 3 - 1);
  int tt = t + dt, aa = a + da, bb = b + db;
  tt += tt < 0 ? d.T : tt >= d.T ? -d.T : 0;
  aa += aa < 0 ? d.A : aa >= d.A ? -d.A : 0;
  bb += bb < 0 ? d.B : bb >= d.B ? -d.B : 0;
  return (tt * d.A + aa) * d.B + bb;
}

__global__ void k_cg_fwd(const __nv_bfloat16* __restrict__ in, int Cin,
                         const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
                         int Cout, Dims d, int relu, __nv_bfloat16* __restrict__ out_h,
                         float* __restrict__ out_f) {
  extern __shared__ float sw[];   // [Cin][27] of output channel co
  const int co = blockIdx.y, n = blockIdx.z, S = d.S();
  for (int e = threadIdx.x; e < Cin * kK; e += blockDim.x) sw[e] = bf(W[(long long)co * Cin * kK + e]);
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= S) return;
  const int t = p / (d.A * d.B), rem = p - t * d.A * d.B, a = rem / d.B, b = rem - a * d.B;
  const __nv_bfloat16* x = in + (long long)n * Cin * S;
  float acc = bias[co];
  for (int k = 0; k < kK; ++k) {
    const int q = neighbour(d, t, a, b, k, 1);
    for (int ci = 0; ci < Cin; ++ci) acc = fmaf(sw[ci * kK + k], bf(x[(long long)ci * S + q]), acc);
  }
  if (relu) out_h[((long long)n * Cout + co) * S + p] = __float2bfloat16_rn(fmaxf(acc, 0.f));
  else out_f[((long long)n * Cout + co) * S + p] = acc;
}

__global__ void k_cg_loss(const float* __restrict__ logits, const int8_t* __restrict__ fields,
                          long long total, float inv_count, __nv_bfloat16* __restrict__ g,
                          double* __restrict__ loss_sum) {
  __shared__ double red[kWThreads / 32];
  double part = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const float l = logits[e];
    const float y = fields[e] > 0 ? 1.f : 0.f;
    // softplus(l) - y l, with softplus(l) = max(l, 0) + log1p(exp(-|l|))
    part += (double)(fmaxf(l, 0.f) + log1pf(expf(-fabsf(l))) - y * l);
    const float sg = 1.f / (1.f + expf(-l));
    g[e] = __float2bfloat16_rn((sg - y) * inv_count);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(loss_sum, s);
  }
}

__global__ void k_cg_bwd_in(const __nv_bfloat16* __restrict__ g, int Cout,
                            const __nv_bfloat16* __restrict__ W, int Cin, Dims d,
                            const __nv_bfloat16* __restrict__ act, __nv_bfloat16* __restrict__ gin) {
  extern __shared__ float sw[];   // [Cout][27] of input channel ci
  const int ci = blockIdx.y, n = blockIdx.z, S = d.S();
  for (int e = threadIdx.x; e < Cout * kK; e += blockDim.x) {
    const int co = e / kK, k = e - co * kK;
    sw[e] = bf(W[((long long)co * Cin + ci) * kK + k]);
  }
  __syncthreads();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= S) return;
  const long long o = ((long long)n * Cin + ci) * S + q;
  if (!(bf(act[o]) > 0.f)) {   // the ReLU's derivative is 0 there
    gin[o] = __float2bfloat16_rn(0.f);
    return;
  }
  const int t = q / (d.A * d.B), rem = q - t * d.A * d.B, a = rem / d.B, b = rem - a * d.B;
  const __nv_bfloat16* gg = g + (long long)n * Cout * S;
  float acc = 0.f;
  for (int k = 0; k < kK; ++k) {
    const int p = neighbour(d, t, a, b, k, -1);   // q - d_k
    for (int co = 0; co < Cout; ++co) acc = fmaf(sw[co * kK + k], bf(gg[(long long)co * S + p]), acc);
  }
  gin[o] = __float2bfloat16_rn(acc);
}

__global__ void __launch_bounds__(kWThreads)
k_cg_bwd_w(const __nv_bfloat16* __restrict__ g, int Cout, const __nv_bfloat16* __restrict__ h,
           int Cin, Dims d, int n, float* __restrict__ gW, float* __restrict__ gb) {
  __shared__ float red[kWThreads / 32][kK + 1];
  const int ci = blockIdx.x, co = blockIdx.y, S = d.S();
  float acc[kK + 1];
#pragma unroll
  for (int k = 0; k <= kK; ++k) acc[k] = 0.f;
  const long long total = (long long)n * S;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int s = (int)(e / S), p = (int)(e - (long long)s * S);
    const float gv = bf(g[((long long)s * Cout + co) * S + p]);
    if (gv == 0.f) continue;
    const int t = p / (d.A * d.B), rem = p - t * d.A * d.B, a = rem / d.B, b = rem - a * d.B;
    const __nv_bfloat16* x = h + ((long long)s * Cin + ci) * S;
#pragma unroll
    for (int k = 0; k < kK; ++k) acc[k] = fmaf(gv, bf(x[neighbour(d, t, a, b, k, 1)]), acc[k]);
    acc[kK] += gv;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k <= kK; ++k) {
    float v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x <= kK) {
    float s = 0.f;
    for (int w = 0; w < kWThreads / 32; ++w) s += red[w][threadIdx.x];
    if (threadIdx.x < kK) gW[((long long)co * Cin + ci) * kK + threadIdx.x] = s;
    else if (ci == 0) gb[co] = s;
  }
}

__global__ void k_cg_adam(float* __restrict__ th, const float* __restrict__ gr,
                          float* __restrict__ m, float* __restrict__ v, long long n, float lr,
                          float c1, float c2, __nv_bfloat16* __restrict__ thb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = gr[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float x = th[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    th[i] = x;
    thb[i] = __float2bfloat16_rn(x);
  }
}

__global__ void k_cg_to_bf16(const float* __restrict__ x, long long n, __nv_bfloat16* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void k_cg_noise(long long n0, int n, int S, uint32_t stream, uint32_t k0, uint32_t k1,
                           __nv_bfloat16* __restrict__ z) {
  const long long total = (long long)n * S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / S), p = (int)(e - (long long)s * S);
    uint32_t c[4] = {(uint32_t)p, (uint32_t)(n0 + s), stream, kTagNoise};
    philox4x32_10(c, k0, k1);
    const float u1 = (float)(((double)c[0] + 0.5) * 2.3283064365386962890625e-10);
    const float u2 = (float)((double)c[1] * 2.3283064365386962890625e-10);
    const float r = sqrtf(-2.f * logf(u1));
    z[e] = __float2bfloat16_rn(r * cosf(6.283185307179586f * u2));
  }
}

__global__ void k_cg_draw(const float* __restrict__ logits, long long n0, int n, int S,
                          uint32_t stream, uint32_t k0, uint32_t k1, int8_t* __restrict__ f) {
  const long long total = (long long)n * S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(e / S), p = (int)(e - (long long)s * S);
    uint32_t c[4] = {(uint32_t)p, (uint32_t)(n0 + s), stream, kTagDraw};
    philox4x32_10(c, k0, k1);
    const double u = (double)c[0] * 2.3283064365386962890625e-10;
    const double pr = 1.0 / (1.0 + exp(-(double)logits[e]));
    f[e] = u < pr ? (int8_t)1 : (int8_t)-1;
  }
}

int grid_for(long long n, int threads) {
  const long long b = (n + threads - 1) / threads;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

struct nmc_cgen {
  Dims d{};
  int C = 0, max_batch = 0;
  uint64_t seed = 0;
  cudaStream_t st = nullptr;
  int device = 0;
  int cin[kLayers], cout[kLayers];
  long long oW[kLayers], ob[kLayers], P = 0;
  float *th = nullptr, *gr = nullptr, *m = nullptr, *v = nullptr, *logits = nullptr;
  __nv_bfloat16 *thb = nullptr, *act[kLayers] = {}, *gA = nullptr, *gB = nullptr;
  double* dloss = nullptr;
  long long steps = 0;
  std::vector<void*> allocs;
};

namespace {

template <typename T>
nmc_status cg_alloc(nmc_cgen* g, T*& p, long long n) {
  if (cudaMalloc((void**)&p, (size_t)(n > 0 ? n : 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
    return NMC_ENOMEM;
  }
  g->allocs.push_back(p);
  return NMC_OK;
}

#define CG_TRY(expr)                  \
  do {                                \
    const nmc_status s_ = (expr);     \
    if (s_ != NMC_OK) return s_;      \
  } while (0)

nmc_status cg_last(void) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? NMC_OK : NMC_ECUDA;
}

void forward(nmc_cgen* g, int n) {
  const int S = g->d.S();
  for (int j = 0; j < kLayers; ++j) {
    const dim3 grid((S + kFwdThreads - 1) / kFwdThreads, g->cout[j], n);
    const bool last = j == kLayers - 1;
    k_cg_fwd<<<grid, kFwdThreads, g->cin[j] * kK * sizeof(float), g->st>>>(
        g->act[j], g->cin[j], g->thb + g->oW[j], g->th + g->ob[j], g->cout[j], g->d, last ? 0 : 1,
        last ? nullptr : g->act[j + 1], last ? g->logits : nullptr);
  }
}

// loss of the current logits against d_fields into g->dloss (sum), gradients into g->gr
void backward(nmc_cgen* g, const int8_t* d_fields, int n) {
  const int S = g->d.S();
  const long long total = (long long)n * S;
  cudaMemsetAsync(g->dloss, 0, sizeof(double), g->st);
  k_cg_loss<<<grid_for(total, kWThreads), kWThreads, 0, g->st>>>(
      g->logits, d_fields, total, 1.f / (float)total, g->gA, g->dloss);
  __nv_bfloat16* gcur = g->gA;
  __nv_bfloat16* gnext = g->gB;
  for (int j = kLayers - 1; j >= 0; --j) {
    k_cg_bwd_w<<<dim3(g->cin[j], g->cout[j]), kWThreads, 0, g->st>>>(
        gcur, g->cout[j], g->act[j], g->cin[j], g->d, n, g->gr + g->oW[j], g->gr + g->ob[j]);
    if (j > 0) {
      const dim3 grid((S + kFwdThreads - 1) / kFwdThreads, g->cin[j], n);
      k_cg_bwd_in<<<grid, kFwdThreads, g->cout[j] * kK * sizeof(float), g->st>>>(
          gcur, g->cout[j], g->thb + g->oW[j], g->cin[j], g->d, g->act[j], gnext);
      __nv_bfloat16* t = gcur;
      gcur = gnext;
      gnext = t;
    }
  }
}

void noise(nmc_cgen* g, long long n0, int n, uint32_t stream) {
  const int S = g->d.S();
  k_cg_noise<<<grid_for((long long)n * S, 256), 256, 0, g->st>>>(
      n0, n, S, stream, (uint32_t)g->seed, (uint32_t)(g->seed >> 32), g->act[0]);
}

}  // namespace

extern "C" {

nmc_status nmc_cgen_create(int Lx, int Ly, int L_tau, int channels, uint64_t seed, int max_batch,
                           void* cuda_stream, nmc_cgen** out) {
  if (!out) return NMC_EINVAL;
  *out = nullptr;
  if (Lx < 1 || Ly < 1 || L_tau < 1 || channels < 1 || channels > 64 || max_batch < 1 ||
      (long long)Lx * Ly * L_tau > (1 << 24) || max_batch > 65535)
    return NMC_EINVAL;
  nmc_cgen* g = new (std::nothrow) nmc_cgen();
  if (!g) return NMC_ENOMEM;
  g->d = Dims{L_tau, Ly, Lx};
  g->C = channels;
  g->max_batch = max_batch;
  g->seed = seed;
  g->st = (cudaStream_t)cuda_stream;
  cudaGetDevice(&g->device);
  const int C = channels;
  const int ci[kLayers] = {1, C, C, C}, co[kLayers] = {C, C, C, 1};
  long long off = 0;
  for (int j = 0; j < kLayers; ++j) {
    g->cin[j] = ci[j];
    g->cout[j] = co[j];
    g->oW[j] = off;
    off += (long long)co[j] * ci[j] * kK;
    g->ob[j] = off;
    off += co[j];
  }
  g->P = off;
  const long long S = g->d.S(), nb = max_batch;
  nmc_status s = NMC_OK;
  if (s == NMC_OK) s = cg_alloc(g, g->th, g->P);
  if (s == NMC_OK) s = cg_alloc(g, g->gr, g->P);
  if (s == NMC_OK) s = cg_alloc(g, g->m, g->P);
  if (s == NMC_OK) s = cg_alloc(g, g->v, g->P);
  if (s == NMC_OK) s = cg_alloc(g, g->thb, g->P);
  if (s == NMC_OK) s = cg_alloc(g, g->logits, nb * S);
  for (int j = 0; j < kLayers && s == NMC_OK; ++j) s = cg_alloc(g, g->act[j], nb * ci[j] * S);
  if (s == NMC_OK) s = cg_alloc(g, g->gA, nb * C * S);
  if (s == NMC_OK) s = cg_alloc(g, g->gB, nb * C * S);
  if (s == NMC_OK) s = cg_alloc(g, g->dloss, 1);
  if (s != NMC_OK) {
    nmc_cgen_destroy(g);
    return s;
  }
  // Glorot-uniform weights, zero biases
  std::vector<float> th((size_t)g->P, 0.f);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int j = 0; j < kLayers; ++j) {
    const double bound = std::sqrt(6.0 / (kK * (double)(ci[j] + co[j])));
    for (long long e = 0; e < (long long)co[j] * ci[j] * kK; ++e) {
      uint32_t c[4] = {(uint32_t)e, (uint32_t)j, 0u, kTagInit};
      philox4x32_10(c, k0, k1);
      const double u = (double)c[0] * 2.3283064365386962890625e-10;
      th[(size_t)(g->oW[j] + e)] = (float)((2.0 * u - 1.0) * bound);
    }
  }
  s = nmc_cgen_set_params(g, th.data());
  if (s != NMC_OK) {
    nmc_cgen_destroy(g);
    return s;
  }
  *out = g;
  return NMC_OK;
}

nmc_status nmc_cgen_n_params(const nmc_cgen* g, long long* n) {
  if (!g || !n) return NMC_EINVAL;
  *n = g->P;
  return NMC_OK;
}

nmc_status nmc_cgen_get_params(const nmc_cgen* g, float* theta) {
  if (!g || !theta) return NMC_EINVAL;
  if (cudaMemcpyAsync(theta, g->th, (size_t)g->P * sizeof(float), cudaMemcpyDeviceToHost, g->st) !=
          cudaSuccess ||
      cudaStreamSynchronize(g->st) != cudaSuccess) {
    cudaGetLastError();
    return NMC_ECUDA;
  }
  return NMC_OK;
}

nmc_status nmc_cgen_set_params(nmc_cgen* g, const float* theta) {
  if (!g || !theta) return NMC_EINVAL;
  const size_t b = (size_t)g->P * sizeof(float);
  if (cudaMemcpyAsync(g->th, theta, b, cudaMemcpyHostToDevice, g->st) != cudaSuccess ||
      cudaMemsetAsync(g->m, 0, b, g->st) != cudaSuccess ||
      cudaMemsetAsync(g->v, 0, b, g->st) != cudaSuccess) {
    cudaGetLastError();
    return NMC_ECUDA;
  }
  k_cg_to_bf16<<<grid_for(g->P, 256), 256, 0, g->st>>>(g->th, g->P, g->thb);
  g->steps = 0;
  if (cudaStreamSynchronize(g->st) != cudaSuccess) {
    cudaGetLastError();
    return NMC_ECUDA;
  }
  return cg_last();
}

nmc_status nmc_cgen_forward(nmc_cgen* g, const float* d_z, int n, float* d_logits) {
  if (!g || !d_z || !d_logits || n < 1 || n > g->max_batch) return NMC_EINVAL;
  const long long total = (long long)n * g->d.S();
  k_cg_to_bf16<<<grid_for(total, 256), 256, 0, g->st>>>(d_z, total, g->act[0]);
  forward(g, n);
  if (cudaMemcpyAsync(d_logits, g->logits, (size_t)total * sizeof(float),
                      cudaMemcpyDeviceToDevice, g->st) != cudaSuccess) {
    cudaGetLastError();
    return NMC_ECUDA;
  }
  return cg_last();
}

nmc_status nmc_cgen_loss_grad(nmc_cgen* g, const float* d_z, const int8_t* d_fields, int n,
                              double* loss, float* d_grad) {
  if (!g || !d_z || !d_fields || !loss || !d_grad || n < 1 || n > g->max_batch) return NMC_EINVAL;
  const long long total = (long long)n * g->d.S();
  k_cg_to_bf16<<<grid_for(total, 256), 256, 0, g->st>>>(d_z, total, g->act[0]);
  forward(g, n);
  backward(g, d_fields, n);
  double sum = 0.0;
  if (cudaMemcpyAsync(d_grad, g->gr, (size_t)g->P * sizeof(float), cudaMemcpyDeviceToDevice,
                      g->st) != cudaSuccess ||
      cudaMemcpyAsync(&sum, g->dloss, sizeof(double), cudaMemcpyDeviceToHost, g->st) != cudaSuccess ||
      cudaStreamSynchronize(g->st) != cudaSuccess) {
    cudaGetLastError();
    return NMC_ECUDA;
  }
  *loss = sum / (double)total;
  return cg_last();
}

nmc_status nmc_cgen_train_step(nmc_cgen* g, const int8_t* d_fields, int n, long long sample0,
                               float lr, double* loss) {
  if (!g || !d_fields || n < 1 || n > g->max_batch || sample0 < 0) return NMC_EINVAL;
  noise(g, sample0, n, 0u);
  forward(g, n);
  backward(g, d_fields, n);
  ++g->steps;
  const float c1 = 1.f - std::pow(0.9f, (float)g->steps);
  const float c2 = 1.f - std::pow(0.999f, (float)g->steps);
  k_cg_adam<<<grid_for(g->P, 256), 256, 0, g->st>>>(g->th, g->gr, g->m, g->v, g->P, lr, c1, c2,
                                                    g->thb);
  if (loss) {
    double sum = 0.0;
    if (cudaMemcpyAsync(&sum, g->dloss, sizeof(double), cudaMemcpyDeviceToHost, g->st) !=
            cudaSuccess ||
        cudaStreamSynchronize(g->st) != cudaSuccess) {
      cudaGetLastError();
      return NMC_ECUDA;
    }
    *loss = sum / ((double)n * g->d.S());
  }
  return cg_last();
}

nmc_status nmc_cgen_sample(nmc_cgen* g, long long n0, int n, int8_t* d_fields, float* d_logits) {
  if (!g || !d_fields || n < 1 || n > g->max_batch || n0 < 0) return NMC_EINVAL;
  const int S = g->d.S();
  noise(g, n0, n, 1u);
  forward(g, n);
  k_cg_draw<<<grid_for((long long)n * S, 256), 256, 0, g->st>>>(
      g->logits, n0, n, S, 1u, (uint32_t)g->seed, (uint32_t)(g->seed >> 32), d_fields);
  if (d_logits &&
      cudaMemcpyAsync(d_logits, g->logits, (size_t)n * S * sizeof(float), cudaMemcpyDeviceToDevice,
                      g->st) != cudaSuccess) {
    cudaGetLastError();
    return NMC_ECUDA;
  }
  if (cudaStreamSynchronize(g->st) != cudaSuccess) {
    cudaGetLastError();
    return NMC_ECUDA;
  }
  return cg_last();
}

void nmc_cgen_destroy(nmc_cgen* g) {
  if (!g) return;
  if (g->st) cudaStreamSynchronize(g->st);
  else cudaDeviceSynchronize();
  for (void* p : g->allocs) cudaFree(p);
  cudaGetLastError();
  delete g;
}

}  // extern "C"
