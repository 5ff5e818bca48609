// Network initialization (Algorithm 1, steps 2-3; SM Sec. II): the generator's transposed
// 3D convolutions (FP32), the Eq. 4 observable loss through the determinant weight with its
// exact gradient (FP64, batched over configurations x spins), Adam, Bernoulli sampling, and
// the C ABI of include/nmc_gen.h.
//
// Loss path for a chunk of configurations (every step one batched launch over 2 x chunk
// matrices, b = 2*config + spin):
//   x = 2p - 1, v = e^{sigma lam x}, vinv = 1/v
//   left stacks L_j = B_{L-1}...B_{jw} (held transposed, U D T), j = nb-1..0
//   anchor j: X = Db_R^{-1} U_R^T U_L Db_L^{-1} + Ds_R T_R T_L^T Ds_L, Xi = X^{-1}
//             G(jw,0) = U_L Db_L^{-1} Xi Ds_R T_R,  H(0,jw) = T_L^T Ds_L Xi Db_R^{-1} U_R^T
//             (j = 0: G_0 = U_L Db_L^{-1} Xi Db_R^{-1} U_R^T with R = I)
//   G~_0 = e^{dtau K/2} G_0 e^{-dtau K/2}; E_k, S per configuration (the sweep's estimator)
//   Gbar = e^{dtau K/2} (dLoss/dG~_0) e^{-dtau K/2}
//   for l: grad x(i,l) = -lam sum_sigma sigma sum_a H(0,l)_ai [Gbar G(l,0)^T]_ai;
//          inside a block G(l+1,0) = B_l G(l,0), H(0,l+1) = H(0,l) B_l^{-1}; the right stack
//          R_j = B_{jw-1}...B_0 is extended block by block for the next anchor.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nmc_gen.h"
#include "nmc_internal.cuh"

namespace nmc_host {
void hopping(int lattice, int Lx, int Ly, double t, std::vector<double>& K);
void jacobi_eigh(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V);
void expk_from_eig(int n, const std::vector<double>& w, const std::vector<double>& V, double c,
                   std::vector<double>& out);
}  // namespace nmc_host

using namespace nmc;

namespace {

constexpr uint32_t kTagGenZ = 2, kTagBernoulli = 3, kTagParam = 4, kTagShuffle = 5;
constexpr int kThreads = 256;
constexpr double kAdamB1 = 0.9, kAdamB2 = 0.999, kAdamEps = 1e-7;

int blocks_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 32));
}

// ---------------------------------------------------------------------------- generator
struct Shape3 {
  int d0, d1, d2;
  __host__ __device__ int size() const { return d0 * d1 * d2; }
};

// out[n][co][o] = act(bias[co] + sum_ci sum_{q + k = o} in[n][ci][q] W[ci][co][k])
__global__ void k_convt_fwd(const float* __restrict__ in, int Cin, Shape3 is,
                            const float* __restrict__ W, const float* __restrict__ bias,
                            int Cout, Shape3 ks, float* __restrict__ out, int n, int sigmoid) {
  const Shape3 os{is.d0 + ks.d0 - 1, is.d1 + ks.d1 - 1, is.d2 + ks.d2 - 1};
  const int osz = os.size(), isz = is.size(), ksz = ks.size();
  const int total = n * Cout * osz;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int nb = e / (Cout * osz);
    const int r = e - nb * Cout * osz;
    const int co = r / osz;
    const int o = r - co * osz;
    const int o0 = o / (os.d1 * os.d2), o1 = (o / os.d2) % os.d1, o2 = o % os.d2;
    const int a0 = max(0, o0 - is.d0 + 1), a1 = max(0, o1 - is.d1 + 1), a2 = max(0, o2 - is.d2 + 1);
    const int b0 = min(ks.d0 - 1, o0), b1 = min(ks.d1 - 1, o1), b2 = min(ks.d2 - 1, o2);
    float acc = bias[co];
    for (int ci = 0; ci < Cin; ++ci) {
      const float* x = in + ((long long)nb * Cin + ci) * isz;
      const float* w = W + ((long long)ci * Cout + co) * ksz;
      for (int k0 = a0; k0 <= b0; ++k0)
        for (int k1 = a1; k1 <= b1; ++k1) {
          const float* xr = x + ((o0 - k0) * is.d1 + (o1 - k1)) * is.d2 + o2;
          const float* wr = w + (k0 * ks.d1 + k1) * ks.d2;
          for (int k2 = a2; k2 <= b2; ++k2) acc = fmaf(xr[-k2], wr[k2], acc);
        }
    }
    out[e] = sigmoid ? 1.0f / (1.0f + expf(-acc)) : acc;
  }
}

// gin[n][ci][q] = sum_co sum_k gout[n][co][q + k] W[ci][co][k]  (every q + k is inside out)
__global__ void k_convt_bwd_in(const float* __restrict__ gout, int Cout, Shape3 is,
                               const float* __restrict__ W, int Cin, Shape3 ks,
                               float* __restrict__ gin, int n) {
  const Shape3 os{is.d0 + ks.d0 - 1, is.d1 + ks.d1 - 1, is.d2 + ks.d2 - 1};
  const int osz = os.size(), isz = is.size(), ksz = ks.size();
  const int total = n * Cin * isz;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int nb = e / (Cin * isz);
    const int r = e - nb * Cin * isz;
    const int ci = r / isz;
    const int q = r - ci * isz;
    const int q0 = q / (is.d1 * is.d2), q1 = (q / is.d2) % is.d1, q2 = q % is.d2;
    float acc = 0.f;
    for (int co = 0; co < Cout; ++co) {
      const float* g = gout + ((long long)nb * Cout + co) * osz;
      const float* w = W + ((long long)ci * Cout + co) * ksz;
      for (int k0 = 0; k0 < ks.d0; ++k0)
        for (int k1 = 0; k1 < ks.d1; ++k1) {
          const float* gr = g + ((q0 + k0) * os.d1 + (q1 + k1)) * os.d2 + q2;
          const float* wr = w + (k0 * ks.d1 + k1) * ks.d2;
          for (int k2 = 0; k2 < ks.d2; ++k2) acc = fmaf(gr[k2], wr[k2], acc);
        }
    }
    gin[e] = acc;
  }
}

// gW[ci][co][k] (+)= sum_n sum_q in[n][ci][q] gout[n][co][q + k]; one warp per weight.
// gb[co] (+)= sum_n sum_o gout[n][co][o]; warps beyond the weights take the biases.
__global__ void k_convt_bwd_w(const float* __restrict__ in, int Cin, Shape3 is,
                              const float* __restrict__ gout, int Cout, Shape3 ks, int n,
                              float* __restrict__ gW, float* __restrict__ gb, int accumulate) {
  const Shape3 os{is.d0 + ks.d0 - 1, is.d1 + ks.d1 - 1, is.d2 + ks.d2 - 1};
  const int osz = os.size(), isz = is.size(), ksz = ks.size();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nW = Cin * Cout * ksz;
  if (warp >= nW + Cout) return;
  float acc = 0.f;
  if (warp < nW) {
    const int ci = warp / (Cout * ksz);
    const int r = warp - ci * Cout * ksz;
    const int co = r / ksz;
    const int k = r - co * ksz;
    const int k0 = k / (ks.d1 * ks.d2), k1 = (k / ks.d2) % ks.d1, k2 = k % ks.d2;
    for (int e = lane; e < n * isz; e += 32) {
      const int nb = e / isz, q = e - nb * isz;
      const int q0 = q / (is.d1 * is.d2), q1 = (q / is.d2) % is.d1, q2 = q % is.d2;
      const int o = ((q0 + k0) * os.d1 + (q1 + k1)) * os.d2 + (q2 + k2);
      acc = fmaf(in[((long long)nb * Cin + ci) * isz + q], gout[((long long)nb * Cout + co) * osz + o], acc);
    }
  } else {
    const int co = warp - nW;
    for (int e = lane; e < n * osz; e += 32) {
      const int nb = e / osz, o = e - nb * osz;
      acc += gout[((long long)nb * Cout + co) * osz + o];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    float* dst = warp < nW ? gW + warp : gb + (warp - nW);
    *dst = accumulate ? *dst + acc : acc;
  }
}

// g <- g * y (1 - y): back through a sigmoid whose output is y
__global__ void k_sigmoid_bwd(float* __restrict__ g, const float* __restrict__ y, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    g[e] *= y[e] * (1.f - y[e]);
}

__global__ void k_gen_input(const long long* __restrict__ ids, long long n0, int n, int zsize,
                            uint32_t stream, uint32_t k0, uint32_t k1, float* __restrict__ z) {
  const int total = n * zsize;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int b = e / zsize, el = e - b * zsize;
    const long long id = ids ? ids[b] : n0 + b;
    uint32_t c[4] = {(uint32_t)el, (uint32_t)id, stream, kTagGenZ};
    philox4x32_10(c, k0, k1);
    z[e] = (c[0] >> 31) ? -1.f : 1.f;
  }
}

// scale[0] = min(1, max_norm / |g|) (1 when max_norm <= 0); one CTA
__global__ void k_clip_scale(const float* __restrict__ g, int n, float max_norm,
                             float* __restrict__ scale) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) s += (double)g[e] * g[e];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    const double nrm = sqrt(t);
    scale[0] = (max_norm > 0.f && nrm > max_norm) ? (float)(max_norm / nrm) : 1.f;
  }
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float c1, float c2,
                       const float* __restrict__ scale) {
  const float sc = scale[0];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float gi = g[e] * sc;
    const float mi = (float)kAdamB1 * m[e] + (1.f - (float)kAdamB1) * gi;
    const float vi = (float)kAdamB2 * v[e] + (1.f - (float)kAdamB2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    th[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + (float)kAdamEps);
  }
}

// ---------------------------------------------------------------------------- fields
// p [n][Lt][A][B] -> x [n][Lt][N], site i = a + A b
__global__ void k_p_to_x(const float* __restrict__ p, int n, int Lt, int A, int B,
                         double* __restrict__ x) {
  const int N = A * B, total = n * Lt * N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e % N, rest = e / N;
    const int a = i % A, b = i / A;
    x[e] = 2.0 * (double)p[(long long)rest * N + a * B + b] - 1.0;
  }
}

// v[2c + s][l][i] = e^{sigma lam x[c][l][i]}, vinv = 1 / v
__global__ void k_x_to_v(const double* __restrict__ x, int n, int LN, double lam,
                         double* __restrict__ v, double* __restrict__ vinv) {
  const int total = n * LN;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int c = e / LN, r = e - c * LN;
    const double a = exp(lam * x[e]), b = exp(-lam * x[e]);
    v[(long long)(2 * c) * LN + r] = a;
    v[(long long)(2 * c + 1) * LN + r] = b;
    vinv[(long long)(2 * c) * LN + r] = b;
    vinv[(long long)(2 * c + 1) * LN + r] = a;
  }
}

// gradient wrt the layer-2 pre-activation: ga[n][l][a][b] = 2 gx[n][l][a + A b] y (1 - y)
__global__ void k_grad_x_to_a2(const double* __restrict__ gx, const float* __restrict__ p, int n,
                               int Lt, int A, int B, float* __restrict__ ga) {
  const int N = A * B, total = n * Lt * N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int bb = e % B, a = (e / B) % A, rest = e / N;
    const float y = p[e];
    ga[e] = (float)(2.0 * gx[(long long)rest * N + a + A * bb]) * y * (1.f - y);
  }
}

__global__ void k_bernoulli(const float* __restrict__ p, long long n0, int n, int Lt, int A, int B,
                            uint32_t stream, uint32_t k0, uint32_t k1, int8_t* __restrict__ s) {
  const int N = A * B, LN = Lt * N, total = n * LN;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int c = e / LN, r = e - c * LN;
    const int l = r / N, i = r - l * N;
    const int a = i % A, b = i / A;
    uint32_t ctr[4] = {(uint32_t)r, (uint32_t)(n0 + c), stream, kTagBernoulli};
    philox4x32_10(ctr, k0, k1);
    const double u = (double)ctr[0] * 0x1p-32;
    s[e] = u < (double)p[(long long)c * LN + (l * A + a) * B + b] ? 1 : -1;
  }
}

// ---------------------------------------------------------------------------- loss pieces
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  if (threadIdx.x == 0) red[0] = s;
  __syncthreads();
  return red[0];
}

// Per configuration (one CTA): observables from the measurement accumulators, Eq. 4 loss,
// and dLoss/dG~ per spin:
//   dS/dG~s_ab  = (1/4N) [p_a p_b (delta_ab - 2 G~s_ba) + 2 delta_ab (sum_i p_i m_i) p_a sgn_s],
//                 m_i = G~dn_ii - G~up_ii, sgn = -1 (up), +1 (dn)
//   dEk/dG~s_ab = -K_ba / N
__global__ void k_loss_gbar(const double* __restrict__ Gt, const double* __restrict__ acc,
                            const double* __restrict__ targets, double w1, double w2,
                            const double* __restrict__ K, int N, int Lx, int lattice,
                            double* __restrict__ Gbt, double* __restrict__ loss,
                            double* __restrict__ obs, int* __restrict__ bad) {
  __shared__ double red[kThreads / 32];
  const int c = blockIdx.x;
  const long long NN = (long long)N * N;
  const double* Gu = Gt + (long long)(2 * c) * NN;
  const double* Gd = Gu + NN;
  const double ek = acc[c * 8 + 1], s = acc[c * 8 + 3];
  double stag = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double pi = site_parity(i, Lx, lattice) ? -1.0 : 1.0;
    stag += pi * (Gd[(long long)i * N + i] - Gu[(long long)i * N + i]);
  }
  stag = block_sum(stag, red);
  if (threadIdx.x == 0) {
    // health check: at half filling on a bipartite lattice the density is 1 for any real
    // field (G_dn = I - P G_up^T P), so a departure flags a failed stabilization
    // (the estimators of a single field configuration are not bounded by the physical
    // ranges, so only the density and finiteness are checked)
    const double dens = acc[c * 8 + 4];
    if (!(fabs(dens - 1.0) <= 1e-6) || !isfinite(s) || !isfinite(ek)) atomicMax(bad, c + 1);
    if (obs) { obs[2 * c] = s; obs[2 * c + 1] = ek; }
    if (loss) {
      const double dS = s - targets[2 * c], dE = ek - targets[2 * c + 1];
      loss[c] = w1 * dS * dS + w2 * dE * dE;
    }
  }
  if (!Gbt) return;
  const double cS = 2.0 * w1 * (s - targets[2 * c]);
  const double cE = 2.0 * w2 * (ek - targets[2 * c + 1]);
  for (int e = threadIdx.x; e < 2 * (int)NN; e += blockDim.x) {
    const int sp = e / (int)NN, r = e - sp * (int)NN;
    const int a = r / N, b = r - a * N;
    const double* G = sp ? Gd : Gu;
    const double pa = site_parity(a, Lx, lattice) ? -1.0 : 1.0;
    const double pb = site_parity(b, Lx, lattice) ? -1.0 : 1.0;
    double d = pa * pb * ((a == b ? 1.0 : 0.0) - 2.0 * G[(long long)b * N + a]);
    if (a == b) d += 2.0 * stag * pa * (sp ? 1.0 : -1.0);
    Gbt[(long long)(2 * c + sp) * NN + r] = cS * d / (4.0 * N) - cE * K[(long long)b * N + a] / N;
  }
}

// grad[c][l][i] = -lam sum_sigma sigma sum_a H_sigma[a][i] Q_sigma[a][i]   (one CTA per config)
__global__ void k_grad_slice(const double* __restrict__ H, const double* __restrict__ Q, int N,
                             double lam, double* __restrict__ grad, long long gstride) {
  const int c = blockIdx.x;
  const long long NN = (long long)N * N;
  const double* Hu = H + (long long)(2 * c) * NN;
  const double* Qu = Q + (long long)(2 * c) * NN;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double su = 0.0, sd = 0.0;
    for (int a = 0; a < N; ++a) {
      su = fma(Hu[(long long)a * N + i], Qu[(long long)a * N + i], su);
      sd = fma(Hu[NN + (long long)a * N + i], Qu[NN + (long long)a * N + i], sd);
    }
    grad[(long long)c * gstride + i] = -lam * (su - sd);
  }
}

__global__ void k_fill(double* p, long long n, double v) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    p[e] = v;
}

struct UDT {
  double* U;
  double* D;
  double* T;
  long long sU, sD, sT;
};

}  // namespace

// ---------------------------------------------------------------------------- context
struct nmc_gen {
  int lattice = 0, Lx = 0, Ly = 0, N = 0, Lt = 0, w = 0, nb = 0, A = 0, B = 0;
  double t = 0, U = 0, beta = 0, dtau = 0, lam = 0;
  uint64_t seed = 0;
  nmc_gen_arch arch{};
  Shape3 zs{}, hs{}, os{}, k1s{}, k2s{};
  int nW1 = 0, nB1 = 0, nW2 = 0, nB2 = 0, nP = 0;
  int Bc = 0;      // configurations per loss chunk
  int Bf = 0;      // configurations per generator chunk
  int device = 0;
  cudaStream_t stream = nullptr;
  long long steps = 0;
  long long epochs = 0;   // epochs trained since creation / set_params (shuffle counter)
  double clip = 0.0;      // global gradient-norm bound (0: none)
  float* dScale = nullptr;
  std::string err;
  std::vector<void*> allocs;
  // parameters [W1 | b1 | W2 | b2], gradients, Adam moments (float32)
  float *dP = nullptr, *dGP = nullptr, *dM = nullptr, *dV = nullptr;
  // generator activations (Bf configurations)
  float *dZ = nullptr, *dH1 = nullptr, *dPo = nullptr, *dGa2 = nullptr, *dGh1 = nullptr;
  long long* dIds = nullptr;
  // FP64 loss path (Bc configurations, 2 Bc matrices)
  double *dEm = nullptr, *dEp = nullptr, *dEph = nullptr, *dEmh = nullptr, *dK = nullptr;
  double *dI = nullptr, *dOnes = nullptr;
  double *dX = nullptr, *dVv = nullptr, *dVi = nullptr;
  double *dLU = nullptr, *dLD = nullptr, *dLT = nullptr;  // left stacks, slots 0..nb-1
  double *dRU = nullptr, *dRD = nullptr, *dRT = nullptr;  // right stack (current)
  double *dRU2 = nullptr, *dRD2 = nullptr, *dRT2 = nullptr;
  double *dW1 = nullptr, *dW2 = nullptr, *dTp = nullptr, *dWS = nullptr;
  double *dM1 = nullptr, *dXs = nullptr, *dXi = nullptr, *dT1 = nullptr, *dT2 = nullptr;
  double *dGl = nullptr, *dGl2 = nullptr, *dH = nullptr, *dH2 = nullptr;
  double *dG0 = nullptr, *dGt = nullptr, *dGbt = nullptr, *dGbar = nullptr, *dQ = nullptr;
  double *dAcc = nullptr, *dSign = nullptr, *dTarg = nullptr, *dLoss = nullptr, *dGx = nullptr;
  int* dBad = nullptr;

  long long NN() const { return (long long)N * N; }
  float* W1() const { return dP; }
  float* b1() const { return dP + nW1; }
  float* W2() const { return dP + nW1 + nB1; }
  float* b2() const { return dP + nW1 + nB1 + nW2; }
};

namespace {

nmc_status gfail(nmc_gen* g, nmc_status s, const std::string& m) {
  if (g) g->err = m;
  return s;
}

#define GEN_CUDA(g, call)                                                              \
  do {                                                                                 \
    const cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                           \
      const nmc_status s_ = e_ == cudaErrorMemoryAllocation ? NMC_ENOMEM : NMC_ECUDA; \
      cudaGetLastError();                                                              \
      return gfail(g, s_, std::string(#call) + ": " + cudaGetErrorString(e_));         \
    }                                                                                  \
  } while (0)

#define GEN_TRY(expr)                       \
  do {                                      \
    const nmc_status s_ = (expr);           \
    if (s_ != NMC_OK) return s_;            \
  } while (0)

template <typename T>
nmc_status galloc(nmc_gen* g, T*& p, long long n) {
  GEN_CUDA(g, cudaMalloc((void**)&p, (size_t)std::max<long long>(n, 1) * sizeof(T)));
  g->allocs.push_back(p);
  return NMC_OK;
}

ScaleDesc vscale(const double* v, long long stride, int kind) {
  ScaleDesc d;
  d.kind = kind;
  d.vec = v;
  d.vstride = stride;
  return d;
}

GemmArgs<double> gbase(const nmc_gen* g, int batch, const double* A, long long sA,
                       const double* B, long long sB, double* C) {
  GemmArgs<double> a;
  a.M = a.N = a.K = g->N;
  a.batch = batch;
  a.A = A; a.sA = sA; a.lda = g->N;
  a.B = B; a.sB = sB; a.ldb = g->N;
  a.C = C; a.sC = g->NN(); a.ldc = g->N;
  return a;
}

// UDT-QRP of X into dst; dst.T = Tp * src.T
void qrp_into(nmc_gen* g, int nb2, const double* X, const UDT& dst, const UDT& src) {
  qrp_udt(X, dst.U, dst.D, g->dTp, g->dWS, g->N, nb2, g->stream);
  gemm(gbase(g, nb2, g->dTp, g->NN(), src.T, src.sT, dst.T), g->stream);
}

UDT identity_udt(const nmc_gen* g) { return UDT{g->dI, g->dOnes, g->dI, 0, 0, 0}; }
UDT left_slot(const nmc_gen* g, int j) {
  const long long per = (long long)2 * g->Bc;
  return UDT{g->dLU + j * per * g->NN(), g->dLD + j * per * g->N, g->dLT + j * per * g->NN(),
             g->NN(), g->N, g->NN()};
}

// L_j^T = B_{jw}^T ... B_{(j+1)w-1}^T L_{j+1}^T, B_l^T = e^{V_l} e^{-dtau K}
void left_update(nmc_gen* g, int nb2, int j, const UDT& src, const UDT& dst) {
  const long long LN = (long long)g->Lt * g->N;
  double* X = g->dW1;
  double* X2 = g->dW2;
  const int lt = (j + 1) * g->w - 1;
  auto a = gbase(g, nb2, g->dEm, 0, src.U, src.sU, X);
  a.bcol = vscale(src.D, src.sD, SC_VEC);
  a.crow = vscale(g->dVv + (long long)lt * g->N, LN, SC_VEC);
  gemm(a, g->stream);
  for (int l = lt - 1; l >= j * g->w; --l) {
    auto h = gbase(g, nb2, g->dEm, 0, X, g->NN(), X2);
    h.crow = vscale(g->dVv + (long long)l * g->N, LN, SC_VEC);
    gemm(h, g->stream);
    std::swap(X, X2);
  }
  qrp_into(g, nb2, X, dst, src);
}

// R_{j+1} = B_{(j+1)w-1} ... B_{jw} R_j
void right_update(nmc_gen* g, int nb2, int j, const UDT& src, const UDT& dst) {
  const long long LN = (long long)g->Lt * g->N;
  double* X = g->dW1;
  double* X2 = g->dW2;
  const int l0 = j * g->w;
  auto a = gbase(g, nb2, g->dEm, 0, src.U, src.sU, X);
  a.brow = vscale(g->dVv + (long long)l0 * g->N, LN, SC_VEC);
  a.bcol = vscale(src.D, src.sD, SC_VEC);
  gemm(a, g->stream);
  for (int l = l0 + 1; l < l0 + g->w; ++l) {
    auto h = gbase(g, nb2, g->dEm, 0, X, g->NN(), X2);
    h.brow = vscale(g->dVv + (long long)l * g->N, LN, SC_VEC);
    gemm(h, g->stream);
    std::swap(X, X2);
  }
  qrp_into(g, nb2, X, dst, src);
}

// From R (= B_{l-1}...B_0) and L (= B_{L-1}...B_l, transposed): G(l,0) -> dGl,
// H(0,l) = (I - G_0) R^{-1} -> dH; if g0: G_0 -> dG0 (valid when R = I).
void anchor(nmc_gen* g, int nb2, const UDT& R, const UDT& L, bool g0) {
  cudaStream_t st = g->stream;
  const long long NN = g->NN();
  auto a1 = gbase(g, nb2, R.U, R.sU, L.U, L.sU, g->dM1);
  a1.transA = 1;
  a1.crow = vscale(R.D, R.sD, SC_INV_MAX1);
  a1.ccol = vscale(L.D, L.sD, SC_INV_MAX1);
  gemm(a1, st);
  auto a2 = gbase(g, nb2, R.T, R.sT, L.T, L.sT, g->dXs);
  a2.transB = 1;
  a2.crow = vscale(R.D, R.sD, SC_MIN1);
  a2.ccol = vscale(L.D, L.sD, SC_MIN1);
  a2.Cin = g->dM1; a2.sCin = NN; a2.ldcin = g->N; a2.beta = 1.0;
  gemm(a2, st);
  solve_stab(g->dXs, g->dI, 0, g->dOnes, 0, g->dXi, g->dWS, g->N, nb2, st);  // X^{-1}
  auto t1 = gbase(g, nb2, g->dXi, NN, R.T, R.sT, g->dT1);                     // Xi Ds_R T_R
  t1.brow = vscale(R.D, R.sD, SC_MIN1);
  gemm(t1, st);
  auto gl = gbase(g, nb2, L.U, L.sU, g->dT1, NN, g->dGl);                     // U_L Db_L^{-1} .
  gl.brow = vscale(L.D, L.sD, SC_INV_MAX1);
  gemm(gl, st);
  auto t2 = gbase(g, nb2, g->dXi, NN, R.U, R.sU, g->dT2);                     // Xi Db_R^{-1} U_R^T
  t2.transB = 1;
  t2.brow = vscale(R.D, R.sD, SC_INV_MAX1);
  gemm(t2, st);
  auto h = gbase(g, nb2, L.T, L.sT, g->dT2, NN, g->dH);                        // T_L^T Ds_L .
  h.transA = 1;
  h.brow = vscale(L.D, L.sD, SC_MIN1);
  gemm(h, st);
  if (g0) {
    auto gg = gbase(g, nb2, L.U, L.sU, g->dT2, NN, g->dG0);                   // U_L Db_L^{-1} .
    gg.brow = vscale(L.D, L.sD, SC_INV_MAX1);
    gemm(gg, st);
  }
}

// Loss path for n <= Bc configurations with fields in g->dX. Writes obs (S, E_k) [n][2],
// loss [n] and grad [n][Lt][N] where requested (device pointers, may be null).
nmc_status loss_chunk(nmc_gen* g, int n, const double* targets, double w1, double w2,
                      double* obs, double* loss, double* grad) {
  cudaStream_t st = g->stream;
  const int nb2 = 2 * n;
  const long long NN = g->NN(), LN = (long long)g->Lt * g->N;
  k_x_to_v<<<blocks_for(n * LN), kThreads, 0, st>>>(g->dX, n, (int)LN, g->lam, g->dVv, g->dVi);
  // left stacks L_j, j = nb-1 .. 0
  for (int j = g->nb - 1; j >= 0; --j)
    left_update(g, nb2, j, j + 1 == g->nb ? identity_udt(g) : left_slot(g, j + 1), left_slot(g, j));
  anchor(g, nb2, identity_udt(g), left_slot(g, 0), true);
  // G~_0 and the estimators
  gemm(gbase(g, nb2, g->dEph, 0, g->dG0, NN, g->dT1), st);
  gemm(gbase(g, nb2, g->dT1, NN, g->dEmh, 0, g->dGt), st);
  k_fill<<<blocks_for(8LL * n), kThreads, 0, st>>>(g->dAcc, 8LL * n, 0.0);
  GEN_CUDA(g, cudaMemsetAsync(g->dBad, 0, sizeof(int), st));
  measure(g->dGt, g->dK, g->dSign, g->N, g->Lx, g->lattice, g->U, g->dAcc, n, 2, st);
  const bool want_grad = grad != nullptr;
  k_loss_gbar<<<n, kThreads, 0, st>>>(g->dGt, g->dAcc, targets, w1, w2, g->dK, g->N, g->Lx,
                                      g->lattice, want_grad ? g->dGbt : nullptr,
                                      targets ? loss : nullptr, obs, g->dBad);
  GEN_CUDA(g, cudaGetLastError());
  {
    int bad = 0;
    GEN_CUDA(g, cudaMemcpyAsync(&bad, g->dBad, sizeof(int), cudaMemcpyDeviceToHost, st));
    GEN_CUDA(g, cudaStreamSynchronize(st));
    if (bad) {
      double a[8];
      GEN_CUDA(g, cudaMemcpy(a, g->dAcc + 8LL * (bad - 1), sizeof a, cudaMemcpyDeviceToHost));
      char buf[200];
      std::snprintf(buf, sizeof buf, "configuration %d of the chunk: density %.3e, S %.3e, E_k %.3e "
                    "(stabilization failed)", bad - 1, a[4], a[3], a[1]);
      return gfail(g, NMC_ENUMERIC, buf);
    }
  }
  if (!want_grad) return NMC_OK;
  gemm(gbase(g, nb2, g->dEph, 0, g->dGbt, NN, g->dT1), st);
  gemm(gbase(g, nb2, g->dT1, NN, g->dEmh, 0, g->dGbar), st);
  UDT R = identity_udt(g);
  UDT Rbuf[2] = {UDT{g->dRU, g->dRD, g->dRT, NN, g->N, NN}, UDT{g->dRU2, g->dRD2, g->dRT2, NN, g->N, NN}};
  for (int j = 0; j < g->nb; ++j) {
    if (j > 0) {
      right_update(g, nb2, j - 1, R, Rbuf[j & 1]);
      R = Rbuf[j & 1];
      anchor(g, nb2, R, left_slot(g, j), false);
    }
    double* Gl = g->dGl;
    double* Gl2 = g->dGl2;
    double* H = g->dH;
    double* H2 = g->dH2;
    for (int k = 0; k < g->w; ++k) {
      const int l = j * g->w + k;
      auto q = gbase(g, nb2, g->dGbar, NN, Gl, NN, g->dQ);
      q.transB = 1;
      gemm(q, st);
      k_grad_slice<<<n, kThreads, 0, st>>>(H, g->dQ, g->N, g->lam, grad + (long long)l * g->N, LN);
      if (k + 1 < g->w) {
        auto pg = gbase(g, nb2, g->dEm, 0, Gl, NN, Gl2);
        pg.brow = vscale(g->dVv + (long long)l * g->N, LN, SC_VEC);
        gemm(pg, st);
        auto ph = gbase(g, nb2, H, NN, g->dEp, 0, H2);
        ph.brow = vscale(g->dVi + (long long)l * g->N, LN, SC_VEC);
        gemm(ph, st);
        std::swap(Gl, Gl2);
        std::swap(H, H2);
      }
    }
  }
  GEN_CUDA(g, cudaGetLastError());
  return NMC_OK;
}

// generator forward for n <= Bf inputs (ids or n0 + b of `stream`) into dH1, dPo
void forward(nmc_gen* g, const long long* d_ids, long long n0, int n, uint32_t stream) {
  cudaStream_t st = g->stream;
  const uint32_t k0 = (uint32_t)g->seed, k1 = (uint32_t)(g->seed >> 32);
  k_gen_input<<<blocks_for((long long)n * g->zs.size()), kThreads, 0, st>>>(
      d_ids, n0, n, g->zs.size(), stream, k0, k1, g->dZ);
  k_convt_fwd<<<blocks_for((long long)n * g->arch.c1 * g->hs.size()), kThreads, 0, st>>>(
      g->dZ, 1, g->zs, g->W1(), g->b1(), g->arch.c1, g->k1s, g->dH1, n, 1);
  k_convt_fwd<<<blocks_for((long long)n * g->os.size()), kThreads, 0, st>>>(
      g->dH1, g->arch.c1, g->hs, g->W2(), g->b2(), 1, g->k2s, g->dPo, n, 1);
}

}  // namespace

// ---------------------------------------------------------------------------- C ABI
extern "C" {

void nmc_gen_paper_arch(nmc_gen_arch* a) {
  if (!a) return;
  *a = nmc_gen_arch{{10, 2, 2}, 20, {16, 6, 3}, {36, 6, 3}};
}

nmc_status nmc_gen_create(int lattice, int Lx, int Ly, double t, double U, double beta,
                          double dtau, int n_wrap, const nmc_gen_arch* arch, uint64_t seed,
                          int max_batch, void* cuda_stream, nmc_gen** out) {
  if (!out) return NMC_EINVAL;
  *out = nullptr;
  if (!arch || max_batch < 1 || max_batch > 4096) return NMC_EINVAL;
  // lattice checks as nmc_create
  const int N = Lx * Ly * (lattice == NMC_HONEYCOMB ? 2 : 1);
  if (lattice != NMC_SQUARE && lattice != NMC_HONEYCOMB) return NMC_EINVAL;
  if (Lx < 1 || Ly < 1 || N < 2 || N > 1024) return NMC_EINVAL;
  if (lattice == NMC_SQUARE && ((Lx > 1 && Lx % 2) || (Ly > 1 && Ly % 2))) return NMC_EINVAL;
  if (!(t > 0) || !(U >= 0) || !(beta > 0) || !(dtau > 0) || n_wrap < 1) return NMC_EINVAL;
  const double ratio = beta / dtau, Ltd = std::round(ratio);
  if (Ltd < 1 || std::fabs(ratio - Ltd) > 1e-9 * ratio || Ltd > 1e6) return NMC_EINVAL;
  const int Lt = (int)Ltd;
  if (Lt % n_wrap) return NMC_EINVAL;
  const nmc_gen_arch& a = *arch;
  for (int d = 0; d < 3; ++d)
    if (a.z[d] < 1 || a.k1[d] < 1 || a.k2[d] < 1) return NMC_EINVAL;
  if (a.c1 < 1 || a.c1 > 1024) return NMC_EINVAL;
  const int A = lattice == NMC_HONEYCOMB ? 2 * Lx : Lx, B = Ly;
  const Shape3 zs{a.z[0], a.z[1], a.z[2]};
  const Shape3 hs{zs.d0 + a.k1[0] - 1, zs.d1 + a.k1[1] - 1, zs.d2 + a.k1[2] - 1};
  const Shape3 os{hs.d0 + a.k2[0] - 1, hs.d1 + a.k2[1] - 1, hs.d2 + a.k2[2] - 1};
  if (os.d0 != Lt || os.d1 != A || os.d2 != B) return NMC_EINVAL;

  nmc_gen* g = new (std::nothrow) nmc_gen();
  if (!g) return NMC_ENOMEM;
  g->lattice = lattice; g->Lx = Lx; g->Ly = Ly; g->N = N; g->Lt = Lt; g->w = n_wrap;
  g->nb = Lt / n_wrap; g->A = A; g->B = B;
  g->t = t; g->U = U; g->beta = beta; g->dtau = dtau; g->seed = seed;
  g->lam = std::acosh(std::exp(dtau * U / 2.0));
  g->arch = a;
  g->zs = zs; g->hs = hs; g->os = os;
  g->k1s = Shape3{a.k1[0], a.k1[1], a.k1[2]};
  g->k2s = Shape3{a.k2[0], a.k2[1], a.k2[2]};
  g->nW1 = a.c1 * g->k1s.size(); g->nB1 = a.c1; g->nW2 = a.c1 * g->k2s.size(); g->nB2 = 1;
  g->nP = g->nW1 + g->nB1 + g->nW2 + g->nB2;
  g->Bc = max_batch;
  g->Bf = std::max(max_batch, 256);
  g->stream = (cudaStream_t)cuda_stream;
  auto bail = [&](nmc_status s) {
    nmc_gen_destroy(g);
    return s;
  };
  if (cudaGetDevice(&g->device) != cudaSuccess) { cudaGetLastError(); return bail(NMC_ECUDA); }

  // host set-up: K and the four exponentials
  std::vector<double> K, Kc, wv, V, Em, Ep, Emh, Eph;
  nmc_host::hopping(lattice, Lx, Ly, t, K);
  Kc = K;
  nmc_host::jacobi_eigh(N, Kc, wv, V);
  nmc_host::expk_from_eig(N, wv, V, -dtau, Em);
  nmc_host::expk_from_eig(N, wv, V, +dtau, Ep);
  nmc_host::expk_from_eig(N, wv, V, -dtau / 2, Emh);
  nmc_host::expk_from_eig(N, wv, V, +dtau / 2, Eph);

  const long long NN = (long long)N * N, LN = (long long)Lt * N, M2 = 2LL * g->Bc;
  nmc_status s = NMC_OK;
  auto A_ = [&](auto*& p, long long n) { if (s == NMC_OK) s = galloc(g, p, n); };
  A_(g->dP, g->nP); A_(g->dGP, g->nP); A_(g->dM, g->nP); A_(g->dV, g->nP);
  A_(g->dZ, (long long)g->Bf * zs.size());
  A_(g->dH1, (long long)g->Bf * a.c1 * hs.size());
  A_(g->dGh1, (long long)g->Bf * a.c1 * hs.size());
  A_(g->dPo, (long long)g->Bf * os.size());
  A_(g->dGa2, (long long)g->Bf * os.size());
  A_(g->dIds, g->Bf);
  for (double** p : {&g->dEm, &g->dEp, &g->dEph, &g->dEmh, &g->dK, &g->dI}) A_(*p, NN);
  A_(g->dOnes, N);
  A_(g->dX, g->Bc * LN); A_(g->dVv, M2 * LN); A_(g->dVi, M2 * LN);
  A_(g->dLU, g->nb * M2 * NN); A_(g->dLD, g->nb * M2 * N); A_(g->dLT, g->nb * M2 * NN);
  A_(g->dRU, M2 * NN); A_(g->dRD, M2 * N); A_(g->dRT, M2 * NN);
  A_(g->dRU2, M2 * NN); A_(g->dRD2, M2 * N); A_(g->dRT2, M2 * NN);
  for (double** p : {&g->dW1, &g->dW2, &g->dTp, &g->dM1, &g->dXs, &g->dXi, &g->dT1, &g->dT2,
                     &g->dGl, &g->dGl2, &g->dH, &g->dH2, &g->dG0, &g->dGt, &g->dGbt, &g->dGbar,
                     &g->dQ})
    A_(*p, M2 * NN);
  A_(g->dWS, 2 * M2 * NN);
  A_(g->dAcc, 8LL * g->Bc); A_(g->dSign, g->Bc); A_(g->dTarg, 2LL * g->Bf);
  A_(g->dLoss, g->Bf); A_(g->dGx, (long long)g->Bc * LN);
  A_(g->dBad, 1);
  A_(g->dScale, 1);
  if (s != NMC_OK) return bail(s);

  std::vector<double> I(NN, 0.0), ones(std::max<long long>(N, g->Bc), 1.0);
  for (int i = 0; i < N; ++i) I[(size_t)i * N + i] = 1.0;
  auto up = [&](double* d, const std::vector<double>& h, size_t n) {
    return cudaMemcpy(d, h.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  };
  if (up(g->dEm, Em, NN) || up(g->dEp, Ep, NN) || up(g->dEph, Eph, NN) || up(g->dEmh, Emh, NN) ||
      up(g->dK, K, NN) || up(g->dI, I, NN) || up(g->dOnes, ones, N) || up(g->dSign, ones, g->Bc)) {
    cudaGetLastError();
    return bail(NMC_ECUDA);
  }
  // Glorot-uniform weights (word 0 of Philox at (index, layer, 0, 4)), zero biases
  std::vector<float> P(g->nP, 0.f);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int rf1 = g->k1s.size(), rf2 = g->k2s.size();
  const double lim1 = std::sqrt(6.0 / (1.0 * rf1 + a.c1 * rf1));
  const double lim2 = std::sqrt(6.0 / (1.0 * a.c1 * rf2 + rf2));
  for (int layer = 0; layer < 2; ++layer) {
    const int n = layer ? g->nW2 : g->nW1;
    const double lim = layer ? lim2 : lim1;
    float* dst = P.data() + (layer ? g->nW1 + g->nB1 : 0);
    for (int e = 0; e < n; ++e) {
      uint32_t c[4] = {(uint32_t)e, (uint32_t)layer, 0u, kTagParam};
      philox4x32_10(c, k0, k1);
      dst[e] = (float)((2.0 * ((double)c[0] * 0x1p-32) - 1.0) * lim);
    }
  }
  if (cudaMemcpy(g->dP, P.data(), P.size() * sizeof(float), cudaMemcpyHostToDevice) ||
      cudaMemset(g->dM, 0, P.size() * sizeof(float)) || cudaMemset(g->dV, 0, P.size() * sizeof(float))) {
    cudaGetLastError();
    return bail(NMC_ECUDA);
  }
  *out = g;
  return NMC_OK;
}

nmc_status nmc_gen_get_params(const nmc_gen* g, float* W1, float* b1, float* W2, float* b2) {
  if (!g) return NMC_EINVAL;
  nmc_gen* m = const_cast<nmc_gen*>(g);
  GEN_CUDA(m, cudaStreamSynchronize(g->stream));
  const float* src[4] = {g->W1(), g->b1(), g->W2(), g->b2()};
  const int n[4] = {g->nW1, g->nB1, g->nW2, g->nB2};
  float* dst[4] = {W1, b1, W2, b2};
  for (int k = 0; k < 4; ++k)
    if (dst[k]) GEN_CUDA(m, cudaMemcpy(dst[k], src[k], n[k] * sizeof(float), cudaMemcpyDeviceToHost));
  return NMC_OK;
}

nmc_status nmc_gen_set_params(nmc_gen* g, const float* W1, const float* b1, const float* W2,
                              const float* b2) {
  if (!g || !W1 || !b1 || !W2 || !b2) return NMC_EINVAL;
  GEN_CUDA(g, cudaStreamSynchronize(g->stream));
  float* dst[4] = {g->W1(), g->b1(), g->W2(), g->b2()};
  const float* src[4] = {W1, b1, W2, b2};
  const int n[4] = {g->nW1, g->nB1, g->nW2, g->nB2};
  for (int k = 0; k < 4; ++k)
    GEN_CUDA(g, cudaMemcpy(dst[k], src[k], n[k] * sizeof(float), cudaMemcpyHostToDevice));
  GEN_CUDA(g, cudaMemset(g->dM, 0, g->nP * sizeof(float)));
  GEN_CUDA(g, cudaMemset(g->dV, 0, g->nP * sizeof(float)));
  g->steps = 0;
  g->epochs = 0;
  return NMC_OK;
}

nmc_status nmc_gen_probs(nmc_gen* g, long long n0, int n, int stream, float* d_p) {
  if (!g || n < 0 || (n > 0 && !d_p) || n0 < 0 || stream < 0) return NMC_EINVAL;
  const long long osz = g->os.size();
  for (int c0 = 0; c0 < n; c0 += g->Bf) {
    const int m = std::min(g->Bf, n - c0);
    forward(g, nullptr, n0 + c0, m, (uint32_t)stream);
    GEN_CUDA(g, cudaMemcpyAsync(d_p + (long long)c0 * osz, g->dPo, m * osz * sizeof(float),
                                cudaMemcpyDeviceToDevice, g->stream));
  }
  GEN_CUDA(g, cudaGetLastError());
  GEN_CUDA(g, cudaStreamSynchronize(g->stream));
  return NMC_OK;
}

nmc_status nmc_gen_sample_fields(nmc_gen* g, long long n0, int n, int stream, int8_t* d_fields) {
  if (!g || n < 0 || (n > 0 && !d_fields) || n0 < 0 || stream < 0) return NMC_EINVAL;
  const long long LN = (long long)g->Lt * g->N;
  const uint32_t k0 = (uint32_t)g->seed, k1 = (uint32_t)(g->seed >> 32);
  for (int c0 = 0; c0 < n; c0 += g->Bf) {
    const int m = std::min(g->Bf, n - c0);
    forward(g, nullptr, n0 + c0, m, (uint32_t)stream);
    k_bernoulli<<<blocks_for(m * LN), kThreads, 0, g->stream>>>(
        g->dPo, n0 + c0, m, g->Lt, g->A, g->B, (uint32_t)stream, k0, k1, d_fields + c0 * LN);
  }
  GEN_CUDA(g, cudaGetLastError());
  GEN_CUDA(g, cudaStreamSynchronize(g->stream));
  return NMC_OK;
}

nmc_status nmc_gen_observables(nmc_gen* g, const double* d_x, int n, double* d_obs) {
  if (!g || n < 0 || (n > 0 && (!d_x || !d_obs))) return NMC_EINVAL;
  const long long LN = (long long)g->Lt * g->N;
  for (int c0 = 0; c0 < n; c0 += g->Bc) {
    const int m = std::min(g->Bc, n - c0);
    GEN_CUDA(g, cudaMemcpyAsync(g->dX, d_x + c0 * LN, m * LN * sizeof(double),
                                cudaMemcpyDeviceToDevice, g->stream));
    GEN_TRY(loss_chunk(g, m, nullptr, 0, 0, d_obs + 2LL * c0, nullptr, nullptr));
  }
  GEN_CUDA(g, cudaStreamSynchronize(g->stream));
  return NMC_OK;
}

nmc_status nmc_gen_generated_observables(nmc_gen* g, long long n0, int n, int stream,
                                         double* d_obs) {
  if (!g || n < 0 || (n > 0 && !d_obs) || n0 < 0 || stream < 0) return NMC_EINVAL;
  const long long LN = (long long)g->Lt * g->N;
  for (int c0 = 0; c0 < n; c0 += g->Bc) {
    const int m = std::min(g->Bc, n - c0);
    forward(g, nullptr, n0 + c0, m, (uint32_t)stream);
    k_p_to_x<<<blocks_for(m * LN), kThreads, 0, g->stream>>>(g->dPo, m, g->Lt, g->A, g->B, g->dX);
    GEN_TRY(loss_chunk(g, m, nullptr, 0, 0, d_obs + 2LL * c0, nullptr, nullptr));
  }
  GEN_CUDA(g, cudaStreamSynchronize(g->stream));
  return NMC_OK;
}

nmc_status nmc_gen_loss_grad(nmc_gen* g, const double* d_x, int n, const double* d_targets,
                             double w1, double w2, double* d_loss, double* d_grad) {
  if (!g || n < 0 || (n > 0 && (!d_x || !d_targets))) return NMC_EINVAL;
  const long long LN = (long long)g->Lt * g->N;
  for (int c0 = 0; c0 < n; c0 += g->Bc) {
    const int m = std::min(g->Bc, n - c0);
    GEN_CUDA(g, cudaMemcpyAsync(g->dX, d_x + c0 * LN, m * LN * sizeof(double),
                                cudaMemcpyDeviceToDevice, g->stream));
    GEN_TRY(loss_chunk(g, m, d_targets + 2LL * c0, w1, w2, nullptr,
                       d_loss ? d_loss + c0 : g->dLoss, d_grad ? d_grad + c0 * LN : nullptr));
  }
  GEN_CUDA(g, cudaStreamSynchronize(g->stream));
  return NMC_OK;
}

nmc_status nmc_gen_train_step(nmc_gen* g, const long long* ids, int n, const double* targets,
                              double w1, double w2, double lr, double* loss_out) {
  if (!g || n < 1 || !ids || !targets || !(lr >= 0)) return NMC_EINVAL;
  for (int k = 0; k < n; ++k)
    if (ids[k] < 0) return NMC_EINVAL;
  cudaStream_t st = g->stream;
  const long long LN = (long long)g->Lt * g->N, osz = g->os.size();
  const int c1 = g->arch.c1;
  double total = 0.0;
  std::vector<double> lossh;
  for (int c0 = 0; c0 < n; c0 += g->Bc) {
    const int m = std::min(g->Bc, n - c0);
    GEN_CUDA(g, cudaMemcpyAsync(g->dIds, ids + c0, m * sizeof(long long), cudaMemcpyHostToDevice, st));
    GEN_CUDA(g, cudaMemcpyAsync(g->dTarg, targets + 2LL * c0, 2LL * m * sizeof(double),
                                cudaMemcpyHostToDevice, st));
    forward(g, g->dIds, 0, m, 0u);
    k_p_to_x<<<blocks_for(m * LN), kThreads, 0, st>>>(g->dPo, m, g->Lt, g->A, g->B, g->dX);
    {
      const nmc_status s = loss_chunk(g, m, g->dTarg, w1, w2, nullptr, g->dLoss, g->dGx);
      if (s != NMC_OK) {
        g->err += "; batch sample ids:";
        for (int k = 0; k < m; ++k) g->err += " " + std::to_string(ids[c0 + k]);
        return s;
      }
    }
    k_grad_x_to_a2<<<blocks_for(m * osz), kThreads, 0, st>>>(g->dGx, g->dPo, m, g->Lt, g->A, g->B,
                                                              g->dGa2);
    const int acc = c0 > 0;
    const int warps2 = g->nW2 + g->nB2, warps1 = g->nW1 + g->nB1;
    k_convt_bwd_w<<<(warps2 * 32 + kThreads - 1) / kThreads, kThreads, 0, st>>>(
        g->dH1, c1, g->hs, g->dGa2, 1, g->k2s, m, g->dGP + g->nW1 + g->nB1,
        g->dGP + g->nW1 + g->nB1 + g->nW2, acc);
    k_convt_bwd_in<<<blocks_for((long long)m * c1 * g->hs.size()), kThreads, 0, st>>>(
        g->dGa2, 1, g->hs, g->W2(), c1, g->k2s, g->dGh1, m);
    k_sigmoid_bwd<<<blocks_for((long long)m * c1 * g->hs.size()), kThreads, 0, st>>>(
        g->dGh1, g->dH1, m * c1 * g->hs.size());
    k_convt_bwd_w<<<(warps1 * 32 + kThreads - 1) / kThreads, kThreads, 0, st>>>(
        g->dZ, 1, g->zs, g->dGh1, c1, g->k1s, m, g->dGP, g->dGP + g->nW1, acc);
    lossh.resize(m);
    GEN_CUDA(g, cudaMemcpyAsync(lossh.data(), g->dLoss, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    GEN_CUDA(g, cudaStreamSynchronize(st));
    for (double v : lossh) total += v;
  }
  g->steps += 1;
  const double c1b = 1.0 - std::pow(kAdamB1, (double)g->steps);
  const double c2b = 1.0 - std::pow(kAdamB2, (double)g->steps);
  k_clip_scale<<<1, kThreads, 0, st>>>(g->dGP, g->nP, (float)g->clip, g->dScale);
  k_adam<<<blocks_for(g->nP), kThreads, 0, st>>>(g->dP, g->dGP, g->dM, g->dV, g->nP, (float)lr,
                                                 (float)c1b, (float)c2b, g->dScale);
  GEN_CUDA(g, cudaGetLastError());
  GEN_CUDA(g, cudaStreamSynchronize(st));
  if (loss_out) *loss_out = total;
  if (!std::isfinite(total)) return gfail(g, NMC_ENUMERIC, "training loss is not finite");
  return NMC_OK;
}

nmc_status nmc_gen_train(nmc_gen* g, const double* targets, int n, int epochs, int batch,
                         double lr, double w1, double w2, double* epoch_loss) {
  if (!g || !targets || n < 1 || epochs < 0 || batch < 1 || !(lr >= 0)) return NMC_EINVAL;
  if (w1 <= 0 || w2 <= 0) {  // inverse variances of the targets
    double m[2] = {0, 0}, v[2] = {0, 0};
    for (int k = 0; k < n; ++k)
      for (int d = 0; d < 2; ++d) m[d] += targets[2 * k + d] / n;
    for (int k = 0; k < n; ++k)
      for (int d = 0; d < 2; ++d) v[d] += (targets[2 * k + d] - m[d]) * (targets[2 * k + d] - m[d]) / n;
    if (w1 <= 0) w1 = v[0] > 0 ? 1.0 / v[0] : 1.0;
    if (w2 <= 0) w2 = v[1] > 0 ? 1.0 / v[1] : 1.0;
  }
  const uint32_t k0 = (uint32_t)g->seed, k1 = (uint32_t)(g->seed >> 32);
  std::vector<long long> order(n), ids;
  std::vector<double> tb;
  for (int e = 0; e < epochs; ++e) {
    for (int k = 0; k < n; ++k) order[k] = k;
    const uint32_t ep = (uint32_t)g->epochs;
    for (int k = n - 1; k > 0; --k) {  // Fisher-Yates, uniforms at (k, epoch, 0, 5)
      uint32_t c[4] = {(uint32_t)k, ep, 0u, kTagShuffle};
      philox4x32_10(c, k0, k1);
      const int r = (int)(((uint64_t)c[0] * (uint64_t)(k + 1)) >> 32);
      std::swap(order[k], order[r]);
    }
    double sum = 0.0;
    for (int s = 0; s < n; s += batch) {
      const int m = std::min(batch, n - s);
      ids.assign(order.begin() + s, order.begin() + s + m);
      tb.resize(2 * m);
      for (int k = 0; k < m; ++k) {
        tb[2 * k] = targets[2 * ids[k]];
        tb[2 * k + 1] = targets[2 * ids[k] + 1];
      }
      double L = 0;
      GEN_TRY(nmc_gen_train_step(g, ids.data(), m, tb.data(), w1, w2, lr, &L));
      sum += L;
    }
    if (epoch_loss) epoch_loss[e] = sum / n;
    ++g->epochs;
  }
  return NMC_OK;
}

long long nmc_gen_steps(const nmc_gen* g) { return g ? g->steps : -1; }

nmc_status nmc_gen_set_clip(nmc_gen* g, double max_norm) {
  if (!g || !(max_norm >= 0)) return NMC_EINVAL;
  g->clip = max_norm;
  return NMC_OK;
}

const char* nmc_gen_last_error(const nmc_gen* g) { return g ? g->err.c_str() : "null generator"; }

void nmc_gen_destroy(nmc_gen* g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (void* p : g->allocs) cudaFree(p);
  cudaGetLastError();
  delete g;
}

}  // extern "C"

// Used by nmc_generate (mode 1): fill d_fields [n][L_tau][N] from the generator's stream 1
// for samples n0..n0+n-1, then make `st` wait for it.
nmc_status nmc_gen_fill_fields(nmc_gen* g, int N, int Lt, long long n0, int n, int8_t* d_fields,
                               cudaStream_t st) {
  if (!g) return NMC_EINVAL;
  if (g->N != N || g->Lt != Lt) return gfail(g, NMC_EINVAL, "generator lattice differs from the context");
  (void)st;  // nmc_gen_sample_fields synchronises the generator's stream before returning
  return nmc_gen_sample_fields(g, n0, n, 1, d_fields);
}
