// Small device kernels: Philox field initialisation, conversions, and the equal-time
// estimators; the dynamic shared-memory limit helper.
#include <mutex>
#include <set>
#include <utility>

#include "nmc_internal.cuh"

namespace nmc {

namespace {

NMC_DEBUG_FLAG

__global__ void k_init_fields(int8_t* s, int n_chains, int L, int N, uint32_t k0, uint32_t k1,
                              long long chain_offset) {
  const long long total = (long long)n_chains * L * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / ((long long)L * N);
    const uint32_t li = (uint32_t)(e - c * L * N);  // l*N + i
    uint32_t ctr[4] = {li, 0u, (uint32_t)(chain_offset + c), kTagInit};
    philox4x32_10(ctr, k0, k1);
    s[e] = (ctr[0] >> 31) ? (int8_t)-1 : (int8_t)1;
  }
}

__global__ void k_init_fields_list(int8_t* s, int L, int N, uint32_t k0, uint32_t k1,
                                   const int* list, const long long* ids, int n) {
  const long long per = (long long)L * N, total = per * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long j = e / per;
    const uint32_t li = (uint32_t)(e - j * per);  // l*N + i
    uint32_t ctr[4] = {li, 0u, (uint32_t)ids[j], kTagInit};
    philox4x32_10(ctr, k0, k1);
    s[(long long)list[j] * per + li] = (ctr[0] >> 31) ? (int8_t)-1 : (int8_t)1;
  }
}

__global__ void k_restart_chain_state(const int* list, const long long* ids, int n, int n_chains,
                                      long long sweep, long long* chain_id,
                                      long long* sweep_base, double* sign,
                                      unsigned long long* counts, unsigned long long* drift) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int c = list[j];
  if (!NMC_DCHECK(c >= 0 && c < n_chains, 501)) return;
  chain_id[c] = ids[j];
  sweep_base[c] = sweep;
  sign[c] = 1.0;
  counts[3 * c] = counts[3 * c + 1] = counts[3 * c + 2] = 0ull;
  drift[c] = 0ull;
}

__global__ void k_default_chain_ids(long long* chain_id, long long* sweep_base, int n,
                                    long long offset) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  chain_id[c] = offset + c;
  sweep_base[c] = 0;
}

__global__ void k_identity(double* U, double* D, double* T, int N, int batch) {
  const long long NN = (long long)N * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < NN * batch;
       e += (long long)gridDim.x * blockDim.x) {
    const long long rc = e % NN;
    const double v = (rc / N == rc % N) ? 1.0 : 0.0;
    if (U) U[e] = v;
    if (T) T[e] = v;
    if (D && rc < N) D[(e / NN) * N + rc] = 1.0;
  }
}

__global__ void k_to_float(const double* x, float* y, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = (float)x[e];
}

__global__ void k_to_double(const float* x, double* y, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = (double)x[e];
}

__global__ void k_normalize(int8_t* s, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    s[e] = (s[e] == 1) ? (int8_t)1 : (int8_t)-1;
}

__global__ void k_philox(const uint32_t* c0, int n, uint32_t c1, uint32_t c2, uint32_t c3,
                         uint32_t k0, uint32_t k1, uint32_t* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  uint32_t ctr[4] = {c0[j], c1, c2, c3};
  philox4x32_10(ctr, k0, k1);
  for (int w = 0; w < 4; ++w) out[4 * j + w] = ctr[w];
}

constexpr int kMeasThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kMeasThreads / 32; ++w) s += red[w];
  return s;  // valid in thread 0
}

// Equal-time estimators on G~ (one CTA per chain), Eq. 3 energy and the S(Q) of Eq. 4:
//  ekin  = -(1/N) sum_sigma sum_ij K_ij G~_ji
//  epot  = (U/N) sum_i (1/2 - G~up_ii)(1/2 - G~dn_ii)
//  docc  = (1/N) sum_i (1 - G~up_ii)(1 - G~dn_ii)
//  dens  = (1/N) sum_i (2 - G~up_ii - G~dn_ii)
//  S     = (1/4N) [ (sum_i p_i m_i)^2 + sum_sigma sum_ij p_i p_j (delta_ij - G~_ji) G~_ij ],
//          m_i = G~dn_ii - G~up_ii, p_i = +-1 the sublattice sign (site_parity)
// With ns = 1 only G~up is stored and G~dn_ij = delta_ij - p_i p_j G~up_ji.
__global__ void __launch_bounds__(kMeasThreads)
k_measure(const double* __restrict__ Gt, const double* __restrict__ K,
          const double* __restrict__ sign, int N, int Lx, int lattice, double U, int ns,
          double* __restrict__ acc, const long long* __restrict__ series_idx) {
  if (series_idx) acc += *series_idx * (long long)gridDim.x * 8;
  __shared__ double red[kMeasThreads / 32];
  const int c = blockIdx.x;
  const long long NN = (long long)N * N;
  const double* Gu = Gt + (long long)c * ns * NN;
  const double* Gd = Gu + NN;  // only read when ns == 2
  double kin = 0.0, conn = 0.0;
  for (int e = threadIdx.x; e < (int)NN; e += blockDim.x) {
    const int i = e / N, j = e - i * N;
    const int ji = j * N + i;
    const double pij = ((site_parity(i, Lx, lattice) ^ site_parity(j, Lx, lattice)) & 1) ? -1.0 : 1.0;
    const double dij = (i == j) ? 1.0 : 0.0;
    const double gu_ij = Gu[e], gu_ji = Gu[ji];
    const double gd_ij = ns == 2 ? Gd[e] : dij - pij * gu_ji;
    const double gd_ji = ns == 2 ? Gd[ji] : dij - pij * gu_ij;
    kin += K[e] * (gu_ji + gd_ji);
    conn += pij * ((dij - gu_ji) * gu_ij + (dij - gd_ji) * gd_ij);
  }
  double epot = 0.0, docc = 0.0, dens = 0.0, stag = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double gu = Gu[(long long)i * N + i];
    const double gd = ns == 2 ? Gd[(long long)i * N + i] : 1.0 - gu;
    epot += (0.5 - gu) * (0.5 - gd);
    docc += (1.0 - gu) * (1.0 - gd);
    dens += 2.0 - gu - gd;
    const double p = site_parity(i, Lx, lattice) ? -1.0 : 1.0;
    stag += p * (gd - gu);
  }
  kin = block_sum(kin, red);
  conn = block_sum(conn, red);
  epot = block_sum(epot, red);
  docc = block_sum(docc, red);
  dens = block_sum(dens, red);
  stag = block_sum(stag, red);
  if (threadIdx.x == 0) {
    const double sg = sign[c];
    const double ekin = -kin / N;
    const double e = ekin + U * epot / N;
    const double s = 0.25 * (stag * stag + conn) / N;
    double* a = acc + (long long)c * 8;
    a[0] += e * sg;
    a[1] += ekin * sg;
    a[2] += docc / N * sg;
    a[3] += s * sg;
    a[4] += dens / N * sg;
    a[5] += sg;
  }
}

// cumulative[c] = max(cumulative[c], stab[c]); hist = max_c stab[c] (one CTA)
__global__ void k_fold_drift(const unsigned long long* stab, unsigned long long* cumulative,
                             unsigned long long* hist, long long cap, long long* idx, int n) {
  __shared__ unsigned long long red[256];
  unsigned long long m = 0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const unsigned long long v = stab[c];
    if (v > cumulative[c]) cumulative[c] = v;
    if (v > m) m = v;
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o && red[threadIdx.x + o] > red[threadIdx.x])
      red[threadIdx.x] = red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long k = *idx;
    if (hist && k < cap) hist[k] = red[0];
    *idx = k + 1;
  }
}

__global__ void k_advance(long long* ctr, int meas) {
  ctr[0] += 1;
  ctr[1] += meas;
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// The dynamic shared-memory limit is a per-function, per-device attribute and is not
// stream-ordered: lowering it for one launch can break a larger launch of the same kernel
// still queued on another stream. So each kernel's limit is raised once per device to the
// device's opt-in maximum and never lowered.
void prefer_max_shared_carveout(const void* func) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({func, dev})) return;
  if (cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess)
    done.insert({func, dev});
  else
    cudaGetLastError();
}

int sm_count() {
  static std::mutex mu;
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 1;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 1;
    }
    cached[dev] = n;
  }
  return cached[dev];
}

void allow_max_dynamic_smem(const void* func) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({func, dev})) return;
  int optin = 0;
  cudaFuncAttributes fa;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, func) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  // the dynamic limit excludes the kernel's static shared memory
  const int limit = optin - (int)fa.sharedSizeBytes;
  if (limit > 0 &&
      cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) == cudaSuccess)
    done.insert({func, dev});
  else
    cudaGetLastError();
}

void init_fields_list(int8_t* s, int L, int N, uint32_t k0, uint32_t k1, const int* list,
                      const long long* ids, int n, cudaStream_t st) {
  if (n <= 0) return;
  k_init_fields_list<<<grid_for((long long)n * L * N), 256, 0, st>>>(s, L, N, k0, k1, list,
                                                                     ids, n);
}

void restart_chain_state(const int* list, const long long* ids, int n, int n_chains, long long sweep,
                         long long* chain_id, long long* sweep_base, double* sign,
                         unsigned long long* counts, unsigned long long* drift,
                         cudaStream_t st) {
  if (n <= 0) return;
  k_restart_chain_state<<<(n + 127) / 128, 128, 0, st>>>(list, ids, n, n_chains, sweep, chain_id,
                                                         sweep_base, sign, counts, drift);
}

void default_chain_ids(long long* chain_id, long long* sweep_base, int n_chains,
                       long long offset, cudaStream_t st) {
  k_default_chain_ids<<<(n_chains + 127) / 128, 128, 0, st>>>(chain_id, sweep_base, n_chains,
                                                             offset);
}

void init_fields(int8_t* s, int n_chains, int L, int N, uint32_t k0, uint32_t k1,
                 long long chain_offset, cudaStream_t st) {
  const long long n = (long long)n_chains * L * N;
  k_init_fields<<<grid_for(n), 256, 0, st>>>(s, n_chains, L, N, k0, k1, chain_offset);
}

void set_identity_batch(double* U, double* D, double* T, int N, int batch, cudaStream_t st) {
  k_identity<<<grid_for((long long)N * N * batch), 256, 0, st>>>(U, D, T, N, batch);
}

void copy_to_float(const double* x, float* y, long long n, cudaStream_t st) {
  k_to_float<<<grid_for(n), 256, 0, st>>>(x, y, n);
}

void copy_to_double(const float* x, double* y, long long n, cudaStream_t st) {
  k_to_double<<<grid_for(n), 256, 0, st>>>(x, y, n);
}

void fields_normalize(int8_t* s, long long n, cudaStream_t st) {
  k_normalize<<<grid_for(n), 256, 0, st>>>(s, n);
}

void philox_batch(const uint32_t* c0, int n, uint32_t c1, uint32_t c2, uint32_t c3,
                  uint32_t k0, uint32_t k1, uint32_t* out, cudaStream_t st) {
  if (n <= 0) return;
  k_philox<<<(n + 255) / 256, 256, 0, st>>>(c0, n, c1, c2, c3, k0, k1, out);
}

void fold_drift(const unsigned long long* stab, unsigned long long* cumulative,
                unsigned long long* hist, long long hist_cap, long long* hist_idx, int n_chains,
                cudaStream_t st) {
  k_fold_drift<<<1, 256, 0, st>>>(stab, cumulative, hist, hist_cap, hist_idx, n_chains);
}

void advance_counters(long long* ctr, int meas, cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(ctr, meas);
}

void measure(const double* Gt, const double* K, const double* sign, int N, int Lx, int lattice,
             double U, double* acc, int n_chains, int ns, cudaStream_t st,
             const long long* series_idx) {
  k_measure<<<n_chains, kMeasThreads, 0, st>>>(Gt, K, sign, N, Lx, lattice, U, ns, acc,
                                               series_idx);
}

NMC_DEBUG_READER(debug_fail_misc)

}  // namespace nmc
