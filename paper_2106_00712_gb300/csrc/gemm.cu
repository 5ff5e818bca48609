// Batched dense GEMM with diagonal scalings (FP64 and FP32, SIMT FMA pipes).
//
// Every matrix product of the DQMC sweep goes through here: the wraps
// G <- e^{-dtau K} e^{V} G e^{-V} e^{dtau K} (and the reverse direction), the UDV stack
// products B_l X = e^{-dtau K} e^{V_l} X, the stabilized recompute of
// G = (I + R L)^{-1}, and the symmetric-Trotter transform of G before measurement.
// The diagonal factors e^{+-V_l} (values e^{+-lam}, selected by the field s(i,l)) and the
// D-splits of the UDV recompute are applied while tiles are staged (B operand) or in
// the epilogue, so no scaled copy of any matrix is ever written.
//
// Tiling: BM x BN output tile per CTA, BK-deep k-steps staged in shared memory,
// TM x TN outputs per thread (strided by BM/TM, BN/TN so a warp reads consecutive
// shared-memory words). Batch over blockIdx.z (batch = 2 * chains).
#include "nmc_internal.cuh"

namespace nmc {

namespace {

NMC_DEBUG_FLAG

__device__ __forceinline__ double nan_max(double a, double b) {
  // max that propagates NaN (fmax would drop it)
  return (b > a || b != b) ? b : a;
}

// The diagonal scalings of one CTA's tile, evaluated once per CTA (a scale can cost an FP64
// division): B's row scale for every k < kMaxK, B's column and C's row and column scales for
// the tile's columns and rows (indices clamped into the matrix; the clamped entries are
// never used).
constexpr int kMaxK = 1024;
template <int BM, int BN>
struct TileScales {
  double brow[kMaxK];
  double bcol[BN];
  double crow[BM];
  double ccol[BN];
};

template <typename T, int BM, int BN>
__device__ void load_scales(TileScales<BM, BN>& sc, const GemmArgs<T>& g, int b, int m0, int n0) {
  for (int k = threadIdx.x; k < g.K && k < kMaxK; k += blockDim.x) sc.brow[k] = scale_at(g.brow, b, k);
  for (int j = threadIdx.x; j < BN; j += blockDim.x) {
    const int gn = min(n0 + j, g.N - 1);
    sc.bcol[j] = scale_at(g.bcol, b, gn);
    sc.ccol[j] = scale_at(g.ccol, b, gn);
  }
  for (int i = threadIdx.x; i < BM; i += blockDim.x) sc.crow[i] = scale_at(g.crow, b, min(m0 + i, g.M - 1));
}

// B's row scale at k (from the table below kMaxK)
template <typename T, int BM, int BN>
__device__ __forceinline__ double brow_at(const TileScales<BM, BN>& sc, const GemmArgs<T>& g, int b,
                                          int k) {
  return k < kMaxK ? sc.brow[k] : scale_at(g.brow, b, k);
}

// Epilogue of one output C[b][gm][gn] from its accumulated value v (FP64): the C scalings
// (rs, cs: the row's and the column's), + beta Cin, the drift against ref, and the FP32 /
// FP32-pair copies.
template <typename T>
__device__ __forceinline__ void store_c(const GemmArgs<T>& g, int b, int gm, int gn, double rs,
                                        double cs, double v, double& dmax) {
  if (!NMC_DCHECK(gm >= 0 && gm < g.M && gn >= 0 && gn < g.N, 401)) return;
  if (g.crow.kind != SC_NONE || g.ccol.kind != SC_NONE) v = v * rs * cs;
  if (g.Cin) v += g.beta * (double)g.Cin[(long long)b * g.sCin + (long long)gm * g.ldcin + gn];
  const T out = (T)v;
  const long long idx = (long long)gm * g.ldc + gn;
  if (g.ref) {
    const long long ri = (long long)b * g.sRef + idx;
    double r;
    if (g.ref_is_float == 2) r = df_to_double(((const df2*)g.ref)[ri]);
    else if (g.ref_is_float == 1) r = (double)((const float*)g.ref)[ri];
    else r = ((const double*)g.ref)[ri];
    dmax = nan_max(dmax, fabs((double)out - r));
  }
  g.C[(long long)b * g.sC + idx] = out;
  if (g.Cf) g.Cf[(long long)b * g.sCf + idx] = (float)out;
  if (g.Cdf) g.Cdf[(long long)b * g.sCdf + idx] = df_from_double((double)out);
}

// The warp's largest drift into the chain's slot (bits of a non-negative double)
template <typename T>
__device__ __forceinline__ void fold_drift_max(const GemmArgs<T>& g, int b, double dmax) {
  if (!g.drift) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = nan_max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if ((threadIdx.x & 31) == 0 && dmax != 0.0)
    atomicMax(g.drift + (g.ns == 2 ? b >> 1 : b), (unsigned long long)__double_as_longlong(dmax));
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm(const GemmArgs<T> g) {
  constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  __shared__ TileScales<BM, BN> sc;
  const int b = blockIdx.z;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const T* __restrict__ A = g.A + (long long)b * g.sA;
  const T* __restrict__ B = g.B + (long long)b * g.sB;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  const bool bscale = g.brow.kind != SC_NONE || g.bcol.kind != SC_NONE;
  load_scales(sc, g, b, m0, n0);
  __syncthreads();

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += NT) {
      int mm, kk;
      if (g.transA) { kk = e / BM; mm = e % BM; } else { mm = e / BK; kk = e % BK; }
      const int gm = m0 + mm, gk = k0 + kk;
      T v = T(0);
      if (gm < g.M && gk < g.K)
        v = g.transA ? A[(long long)gk * g.lda + gm] : A[(long long)gm * g.lda + gk];
      As[kk][mm] = v;
    }
    for (int e = tid; e < BK * BN; e += NT) {
      int kk, nn;
      if (g.transB) { nn = e / BK; kk = e % BK; } else { kk = e / BN; nn = e % BN; }
      const int gk = k0 + kk, gn = n0 + nn;
      T v = T(0);
      if (gk < g.K && gn < g.N) {
        v = g.transB ? B[(long long)gn * g.ldb + gk] : B[(long long)gk * g.ldb + gn];
        if (bscale) v = (T)((double)v * brow_at(sc, g, b, gk) * sc.bcol[nn]);
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * NTY];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + j * NTX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }

  double dmax = 0.0;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + i * NTY;
    if (gm >= g.M) continue;
    const double rs = sc.crow[ty + i * NTY];
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + j * NTX;
      if (gn < g.N) store_c(g, b, gm, gn, rs, sc.ccol[tx + j * NTX], (double)acc[i][j], dmax);
    }
  }
  fold_drift_max(g, b, dmax);
}

// FP64 operands and results with the products accumulated in FP32 pairs on the FP32 pipe:
// tiles are staged as FP32 pairs (the B scalings applied in FP64 first), each thread's
// outputs accumulate with error-free products and sums (df_fma_acc), and the epilogue is
// the FP64 one above. Operands must lie within the FP32 range (|x| < 3.4e38); entries
// below ~1e-38 lose relative precision (they keep their absolute error ~1e-45).
template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm_pair(const GemmArgs<double> g) {
  constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
  __shared__ df2 As[BK][BM + 1];
  __shared__ df2 Bs[BK][BN + 1];
  __shared__ TileScales<BM, BN> sc;
  const int b = blockIdx.z;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const double* __restrict__ A = g.A + (long long)b * g.sA;
  const double* __restrict__ B = g.B + (long long)b * g.sB;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  const bool bscale = g.brow.kind != SC_NONE || g.bcol.kind != SC_NONE;
  load_scales(sc, g, b, m0, n0);
  __syncthreads();

  df2 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = df_zero();

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += NT) {
      int mm, kk;
      if (g.transA) { kk = e / BM; mm = e % BM; } else { mm = e / BK; kk = e % BK; }
      const int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < g.M && gk < g.K)
        v = g.transA ? A[(long long)gk * g.lda + gm] : A[(long long)gm * g.lda + gk];
      As[kk][mm] = df_from_double(v);
    }
    for (int e = tid; e < BK * BN; e += NT) {
      int kk, nn;
      if (g.transB) { nn = e / BK; kk = e % BK; } else { kk = e / BN; nn = e % BN; }
      const int gk = k0 + kk, gn = n0 + nn;
      double v = 0.0;
      if (gk < g.K && gn < g.N) {
        v = g.transB ? B[(long long)gn * g.ldb + gk] : B[(long long)gk * g.ldb + gn];
        if (bscale) v = v * brow_at(sc, g, b, gk) * sc.bcol[nn];
      }
      Bs[kk][nn] = df_from_double(v);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      df2 a[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * NTY];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + j * NTX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) df_fma_acc(acc[i][j], a[i], bv[j]);
    }
    __syncthreads();
  }

  double dmax = 0.0;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + i * NTY;
    if (gm >= g.M) continue;
    const double rs = sc.crow[ty + i * NTY];
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + j * NTX;
      if (gn < g.N)
        store_c(g, b, gm, gn, rs, sc.ccol[tx + j * NTX], df_to_double(df_finish(acc[i][j])), dmax);
    }
  }
  fold_drift_max(g, b, dmax);
}

bool use_tiles_64(const GemmArgs<double>& g, int mx) {
  return mx >= 48 && prefer_tiles_64(g.M, g.N, g.batch);
}
bool use_tiles_64(const GemmArgs<float>&, int mx) { return mx >= 48; }

template <typename T>
void launch(const GemmArgs<T>& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  const int mx = g.M > g.N ? g.M : g.N;
  if (use_tiles_64(g, mx)) {
    dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, g.batch);
    k_gemm<T, 64, 64, 16, 4, 4><<<grid, 256, 0, st>>>(g);
  } else if (mx >= 24) {
    dim3 grid((g.N + 31) / 32, (g.M + 31) / 32, g.batch);
    k_gemm<T, 32, 32, 16, 2, 2><<<grid, 256, 0, st>>>(g);
  } else {
    dim3 grid((g.N + 15) / 16, (g.M + 15) / 16, g.batch);
    k_gemm<T, 16, 16, 16, 1, 1><<<grid, 256, 0, st>>>(g);
  }
}

void launch_pair(const GemmArgs<double>& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  const int mx = g.M > g.N ? g.M : g.N;
  if (use_tiles_64(g, mx)) {
    dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, g.batch);
    k_gemm_pair<64, 64, 16, 4, 4><<<grid, 256, 0, st>>>(g);
  } else if (mx >= 24) {
    dim3 grid((g.N + 31) / 32, (g.M + 31) / 32, g.batch);
    k_gemm_pair<32, 32, 16, 2, 2><<<grid, 256, 0, st>>>(g);
  } else {
    dim3 grid((g.N + 15) / 16, (g.M + 15) / 16, g.batch);
    k_gemm_pair<16, 16, 16, 1, 1><<<grid, 256, 0, st>>>(g);
  }
}

}  // namespace

void gemm(const GemmArgs<double>& g, cudaStream_t st) { launch(g, st); }
void gemm_pair(const GemmArgs<double>& g, cudaStream_t st) { launch_pair(g, st); }
void gemm(const GemmArgs<float>& g, cudaStream_t st) { launch(g, st); }

NMC_DEBUG_READER(debug_fail_gemm)

}  // namespace nmc
