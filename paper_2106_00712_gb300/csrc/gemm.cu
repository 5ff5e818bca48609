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

__device__ __forceinline__ double nan_max(double a, double b) {
  // max that propagates NaN (fmax would drop it)
  return (b > a || b != b) ? b : a;
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm(const GemmArgs<T> g) {
  constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int b = blockIdx.z;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const T* __restrict__ A = g.A + (long long)b * g.sA;
  const T* __restrict__ B = g.B + (long long)b * g.sB;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  const bool bscale = g.brow.kind != SC_NONE || g.bcol.kind != SC_NONE;

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
        if (bscale) v = (T)((double)v * scale_at(g.brow, b, gk) * scale_at(g.bcol, b, gn));
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

  T* __restrict__ C = g.C + (long long)b * g.sC;
  double dmax = 0.0;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + i * NTY;
    if (gm >= g.M) continue;
    const double rs = scale_at(g.crow, b, gm);
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + j * NTX;
      if (gn >= g.N) continue;
      double v = (double)acc[i][j];
      if (g.crow.kind != SC_NONE || g.ccol.kind != SC_NONE) v = v * rs * scale_at(g.ccol, b, gn);
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
      C[idx] = out;
      if (g.Cf) g.Cf[(long long)b * g.sCf + idx] = (float)out;
      if (g.Cdf) g.Cdf[(long long)b * g.sCdf + idx] = df_from_double((double)out);
    }
  }
  if (g.drift) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = nan_max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((tid & 31) == 0 && dmax != 0.0)
      atomicMax(g.drift + (g.ns == 2 ? b >> 1 : b), (unsigned long long)__double_as_longlong(dmax));
  }
}

template <typename T>
void launch(const GemmArgs<T>& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  const int mx = g.M > g.N ? g.M : g.N;
  if (mx >= 48) {
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

}  // namespace

void gemm(const GemmArgs<double>& g, cudaStream_t st) { launch(g, st); }
void gemm(const GemmArgs<float>& g, cudaStream_t st) { launch(g, st); }

}  // namespace nmc
