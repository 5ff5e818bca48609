// Batched double-float GEMM for the compensated precision mode.
//
// Same tiling as the FP64 SIMT GEMM, with every operand an FP32 pair (hi, lo) and every
// multiply-add an error-free TwoProd + TwoSum accumulation (df.cuh): about 2^-44 relative
// error per product, on the FP32 pipes (12 FP32 operations per multiply-add against one
// operation of the 64x slower FP64 pipe). Used for the wraps
// G <- e^{-dtau K} e^{V} G e^{-V} e^{dtau K} (and the reverse) and for the products
// B_l X of the UDV stacks.
#include "nmc_internal.cuh"

namespace nmc {

namespace {

__device__ __forceinline__ int field_m(const int8_t* f, long long fstride, int ns, int b, int r,
                                       int c, int kr, int kc) {
  const int sg = (ns == 2 && (b & 1)) ? -1 : 1;
  const int8_t* fb = f + (long long)(ns == 2 ? b >> 1 : b) * fstride;
  int m = 0;
  if (kr) m += kr * (fb[r] > 0 ? 1 : -1);
  if (kc) m += kc * (fb[c] > 0 ? 1 : -1);
  return sg * m;
}

template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) k_gemm_df(const DfGemmArgs g) {
  constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
  __shared__ df2 As[BK][BM + 1];
  __shared__ df2 Bs[BK][BN + 1];
  const int b = blockIdx.z;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const df2* __restrict__ A = g.A + (long long)b * g.sA;
  const df2* __restrict__ B = g.B + (long long)b * g.sB;
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  const bool bscale = g.bfields != nullptr;

  df2 acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = df_zero();

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += NT) {
      const int mm = e / BK, kk = e % BK;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < g.M && gk < g.K) ? A[(long long)gm * g.lda + gk] : df_zero();
    }
    for (int e = tid; e < BK * BN; e += NT) {
      const int kk = e / BN, nn = e % BN;
      const int gk = k0 + kk, gn = n0 + nn;
      df2 v = df_zero();
      if (gk < g.K && gn < g.N) {
        v = B[(long long)gk * g.ldb + gn];
        if (bscale) {
          const int m = field_m(g.bfields, g.fstride, g.ns, b, gk, gn, g.br, g.bc);
          if (m) v = df_mul(v, g.e[m + 2]);
        }
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll 4
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

#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + i * NTY;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + j * NTX;
      if (gn >= g.N) continue;
      df2 v = df_finish(acc[i][j]);
      if (g.cfields) {
        const int m = field_m(g.cfields, g.fstride, g.ns, b, gm, gn, g.cr, g.cc);
        if (m) v = df_mul(v, g.e[m + 2]);
      }
      const long long idx = (long long)b * g.sC + (long long)gm * g.ldc + gn;
      if (g.Cd) {
        double d = df_to_double(v);
        if (g.colscale) d *= g.colscale[(long long)b * g.sColscale + gn];
        g.Cd[idx] = d;
      } else {
        g.C[idx] = v;
      }
    }
  }
}

__global__ void k_split(const double* x, df2* y, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = df_from_double(x[e]);
}

}  // namespace

void gemm_df(const DfGemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
  const int mx = g.M > g.N ? g.M : g.N;
  if (mx >= 48 && prefer_tiles_64(g.M, g.N, g.batch)) {
    dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, g.batch);
    k_gemm_df<64, 64, 16, 4, 4><<<grid, 256, 0, st>>>(g);
  } else if (mx >= 24) {
    dim3 grid((g.N + 31) / 32, (g.M + 31) / 32, g.batch);
    k_gemm_df<32, 32, 16, 2, 2><<<grid, 256, 0, st>>>(g);
  } else {
    dim3 grid((g.N + 15) / 16, (g.M + 15) / 16, g.batch);
    k_gemm_df<16, 16, 16, 1, 1><<<grid, 256, 0, st>>>(g);
  }
}

void split_to_df(const double* x, df2* y, long long n, cudaStream_t st) {
  long long grid = (n + 255) / 256;
  if (grid > 152 * 16) grid = 152 * 16;
  if (grid < 1) grid = 1;
  k_split<<<(int)grid, 256, 0, st>>>(x, y, n);
}

}  // namespace nmc
