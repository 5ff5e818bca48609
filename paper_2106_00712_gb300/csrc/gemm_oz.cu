// FP64-class products on the BF16 tensor cores by exact integer slicing (Ozaki-style
// error-free splitting; Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 2012).
//
// Each row of A (or column of B) is scaled by a power of two 2^e so its entries lie in
// (-1/2, 1/2), then cut into S integer slices: x = 2^e sum_s a_s 2^{-8s}, |a_s| <= 129.
// Integers of that size are exact in BF16, a slice product a_s b_t is exact, and a K = 64
// sum of such products stays below 2^24 and is exact in the FP32 accumulator. The product is
//     C_ij = 2^{e_i + f_j} sum_g 2^{-8g} P_g(i,j),   P_g = sum_{s+t=g} A_s B_t,
// with each group g = s + t accumulated separately (at most 7 pairs: every group sum stays
// below 7.5e6 < 2^24) and the groups combined in double-float in the epilogue. With S = 7
// and g <= S + 1 (28 slice products) the dropped terms are ~2^-49 of the row/column maxima
// -- the precision of the double-float SIMT path, at tensor-core throughput.
//
// Two CTAs per N x N product (N <= 64, zero-padded to 64), each computing one 64 x 32 half
// with 8 warps; each warp a 16 x 16 output block (two m16n8k16 n-tiles) with 7 group
// accumulators. One operand is a shared
// constant (e^{-+dtau K}, e^{-+dtau K/2}), sliced once per context; the other is the chain's
// matrix (FP32 pairs), scaled by the field factors while staged, sliced in shared memory.
#include <cuda_bf16.h>

#include "nmc_internal.cuh"
#include "oz_slice.cuh"

namespace nmc {

namespace {

constexpr int kS = kOzS;       // slices per operand
constexpr int kG = kS;         // groups g = 2..S+1
constexpr int kNP = 64;        // padded matrix size
constexpr int kLd = kNP + 8;   // padded row (bf16) -> conflict-free ldmatrix

__device__ __forceinline__ void ldsm_x4(uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3,
                                        const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(a));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                          uint32_t& r3, const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(a));
}

// Asynchronous global -> shared copies (LDGSTS): issued back to back by every thread, so
// the operand loads of a CTA cost one memory latency instead of one per loop iteration.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory"); }

// sigma * lam multiple m = sigma (kr s(r) + kc s(c)) from a chain's field row held in shared
// memory (sf[i] = s(i, l) in {-1, +1})
__device__ __forceinline__ int field_m_sm(const int8_t* sf, int sg, int r, int c, int kr, int kc) {
  return sg * (kr * sf[r] + kc * sf[c]);
}

// Work split: each CTA computes half of one product, the output columns n_off..n_off+31
// when the chain operand is B (it then needs only those 32 columns of B) or the output rows
// m_off..m_off+31 when the chain operand is A (only those rows of A), so the chain operand is
// sliced once in total and two CTAs share an SM: while one slices, the other's MMAs run.
// Shared memory: constant slices [kS][kNP][kLd] bf16 (the whole constant), chain slices
// [kS][64][40] (B half) or [kS][32][kLd] (A half) bf16; the chain operand goes from global
// memory to registers to slices (no staging buffer).
constexpr int kHalf = kNP / 2;
constexpr int kLdH = kHalf + 8;  // padded row of a B half -> conflict-free ldmatrix
constexpr int kThreadsH = 256;   // 8 warps, each a 16 x 16 output block of the 64 x 32 half
constexpr size_t kSliceBytes = (size_t)kS * kNP * kLd * sizeof(__nv_bfloat16);
constexpr size_t kHalfBytesB = (size_t)kS * kNP * kLdH * sizeof(__nv_bfloat16);
constexpr size_t kHalfBytesA = (size_t)kS * kHalf * kLd * sizeof(__nv_bfloat16);
constexpr size_t kHalfBytes = kHalfBytesB > kHalfBytesA ? kHalfBytesB : kHalfBytesA;
constexpr size_t kSmemBytes = kSliceBytes + kHalfBytes;
constexpr int kPerThread = kNP * kHalf / kThreadsH;  // chain elements per thread (8)

template <bool CONST_A>
__global__ void __launch_bounds__(kThreadsH, 2) k_gemm_oz(const DfGemmArgs g) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __nv_bfloat16* Cs = (__nv_bfloat16*)smraw;                   // constant operand slices
  __nv_bfloat16* Xs = (__nv_bfloat16*)(smraw + kSliceBytes);   // chain operand half slices
  __shared__ int8_t sfb[kNP], sfc[kNP];   // field rows of this chain (B staging, epilogue)
  __shared__ int smax[kHalf];             // per chain column (B) / row (A): max |hi| bits
  __shared__ int xexp[kHalf];
  const int N = g.N, b = blockIdx.x >> 1, half = blockIdx.x & 1, tid = threadIdx.x;
  const int off = half * kHalf;          // n_off (chain = B) or m_off (chain = A)
  if (off >= N) return;                  // nothing of this product in the upper half
  const int warp = tid >> 5, lane = tid & 31;
  const int sg = (g.ns == 2 && (b & 1)) ? -1 : 1;
  const long long fchain = (long long)(g.ns == 2 ? b >> 1 : b) * g.fstride;

  // constant operand slices (prepared with the matching row/column scaling): asynchronous,
  // needed only by the MMAs
  {
    const uint4* src = (const uint4*)g.oz_const;
    for (int e = tid; e < (int)(kSliceBytes / 16); e += kThreadsH) cp_async16(Cs + e * 8, src + e);
  }
  cp_async_commit();
  if (tid < kNP) {
    sfb[tid] = (g.bfields && tid < N) ? (g.bfields[fchain + tid] > 0 ? 1 : -1) : 1;
    sfc[tid] = (g.cfields && tid < N) ? (g.cfields[fchain + tid] > 0 ? 1 : -1) : 1;
  }
  if (tid < kHalf) smax[tid] = 0;
  // chain operand half into registers: element j of this thread is e = tid + j * 256 of the
  // 64 x 32 (B: rows k, columns off + c) or 32 x 64 (A: rows off + r, columns k) block
  const df2* X = CONST_A ? g.B + (long long)b * g.sB : g.A + (long long)b * g.sA;
  const int ldx = CONST_A ? g.ldb : g.lda;
  df2 v[kPerThread];
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const int e = tid + j * kThreadsH;
    const int r = CONST_A ? (e >> 5) : off + (e >> 6);
    const int c = CONST_A ? off + (e & 31) : (e & 63);
    v[j] = (r < N && c < N) ? X[(long long)r * ldx + c] : df_zero();
  }
  __syncthreads();   // field rows and smax initialised
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const int e = tid + j * kThreadsH;
    const int r = CONST_A ? (e >> 5) : off + (e >> 6);
    const int c = CONST_A ? off + (e & 31) : (e & 63);
    if (CONST_A && g.bfields) {
      const int m = field_m_sm(sfb, sg, r, c, g.br, g.bc);
      if (m && r < N && c < N) v[j] = df_mul(v[j], g.e[m + 2]);
    }
    // non-negative floats order like their bit patterns
    atomicMax(&smax[CONST_A ? (e & 31) : (e >> 6)], __float_as_int(fabsf(v[j].hi)));
  }
  __syncthreads();
  if (tid < kHalf) {
    const float mx = __int_as_float(smax[tid]);
    // |hi + lo| <= |hi| (1 + 2^-24): one extra bit of headroom
    xexp[tid] = scale_exp(mx) + (mx > 0.f ? 1 : 0);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kPerThread; ++j) {
    const int e = tid + j * kThreadsH;
    if (CONST_A) {
      const int r = e >> 5, c = e & 31;
      slice_value(v[j], xexp[c], Xs + r * kLdH + c, kNP * kLdH);
    } else {
      const int r = e >> 6, c = e & 63;
      slice_value(v[j], xexp[r], Xs + r * kLd + c, kHalf * kLd);
    }
  }
  cp_async_wait<0>();   // the constant slices have landed (this thread's copies)
  __syncthreads();

  // A operand [m][k], B operand [k][n]; warp block: 16 rows x 16 columns
  const __nv_bfloat16* As = CONST_A ? Cs : Xs;
  const __nv_bfloat16* Bs = CONST_A ? Xs : Cs;
  const int ldA = kLd, sliceA = CONST_A ? kNP * kLd : kHalf * kLd;
  const int ldB = CONST_A ? kLdH : kLd, sliceB = CONST_A ? kNP * kLdH : kNP * kLd;
  // local block origin: B half 64 x 32 -> 4 x 2 warps; A half 32 x 64 -> 2 x 4 warps
  const int m0 = CONST_A ? (warp >> 1) * 16 : (warp >> 2) * 16;
  const int n0 = CONST_A ? (warp & 1) * 16 : (warp & 3) * 16;
  float acc[kG][2][4];
#pragma unroll
  for (int q = 0; q < kG; ++q)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[q][j][w] = 0.f;

#pragma unroll 1
  for (int k0 = 0; k0 < kNP; k0 += 16) {
    uint32_t bf[kS][4];
#pragma unroll
    for (int t = 0; t < kS; ++t) {
      const __nv_bfloat16* pb =
          Bs + t * sliceB + (k0 + (lane & 7) + ((lane >> 3) & 1) * 8) * ldB + n0 + (lane >> 4) * 8;
      ldsm_x4_t(bf[t][0], bf[t][1], bf[t][2], bf[t][3], pb);
    }
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      uint32_t af[4];
      const __nv_bfloat16* pa = As + s * sliceA + (m0 + (lane & 15)) * ldA + k0 + (lane >> 4) * 8;
      ldsm_x4(af[0], af[1], af[2], af[3], pa);
#pragma unroll
      for (int t = 0; t < kS; ++t)
        if (s + t < kG) {  // group g = s + t + 2 <= kS + 1
          mma_bf16(acc[s + t][0], af, bf[t][0], bf[t][1]);
          mma_bf16(acc[s + t][1], af, bf[t][2], bf[t][3]);
        }
    }
  }

  // epilogue: C = 2^{e_i + f_j} sum_g 2^{-8g} P_g, smallest groups first, in FP32 pairs
  const int* cexp = g.oz_const_exp;
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int il = m0 + (lane >> 2) + ((w >> 1) << 3);
      const int cl = n0 + j * 8 + (lane & 3) * 2 + (w & 1);
      const int i = CONST_A ? il : off + il;
      const int c = CONST_A ? off + cl : cl;
      if (i >= N || c >= N) continue;
      df2 sum = df_zero();
#pragma unroll
      for (int q = kG - 1; q >= 0; --q)
        sum = df_add(sum, df2{acc[q][j][w] * pow2f(-8 * (q + 2)), 0.f});
      const int ex = CONST_A ? cexp[i] + xexp[cl] : xexp[il] + cexp[c];
      const float se = pow2f(ex);
      df2 out{sum.hi * se, sum.lo * se};
      if (g.cfields) {
        const int m = field_m_sm(sfc, sg, i, c, g.cr, g.cc);
        if (m) out = df_mul(out, g.e[m + 2]);
      }
      const long long idx = (long long)b * g.sC + (long long)i * g.ldc + c;
      if (g.Cd) {
        double d = df_to_double(out);
        if (g.colscale) d *= g.colscale[(long long)b * g.sColscale + c];
        g.Cd[idx] = d;
      } else {
        g.C[idx] = out;
      }
    }
}

// Slices of a constant N x N FP64 matrix for use as A (row scaling, as_b = 0) or as B
// (column scaling, as_b = 1): out [kS][kNP][kLd] bf16, exponents [kNP].
__global__ void k_slice_const(const double* M, int N, int as_b, __nv_bfloat16* out, int* exps) {
  __shared__ int ex[kNP];
  const int tid = threadIdx.x;
  if (tid < kNP) {
    double mx = 0.0;
    for (int k = 0; k < N && tid < N; ++k)
      mx = fmax(mx, fabs(as_b ? M[(long long)k * N + tid] : M[(long long)tid * N + k]));
    ex[tid] = scale_exp((float)mx) + (mx > 0.0 ? 1 : 0);
    exps[tid] = ex[tid];
  }
  __syncthreads();
  for (int e = tid; e < kS * kNP * kLd; e += blockDim.x) out[e] = __float2bfloat16_rn(0.f);
  __syncthreads();
  for (int e = tid; e < kNP * kNP; e += blockDim.x) {
    const int r = e >> 6, c = e & 63;
    df2 v = df_zero();
    if (r < N && c < N) v = df_from_double(M[(long long)r * N + c]);
    slice_value(v, as_b ? ex[c] : ex[r], out + r * kLd + c, kNP * kLd);
  }
}

}  // namespace

size_t oz_const_elems() { return (size_t)kS * kNP * kLd; }

void slice_const(const double* M, int N, int as_b, void* out, int* exps, cudaStream_t st) {
  k_slice_const<<<1, 256, 0, st>>>(M, N, as_b, (__nv_bfloat16*)out, exps);
}

bool gemm_oz_supported(int N) { return N <= kNP; }

void gemm_oz(const DfGemmArgs& g, bool const_is_a, cudaStream_t st) {
  if (g.batch <= 0) return;
  const void* f = const_is_a ? (const void*)k_gemm_oz<true> : (const void*)k_gemm_oz<false>;
  allow_max_dynamic_smem(f);
  prefer_max_shared_carveout(f);
  if (const_is_a)
    k_gemm_oz<true><<<2 * g.batch, kThreadsH, kSmemBytes, st>>>(g);
  else
    k_gemm_oz<false><<<2 * g.batch, kThreadsH, kSmemBytes, st>>>(g);
}

}  // namespace nmc
