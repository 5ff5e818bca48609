// Local Metropolis updates of one time slice with rank-k delayed Green's function updates.
//
// One CTA per chain handles both spins. For slice l the CTA draws the N Philox uniforms
// u_i (counter (l*N+i, sweep, chain, 0)), then visits i = 0..N-1 in order:
//   G^_ii = G0_ii + sum_{q<m} a_q[i] b_q[i]                    (warp 0, both spins)
//   R^sigma = 1 + Delta^sigma (1 - G^_ii), Delta^sigma = e^{-2 sigma lam s} - 1 (FP64)
//   accept iff u_i < |R^up R^dn|
// and on acceptance appends the Sherman-Morrison vectors of the flip,
//   a_m = -(Delta/R^sigma) (e_i - G^_{:,i}),   b_m = G^_{i,:},
// each computed from G0 and the m earlier pairs (all threads). When m reaches k, or at
// the end of the slice, the k pairs are folded into G0 as one rank-k update
// G0 += A B^T. In exact arithmetic this equals applying each rank-1 update at once.
// G0 of both spins sits in shared memory when it fits (N <= 64 in FP64), else in global
// memory (L2); the panels always live in shared memory (k is clamped to fit).
#include "nmc_internal.cuh"
#include "oz_slice.cuh"

namespace nmc {

namespace {

NMC_DEBUG_FLAG

constexpr int kThreads = 256;
// compensated kernel: 256 threads for the panel entries (one entry of G^'s column or row each
// at N = 64) plus one warp whose first thread evaluates the ratio meanwhile
constexpr int kPanelThreads = 256;
constexpr int kThreadsDf = kPanelThreads + 32;

// Thread t owns column c = t % N of rows t / N, t / N + rows_per_pass, ... of both spins:
// 32-bit index arithmetic only, consecutive threads on consecutive columns.
template <typename T>
__device__ void flush(T* G, const T* Ap, const T* Bp, int m, int N, int KK, long long NN,
                      int ns) {
  // G[sp][r][c] += sum_{q<m} A[sp][q][r] * B[sp][q][c]
  const int nthr = blockDim.x;
  if ((int)threadIdx.x >= (nthr / N) * N && nthr >= N) return;
  const int c0 = threadIdx.x % N, r0 = threadIdx.x / N;
  const int rstep = nthr >= N ? nthr / N : 1;
  for (int sp = 0; sp < ns; ++sp) {
    const T* A_ = Ap + sp * KK * N;
    const T* B_ = Bp + sp * KK * N;
    T* Gs = G + sp * NN;
    for (int c = c0; c < N; c += (nthr >= N ? N : nthr)) {
      for (int r = (nthr >= N ? r0 : 0); r < N; r += rstep) {
        T v = Gs[r * N + c];
        for (int q = 0; q < m; ++q) v = fma(A_[q * N + r], B_[q * N + c], v);
        Gs[r * N + c] = v;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 2) k_flip(const FlipArgs<T> f) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_accept[2];  // by attempt parity: see the loop
  __shared__ double s_coef[2];
  __shared__ double s_sign;
  __shared__ unsigned long long s_cnt[3];

  const int c = blockIdx.x;
  const int N = f.N, KK = f.kk;
  const long long NN = (long long)N * N;
  const int ns = f.ns;
  T* Ap = (T*)smraw;                // [ns][KK][N]
  T* Bp = Ap + ns * KK * N;         // [ns][KK][N]
  T* diag = Bp + ns * KK * N;       // [ns][N]
  T* Gs = diag + ns * N;            // [ns][N][N] when g_in_smem
  double* u = (double*)(((uintptr_t)(Gs + (f.g_in_smem ? ns * NN : 0)) + 15) & ~(uintptr_t)15);
  int8_t* sl = (int8_t*)(u + N);

  T* Gg = f.G + (long long)c * ns * NN;
  T* G = f.g_in_smem ? Gs : Gg;
  int8_t* fl = f.fields + ((long long)c * f.L + f.l) * N;
  // Philox counter words of this chain: its global index, and sweeps since its start
  const uint32_t gchain = (uint32_t)(f.chain_id ? f.chain_id[c] : f.chain_offset + c);
  const uint32_t sweep = (uint32_t)((f.ctr ? f.ctr[0] : (long long)f.sweep) -
                                    (f.sweep_base ? f.sweep_base[c] : 0));
  const uint8_t* rp = f.replay ? f.replay + ((long long)c * f.L + f.l) * N : nullptr;

  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sl[i] = fl[i];
    uint32_t ctr[4] = {(uint32_t)(f.l * N + i), sweep, gchain, kTagFlip};
    philox4x32_10(ctr, f.key0, f.key1);
    u[i] = (double)ctr[0] * 2.3283064365386962890625e-10;  // 2^-32
  }
  if (f.g_in_smem)
    for (long long e = threadIdx.x; e < ns * NN; e += blockDim.x) Gs[e] = Gg[e];
  if (threadIdx.x == 0) {
    s_sign = f.sign[c];
    s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ns * N; i += blockDim.x) {
    const int sp = i / N, r = i % N;
    diag[i] = G[sp * NN + (long long)r * N + r];
  }
  __syncthreads();

  // The accept flag is double-buffered by attempt parity: after a rejection there is one
  // barrier per attempt, so thread 0 may write the next attempt's flag while slower threads
  // still read this one. It cannot write this slot again (attempt i+2) before every thread
  // has passed attempt i+1's barrier, which follows its read of attempt i's flag.
  int m = 0;
  for (int i = 0; i < N; ++i) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x, sp = lane >> 4, q0 = lane & 15;
      const T* A_ = Ap + sp * KK * N;
      const T* B_ = Bp + sp * KK * N;
      T sum = T(0);
      if (sp < ns)
        for (int q = q0; q < m; q += 16) sum = fma(A_[q * N + i], B_[q * N + i], sum);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      const T sum_dn = __shfl_sync(0xffffffffu, sum, 16);
      if (lane == 0) {
        const double gu = (double)(diag[i] + sum);
        const int s = sl[i];
        const double du = (s > 0) ? f.dm : f.dp;  // e^{-2 lam s} - 1
        const double dd = (s > 0) ? f.dp : f.dm;  // e^{+2 lam s} - 1
        const double Ru = 1.0 + du * (1.0 - gu);
        // spin down: 1 - G^dn_ii, or G^up_ii when G_dn = I - P G_up^T P
        const double Rd = 1.0 + dd * (ns == 2 ? 1.0 - (double)(diag[N + i] + sum_dn) : gu);
        const double R = Ru * Rd;
        const bool mine = u[i] < fabs(R);
        bool acc = mine;
        if (rp) {
          acc = rp[i] != 0;
          if (acc != mine) s_cnt[2]++;
        }
        s_cnt[0]++;
        s_accept[i & 1] = acc ? 1 : 0;
        if (acc) {
          s_coef[0] = -du / Ru;
          s_coef[1] = -dd / Rd;
          if (R < 0.0) s_sign = -s_sign;
          s_cnt[1]++;
          sl[i] = (int8_t)(-s);
        }
      }
    }
    __syncthreads();
    if (s_accept[i & 1]) {
      const T coef0 = (T)s_coef[0], coef1 = (T)s_coef[1];
      for (int t = threadIdx.x; t < 2 * ns * N; t += blockDim.x) {
        const int sp = t / (2 * N);
        const int kind = (t / N) & 1;
        const int r = t % N;
        const T* Gsp = G + sp * NN;
        const T* A_ = Ap + sp * KK * N;
        const T* B_ = Bp + sp * KK * N;
        if (kind == 0) {  // column i of G^: a_m = coef (e_i - G^_{:,i})
          T v = Gsp[(long long)r * N + i];
          for (int q = 0; q < m; ++q) v = fma(A_[q * N + r], B_[q * N + i], v);
          if (NMC_DCHECK(m < KK && sp < ns && r < N, 111))
            Ap[(sp * KK + m) * N + r] = (sp ? coef1 : coef0) * ((r == i ? T(1) : T(0)) - v);
        } else {          // row i of G^: b_m = G^_{i,:}
          T v = Gsp[(long long)i * N + r];
          for (int q = 0; q < m; ++q) v = fma(A_[q * N + i], B_[q * N + r], v);
          if (NMC_DCHECK(m < KK && sp < ns && r < N, 112)) Bp[(sp * KK + m) * N + r] = v;
        }
      }
      ++m;
      __syncthreads();
      if (m == KK) {
        flush(G, Ap, Bp, m, N, KK, NN, f.ns);
        m = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < ns * N; j += blockDim.x) {
          const int sp = j / N, r = j % N;
          diag[j] = G[sp * NN + (long long)r * N + r];
        }
        __syncthreads();
      }
    }
  }
  if (m > 0) {
    flush(G, Ap, Bp, m, N, KK, NN, f.ns);
    __syncthreads();
  }
  if (f.g_in_smem)
    for (long long e = threadIdx.x; e < ns * NN; e += blockDim.x) Gg[e] = Gs[e];
  for (int i = threadIdx.x; i < N; i += blockDim.x) fl[i] = sl[i];
  if (threadIdx.x == 0) {
    f.sign[c] = s_sign;
    f.counts[3 * c + 0] += s_cnt[0];
    f.counts[3 * c + 1] += s_cnt[1];
    f.counts[3 * c + 2] += s_cnt[2];
  }
}

// Double-float variant. G0, the rank-k panels and every multiply-add are FP32 pairs
// (df.cuh), and a running diagonal dg_j = G^_jj is updated with each accepted flip
// (dg_j += a_m[j] b_m[j]), so an attempt reads G^_ii directly instead of reducing over
// the panels. The acceptance is the FP64 decision u < |R|: R is first evaluated in
// double-float (relative error ~1e-13); when |u - |R|| exceeds a margin of 1e-10 (|R| + 1)
// that value decides, and only inside the margin is R recomputed in FP64 from the same
// G^_ii -- both give the FP64 decision. The update coefficient -Delta/R^sigma uses a
// double-float reciprocal.
__device__ void flush_df(df2* G, const df2* Ap, const df2* Bp, int m, int N, int KK,
                         long long NN, int ns) {
  const int nthr = blockDim.x;
  if ((int)threadIdx.x >= (nthr / N) * N && nthr >= N) return;
  const int c0 = threadIdx.x % N, r0 = threadIdx.x / N;
  const int rstep = nthr >= N ? nthr / N : 1;
  for (int sp = 0; sp < ns; ++sp) {
    const df2* A_ = Ap + sp * KK * N;
    const df2* B_ = Bp + sp * KK * N;
    df2* Gs = G + sp * NN;
    for (int c = c0; c < N; c += (nthr >= N ? N : nthr)) {
      int r = nthr >= N ? r0 : 0;
      // four rows at a time: four independent accumulation chains share each B load
      // (every output still sees the same operations in the same order)
      for (; r + 3 * rstep < N; r += 4 * rstep) {
        df2 a0 = Gs[r * N + c], a1 = Gs[(r + rstep) * N + c];
        df2 a2 = Gs[(r + 2 * rstep) * N + c], a3 = Gs[(r + 3 * rstep) * N + c];
        for (int q = 0; q < m; ++q) {
          const df2 bq = B_[q * N + c];
          const df2* Aq = A_ + q * N + r;
          df_fma_acc(a0, Aq[0], bq);
          df_fma_acc(a1, Aq[rstep], bq);
          df_fma_acc(a2, Aq[2 * rstep], bq);
          df_fma_acc(a3, Aq[3 * rstep], bq);
        }
        Gs[r * N + c] = df_finish(a0);
        Gs[(r + rstep) * N + c] = df_finish(a1);
        Gs[(r + 2 * rstep) * N + c] = df_finish(a2);
        Gs[(r + 3 * rstep) * N + c] = df_finish(a3);
      }
      for (; r < N; r += rstep) {
        df2 acc = Gs[r * N + c];
        for (int q = 0; q < m; ++q) df_fma_acc(acc, A_[q * N + r], B_[q * N + c]);
        Gs[r * N + c] = df_finish(acc);
      }
    }
  }
}

// The same fold on the BF16 tensor cores: G += P Q with P[r][q] = A[q][r], Q[q][c] = B[q][c]
// (q < m <= 16), both cut into exact integer slices (oz_slice.cuh) with one scale per row of
// P and per column of Q; the products of slices s and t go to group s + t (exact in FP32),
// and each group is scaled and added into G in FP32 pairs. The fragments are sliced in
// registers straight from the panels. sEr, sFc: shared scratch of ns * N ints each.
// Used for k <= 16 (one k-step: each warp slices a 16-row block of P once) and N > 64.
// Measured (one compensated sweep, k = 16): N = 144 flips 41.0 ms vs 48.6 ms with the SIMT
// fold; N = 64 slower than the SIMT fold (1.27 vs 1.48 TFLOP/s of flip work), where the
// per-output slicing and scaling outweigh a 16-term double-float sum. For k = 32 at N = 256 a
// version that re-sliced P per n-tile took 1198 ms against 625 ms for the SIMT fold.
constexpr int kTcFlushMaxK = 16;
#ifndef NMC_TC_FLUSH_MIN_N
#define NMC_TC_FLUSH_MIN_N 65
#endif
constexpr int kTcFlushMinN = NMC_TC_FLUSH_MIN_N;

// A fragment (row-major 16 x 16) of P rows r_lo / r_hi = r_lo + 8, k = k0..k0+15: register v
// holds row (v & 1 ? r_hi : r_lo), k = k0 + 2tq + {0, 1} (+8 for v >= 2); the lower half of
// each register holds the lower k.
__device__ __forceinline__ void flush_a_frag(uint32_t (&af)[kOzS][4], const df2* A_, const int* er,
                                             int r_lo, int k0, int m, int N, int tq) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int r = r_lo + ((v & 1) << 3);
    const int q = k0 + 2 * tq + ((v >> 1) << 3);
    const bool rok = r < N;
    const df2 x0 = (rok && q < m) ? A_[q * N + r] : df_zero();
    const df2 x1 = (rok && q + 1 < m) ? A_[(q + 1) * N + r] : df_zero();
    const int e = rok ? er[r] : 0;
    unsigned short s0[kOzS], s1[kOzS];
    slice_bits(x0, e, s0);
    slice_bits(x1, e, s1);
#pragma unroll
    for (int s = 0; s < kOzS; ++s) af[s][v] = (uint32_t)s0[s] | ((uint32_t)s1[s] << 16);
  }
}

// B fragment (16 x 8) of Q column c: register v holds k = k0 + 2tq + {0, 1} (+8 for v = 1).
__device__ __forceinline__ void flush_b_frag(uint32_t (&bf)[kOzS][2], const df2* B_, const int* fc,
                                             int c, int k0, int m, int N, int tq) {
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    const int q = k0 + 2 * tq + (v << 3);
    const bool cok = c < N;
    const df2 y0 = (cok && q < m) ? B_[q * N + c] : df_zero();
    const df2 y1 = (cok && q + 1 < m) ? B_[(q + 1) * N + c] : df_zero();
    const int fe = cok ? fc[c] : 0;
    unsigned short s0[kOzS], s1[kOzS];
    slice_bits(y0, fe, s0);
    slice_bits(y1, fe, s1);
#pragma unroll
    for (int s = 0; s < kOzS; ++s) bf[s][v] = (uint32_t)s0[s] | ((uint32_t)s1[s] << 16);
  }
}

__device__ __forceinline__ void flush_mma(float (&acc)[kOzS][4], const uint32_t (&af)[kOzS][4],
                                          const uint32_t (&bf)[kOzS][2]) {
#pragma unroll
  for (int s = 0; s < kOzS; ++s)
#pragma unroll
    for (int t = 0; t < kOzS; ++t)
      if (s + t < kOzS) mma_bf16(acc[s + t], af[s], bf[t][0], bf[t][1]);
}

// C fragment: register w holds row (w >> 1 ? r_lo + 8 : r_lo), column c0 + 2tq + (w & 1).
__device__ __forceinline__ void flush_store(df2* Gsp, const float (&acc)[kOzS][4], const int* er,
                                            const int* fc, int r_lo, int c0, int N, int tq) {
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const int r = r_lo + ((w >> 1) << 3);
    const int cc = c0 + 2 * tq + (w & 1);
    if (r >= N || cc >= N) continue;
    df2 sum = df_zero();
#pragma unroll
    for (int q = kOzS - 1; q >= 0; --q)
      sum = df_add(sum, df2{acc[q][w] * pow2f(-8 * (q + 2)), 0.f});
    const int ex = er[r] + fc[cc];
    df2* gp = Gsp + (long long)r * N + cc;
    const float se = pow2f(ex);
    *gp = df_add(*gp, df2{sum.hi * se, sum.lo * se});
  }
}

// KS k-steps of 16 (m <= 16 KS): a warp slices a 16-row block of P once and sweeps it across
// all 8-column n-tiles of its spin.
template <int KS>
__device__ __forceinline__ void flush_rows(df2* G, const df2* Ap, const df2* Bp, int m, int N,
                                           int KK, long long NN, int ns, const int* sEr,
                                           const int* sFc, int warp, int nw, int g, int tq,
                                           int nb) {
  for (int job = warp; job < ns * nb; job += nw) {
    const int sp = job / nb, rb = job - sp * nb;
    const int r_lo = rb * 16 + g;
    const df2* A_ = Ap + sp * KK * N;
    const df2* B_ = Bp + sp * KK * N;
    const int* er = sEr + sp * N;
    const int* fc = sFc + sp * N;
    uint32_t af[KS][kOzS][4];
#pragma unroll
    for (int k = 0; k < KS; ++k) flush_a_frag(af[k], A_, er, r_lo, 16 * k, m, N, tq);
#pragma unroll 1
    for (int cn = 0; cn < 2 * nb; ++cn) {
      float acc[kOzS][4];
#pragma unroll
      for (int q = 0; q < kOzS; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[q][w] = 0.f;
#pragma unroll
      for (int k = 0; k < KS; ++k) {
        uint32_t bf[kOzS][2];
        flush_b_frag(bf, B_, fc, cn * 8 + g, 16 * k, m, N, tq);
        flush_mma(acc, af[k], bf);
      }
      flush_store(G + sp * NN, acc, er, fc, r_lo, cn * 8, N, tq);
    }
  }
}

__device__ void flush_tc(df2* G, const df2* Ap, const df2* Bp, int m, int N, int KK,
                         long long NN, int ns, int* sEr, int* sFc) {
  for (int t = threadIdx.x; t < 2 * ns * N; t += blockDim.x) {
    const int which = t / (ns * N), rem = t - which * ns * N;
    const int sp = rem / N, x = rem - sp * N;
    const df2* P = (which ? Bp : Ap) + sp * KK * N + x;
    float mx = 0.f;
    for (int q = 0; q < m; ++q) mx = fmaxf(mx, fabsf(P[q * N].hi));
    // |hi + lo| <= |hi| (1 + 2^-24): one extra bit of headroom
    (which ? sFc : sEr)[rem] = scale_exp(mx) + (mx > 0.f ? 1 : 0);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int nb = (N + 15) >> 4;
  flush_rows<1>(G, Ap, Bp, m, N, KK, NN, ns, sEr, sFc, warp, nw, g, tq, nb);   // m <= 16
}

// TC: fold on the tensor cores (flush_tc) instead of the double-float loop (flush_df); a
// separate instantiation, so the FP32-pipe variant keeps its smaller register footprint.
template <bool TC>
__global__ void __launch_bounds__(kThreadsDf, 2) k_flip_df(const FlipArgs<df2> f) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_accept[2];  // by attempt parity: see the loop
  __shared__ df2 s_coef[2];
  __shared__ double s_sign;
  __shared__ unsigned long long s_cnt[3];

  const int c = blockIdx.x;
  const int N = f.N, KK = f.kk;
  const long long NN = (long long)N * N;
  const int ns = f.ns;
  df2* Ap = (df2*)smraw;
  df2* Bp = Ap + ns * KK * N;
  df2* dg = Bp + ns * KK * N;         // running diagonal of G^, [ns][N]
  df2* Gs = dg + ns * N;
  // uniforms as FP32 pairs: u = x0 * 2^-32 has at most 32 significant bits, so the pair
  // holds it exactly
  df2* udf = (df2*)(((uintptr_t)(Gs + (f.g_in_smem ? ns * NN : 0)) + 15) & ~(uintptr_t)15);
  int8_t* sl = (int8_t*)(udf + N);
  int* sEr = (int*)(((uintptr_t)(sl + N) + 15) & ~(uintptr_t)15);   // flush scales
  int* sFc = sEr + ns * N;

  df2* Gg = f.G + (long long)c * ns * NN;
  df2* G = f.g_in_smem ? Gs : Gg;
  int8_t* fl = f.fields + ((long long)c * f.L + f.l) * N;
  // Philox counter words of this chain: its global index, and sweeps since its start
  const uint32_t gchain = (uint32_t)(f.chain_id ? f.chain_id[c] : f.chain_offset + c);
  const uint32_t sweep = (uint32_t)((f.ctr ? f.ctr[0] : (long long)f.sweep) -
                                    (f.sweep_base ? f.sweep_base[c] : 0));
  const uint8_t* rp = f.replay ? f.replay + ((long long)c * f.L + f.l) * N : nullptr;

  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sl[i] = fl[i];
    uint32_t ctr[4] = {(uint32_t)(f.l * N + i), sweep, gchain, kTagFlip};
    philox4x32_10(ctr, f.key0, f.key1);
    udf[i] = df_from_double((double)ctr[0] * 2.3283064365386962890625e-10);  // 2^-32
  }
  if (f.g_in_smem)
    for (long long e = threadIdx.x; e < ns * NN; e += blockDim.x) Gs[e] = Gg[e];
  if (threadIdx.x == 0) {
    s_sign = f.sign[c];
    s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ns * N; i += blockDim.x) {
    const int sp = i / N, r = i % N;
    dg[i] = G[sp * NN + (long long)r * N + r];
  }
  __syncthreads();

  // Per attempt: every thread first computes its entries of column i and row i of G^ into
  // panel slot m (they do not depend on the decision) while the last thread evaluates the
  // ratio; after the barrier an acceptance only scales the column by the coefficient and
  // updates the running diagonal, and a rejection leaves slot m to the next attempt. The
  // ratio's latency thus hides behind the panel products instead of adding to them. Flags
  // are double-buffered by attempt parity (see k_flip).
  const df2 one{1.f, 0.f};
  const int rt = kPanelThreads;   // the ratio thread: lane 0 of the last warp
  // entry t of the panels (kind 0: column i of G^, kind 1: row i; spin sp; index r)
  auto panel_entry = [&](int t, int i, int m) {
    const int kind = t / (ns * N), e = t - kind * ns * N;
    const int sp = e / N, r = e % N;
    const df2* Gsp = G + sp * NN;
    const df2* A_ = Ap + sp * KK * N;
    const df2* B_ = Bp + sp * KK * N;
    if (kind == 0) {   // column i of G^, row r
      df2 ca = Gsp[(long long)r * N + i];
      for (int q = 0; q < m; ++q) df_fma_acc(ca, A_[q * N + r], B_[q * N + i]);
      df2 v = df_neg(df_finish(ca));
      if (r == i) v = df_add(v, one);
      if (NMC_DCHECK(m < KK && sp < ns && r < N, 101))
        Ap[(sp * KK + m) * N + r] = v;        // times the coefficient once accepted
    } else {           // row i of G^, column r
      df2 rb = Gsp[(long long)i * N + r];
      for (int q = 0; q < m; ++q) df_fma_acc(rb, A_[q * N + i], B_[q * N + r]);
      if (NMC_DCHECK(m < KK && sp < ns && r < N, 102)) Bp[(sp * KK + m) * N + r] = df_finish(rb);
    }
  };
  // When one pass of the panel threads covers both panels (2 ns N <= 256, so N <= 64), each
  // thread keeps one entry for the whole slice: its column or row, spin and index are
  // computed once here instead of by integer divisions at every attempt.
  const bool one_pass = 2 * ns * N <= kPanelThreads;
  const int tp = threadIdx.x;
  const bool has_entry = tp < 2 * ns * N && tp < kPanelThreads;
  const int p_kind = has_entry ? tp / (ns * N) : 0;
  const int p_e = tp - p_kind * ns * N;
  const int p_sp = has_entry ? p_e / N : 0, p_r = has_entry ? p_e % N : 0;
  const df2* const pG = G + p_sp * NN;
  const df2* const pA = Ap + p_sp * KK * N;
  const df2* const pB = Bp + p_sp * KK * N;
  df2* const pOut = (p_kind == 0 ? Ap : Bp) + p_sp * KK * N + p_r;   // + m N
  int m = 0;
  for (int i = 0; i < N; ++i) {
    if (one_pass) {
      if (has_entry) {
        // the same operations as panel_entry, on this thread's fixed entry
        if (p_kind == 0) {   // column i of G^, row p_r
          df2 ca = pG[(long long)p_r * N + i];
          for (int q = 0; q < m; ++q) df_fma_acc(ca, pA[q * N + p_r], pB[q * N + i]);
          df2 v = df_neg(df_finish(ca));
          if (p_r == i) v = df_add(v, one);
          if (NMC_DCHECK(m < KK, 104)) pOut[m * N] = v;
        } else {             // row i of G^, column p_r
          df2 rb = pG[(long long)i * N + p_r];
          for (int q = 0; q < m; ++q) df_fma_acc(rb, pA[q * N + i], pB[q * N + p_r]);
          if (NMC_DCHECK(m < KK, 105)) pOut[m * N] = df_finish(rb);
        }
      }
    } else if (threadIdx.x < kPanelThreads) {
      for (int t = threadIdx.x; t < 2 * ns * N; t += kPanelThreads) panel_entry(t, i, m);
    }
    if (threadIdx.x == rt) {
      const int s = sl[i];
      const df2 gu = dg[i];
      const df2 du = (s > 0) ? f.dm2 : f.dp2;  // e^{-2 lam s} - 1
      const df2 dd = (s > 0) ? f.dp2 : f.dm2;  // e^{+2 lam s} - 1
      const df2 Ru = df_add(one, df_mul(du, df_add(one, df_neg(gu))));
      // spin down: 1 - G^dn_ii, or G^up_ii when G_dn = I - P G_up^T P
      const df2 omd = ns == 2 ? df_add(one, df_neg(dg[N + i])) : gu;
      const df2 Rd = df_add(one, df_mul(dd, omd));
      const df2 R = df_mul(Ru, Rd);
      const df2 diff = df_add(udf[i], df_neg(df_abs(R)));
      const float margin = 1e-10f * (fabsf(R.hi) + 1.f);
      bool mine;
      double Rsign = R.hi;
      if (fabsf(diff.hi) > margin) {
        mine = diff.hi < 0.f;
      } else {  // certified FP64 evaluation from the same G^_ii
        const double g64u = df_to_double(gu);
        const double omd64 = ns == 2 ? 1.0 - df_to_double(dg[N + i]) : g64u;
        const double d64u = (s > 0) ? f.dm : f.dp, d64d = (s > 0) ? f.dp : f.dm;
        const double R64 = (1.0 + d64u * (1.0 - g64u)) * (1.0 + d64d * omd64);
        mine = df_to_double(udf[i]) < fabs(R64);
        Rsign = R64;
      }
      bool acc_flip = mine;
      if (rp) {
        acc_flip = rp[i] != 0;
        if (acc_flip != mine) s_cnt[2]++;
      }
      s_cnt[0]++;
      s_accept[i & 1] = acc_flip ? 1 : 0;
      if (acc_flip) {
        s_coef[0] = df_neg(df_mul(du, df_rcp(Ru)));
        s_coef[1] = df_neg(df_mul(dd, df_rcp(Rd)));
        if (Rsign < 0.0) s_sign = -s_sign;
        s_cnt[1]++;
        sl[i] = (int8_t)(-s);
      }
    }
    __syncthreads();
    if (s_accept[i & 1]) {
      if (one_pass) {   // thread t < ns N: spin t / N, index t % N (ns N <= 128 <= threads)
        if (tp < ns * N && NMC_DCHECK(m < KK, 103)) {
          const int sp = tp >= N ? 1 : 0, r = tp - sp * N;
          const long long o = (long long)(sp * KK + m) * N + r;
          const df2 a = df_mul(s_coef[sp], Ap[o]);
          Ap[o] = a;
          dg[tp] = df_add(dg[tp], df_mul(a, Bp[o]));
        }
      } else {
        for (int t = threadIdx.x; t < ns * N; t += blockDim.x) {
          const int sp = t / N, r = t % N;
          const long long o = (long long)(sp * KK + m) * N + r;
          if (!NMC_DCHECK(m < KK, 103)) continue;
          const df2 a = df_mul(s_coef[sp], Ap[o]);
          Ap[o] = a;
          dg[t] = df_add(dg[t], df_mul(a, Bp[o]));
        }
      }
      ++m;
      __syncthreads();
      if (m == KK) {
        if constexpr (TC) flush_tc(G, Ap, Bp, m, N, KK, NN, ns, sEr, sFc);
        else flush_df(G, Ap, Bp, m, N, KK, NN, ns);
        m = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < ns * N; j += blockDim.x) {
          const int sp = j / N, r = j % N;
          dg[j] = G[sp * NN + (long long)r * N + r];
        }
        __syncthreads();
      }
    }
  }
  if (m > 0) {
    if constexpr (TC) flush_tc(G, Ap, Bp, m, N, KK, NN, ns, sEr, sFc);
    else flush_df(G, Ap, Bp, m, N, KK, NN, ns);
    __syncthreads();
  }
  if (f.g_in_smem)
    for (long long e = threadIdx.x; e < ns * NN; e += blockDim.x) Gg[e] = Gs[e];
  for (int i = threadIdx.x; i < N; i += blockDim.x) fl[i] = sl[i];
  if (threadIdx.x == 0) {
    f.sign[c] = s_sign;
    f.counts[3 * c + 0] += s_cnt[0];
    f.counts[3 * c + 1] += s_cnt[1];
    f.counts[3 * c + 2] += s_cnt[2];
  }
}

}  // namespace

size_t flip_smem_bytes(int N, int kk, size_t elem, int g_in_smem, int ns) {
  size_t b = (size_t)(2 * ns * kk * N + ns * N) * elem;
  if (g_in_smem) b += (size_t)ns * N * N * elem;
  b = (b + 15) & ~(size_t)15;
  b += (size_t)N * sizeof(double) + (size_t)N + 16;
  b += 2 * (size_t)ns * N * sizeof(int) + 16;   // scales of the tensor-core flush
  return b;
}

template <typename T>
void flip_slice(const FlipArgs<T>& f, int n_chains, cudaStream_t st) {
  const size_t bytes = flip_smem_bytes(f.N, f.kk, sizeof(T), f.g_in_smem, f.ns);
  allow_max_dynamic_smem((const void*)k_flip<T>);
  k_flip<T><<<n_chains, kThreads, bytes, st>>>(f);
}

template void flip_slice<double>(const FlipArgs<double>&, int, cudaStream_t);
template void flip_slice<float>(const FlipArgs<float>&, int, cudaStream_t);

template <>
void flip_slice<df2>(const FlipArgs<df2>& f, int n_chains, cudaStream_t st) {
  const size_t bytes = flip_smem_bytes(f.N, f.kk, sizeof(df2), f.g_in_smem, f.ns);
  if (f.tc_fold && f.kk <= kTcFlushMaxK && f.N >= kTcFlushMinN) {
    allow_max_dynamic_smem((const void*)k_flip_df<true>);
    k_flip_df<true><<<n_chains, kThreadsDf, bytes, st>>>(f);
  } else {
    allow_max_dynamic_smem((const void*)k_flip_df<false>);
    k_flip_df<false><<<n_chains, kThreadsDf, bytes, st>>>(f);
  }
}

NMC_DEBUG_READER(debug_fail_flip)

}  // namespace nmc
