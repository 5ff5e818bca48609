// FP64-class products on the Blackwell tensor cores (tcgen05, accumulators in tensor memory,
// operands staged in shared memory, the constant operand brought in by TMA), by exact
// integer slicing (Ozaki-style error-free splitting; Ozaki, Ogita, Oishi, Rump, Numer.
// Algorithms 2012).
//
// Every propagation product of the sweep has one constant operand (e^{-+dtau K},
// e^{-+dtau K/2}, shared by all chains) and one chain operand X (an FP32-pair matrix of one
// chain and spin). The kernel forms D = A B^T with A = rows of the chain operand and
// B = rows of the constant, each row scaled by a power of two 2^-e so that its entries lie
// in (-1/2, 1/2) and cut into 6 slices c_s, multiples of q_s = 2^{-8(s+1)} with
// |c_s| <= 256 q_s, each exact in BF16 (stored pre-scaled, so a slice product c_s d_t
// carries its own weight):
//     x 2^-e = sum_s c_s   (hi part: slices 0..5; lo part, |lo| < 2^-25: slices 3..5;
//                           what is left is below 2^-49).
// Slice products are exact in FP32. The tensor core accumulates them in four accumulators:
// the groups g = s + t = 0, 1, 2 each in its own (each group sum is an integer multiple of
// 2^{-8(g+2)} below 2^24 such units for K <= 340, hence exact), and the groups 3..5
// together (their rounding is ~2^-24 of a term that is itself ~2^-24 of the product). The
// 21 slice pairs with s + t <= 5 are issued; the dropped pairs weigh < 2^-48 of the row and
// column maxima. The epilogue adds the four accumulators in FP32 pairs and scales by
// 2^{e_row + f_col}.
//
// Matrix shapes: all batch x N rows of the chain operand are one long M dimension (the
// constant is shared), cut into tiles of 128 rows (one tensor-memory lane per row); the
// output columns are cut into tiles of NT <= 64 (four accumulators x NT columns of tensor
// memory), K into chunks of KC = 32 (16 for N <= 16). One CTA of 128 threads per (row
// tile, column tile): every thread slices its row of the chain operand, thread 0 issues the
// TMA copy of the constant's slices and the MMAs, every thread reads its accumulator lane.
// Two CTAs share an SM (about 72 KB of operands and 256 tensor-memory columns each), so
// one's slicing and epilogue overlap the other's MMAs.
//
// C = Cst X (constant on the left) is computed transposed: C^T = X^T Cst^T, so the rows of
// the chain operand are the columns of X, and the epilogue writes C^T's rows as C's columns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "nmc_internal.cuh"

namespace nmc {

namespace {

constexpr int kS = 6;            // slices per operand
constexpr int kLoFirst = 3;      // first slice of the lo part of an FP32 pair
constexpr int kAcc = 4;          // accumulators: groups 0, 1, 2 exact, 3..5 merged
constexpr int kM = 128;          // tile rows = tensor-memory lanes
constexpr int kThreads = 128;
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz: a bounded wait
constexpr int kMaxTcN = 320;     // exactness of the group-2 sums needs K <= 340

// ---------------------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete, at most kWaitCycles; on expiry
// record `code` in *err and return false.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      if (err) atomicExch(err, code);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// shared-memory matrix descriptor: start address, leading-dimension byte offset (between
// 8x16-byte core matrices adjacent in K), stride byte offset (between core matrices adjacent
// in M/N), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------- slicing
// 2^k exactly (k in the normal range)
__device__ __forceinline__ float p2(int k) { return __int_as_float((k + 127) << 23); }

// Round r to the nearest multiple of q = 2^-8(s+1) by adding and removing 1.5 * 2^23 q.
__device__ __forceinline__ float round_to_slice(float r, int s) {
  const float M = p2(23 - 8 * (s + 1)) * 1.5f;   // 1.5 * 2^{23 - 8(s+1)}
  return __fsub_rn(__fadd_rn(r, M), M);
}

// Cut 8 values (FP32 pairs already scaled into (-1/2, 1/2)) into kS pre-scaled slices and
// pack each slice's 8 values as BF16 (exact: integers <= 256 times a power of two).
__device__ __forceinline__ void slice8(const df2 (&v)[8], uint4 (&out)[kS]) {
  float c[kS][8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float r = v[j].hi;
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      const float cs = round_to_slice(r, s);
      r = __fsub_rn(r, cs);   // exact
      c[s][j] = cs;
    }
    float q = v[j].lo;        // |lo| < 2^-25: its first slice is s = 3
#pragma unroll
    for (int s = kLoFirst; s < kS; ++s) {
      const float cs = round_to_slice(q, s);
      q = __fsub_rn(q, cs);
      c[s][j] = __fadd_rn(c[s][j], cs);   // exact: both multiples of q_s, sum <= 256 q_s
    }
  }
#pragma unroll
  for (int s = 0; s < kS; ++s) {
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(c[s][2 * h], c[s][2 * h + 1]);
      w[h] = *reinterpret_cast<const uint32_t*>(&b);
    }
    out[s] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// exponent e with |x| < 2^(e-1) for every |x| <= m (one bit of headroom), 0 for m = 0
__device__ __forceinline__ int row_exponent(float m) {
  if (!(m > 0.f)) return 0;
  int e;
  frexpf(m, &e);   // m = f 2^e, f in [0.5, 1)
  return e + 1;
}

__device__ __forceinline__ int field_sign(const int8_t* f, long long idx) {
  return f[idx] > 0 ? 1 : -1;
}

struct TcGeom {
  int NT, KC, KP, n_chunks, n_tiles;
  long long rows;     // batch * N
  int* err;           // device error flag (bounded waits)
};

// Shared-memory layout (bytes, from a 1024-aligned base): A slices [kS][kM/8][KC/8][8][8] bf16,
// then B slices [kS][NT/8][KC/8][8][8] bf16, then barriers and per-row/column exponents.
__host__ __device__ inline int a_bytes(int KC) { return kS * kM * KC * 2; }
__host__ __device__ inline int b_bytes(int NT, int KC) { return kS * NT * KC * 2; }

template <bool CONST_A>
__global__ void __launch_bounds__(kThreads, 2)
    k_gemm_tc(const DfGemmArgs g, const TcGeom geo, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ uint8_t smraw[];
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int fexp[64];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = g.N, NT = geo.NT, KC = geo.KC;
  const int n_tile = blockIdx.y;
  uint8_t* base = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  uint8_t* As = base;
  uint8_t* Bs = base + a_bytes(KC);
  const uint32_t tmem_cols = (uint32_t)(kAcc * NT <= 64 ? 64 : kAcc * NT <= 128 ? 128 : 256);

  if (tid == 0) {
    mbar_init(&bar_tma, 1);
    mbar_init(&bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base_sh)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid < NT) {
    const int n = n_tile * NT + tid;
    fexp[tid] = n < N ? g.oz_const_exp[n] : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  // this thread's row of the chain operand: matrix b, index i (a row of X, or a column of X
  // when the constant is on the left)
  const long long grow = (long long)blockIdx.x * kM + tid;
  const bool valid = grow < geo.rows;
  const int b = valid ? (int)(grow / N) : 0;
  const int i = valid ? (int)(grow % N) : 0;
  const df2* X = CONST_A ? g.B + (long long)b * g.sB : g.A + (long long)b * g.sA;
  const int ldx = CONST_A ? g.ldb : g.lda;
  const int sg = (g.ns == 2 && (b & 1)) ? -1 : 1;
  const long long fchain = (long long)(g.ns == 2 ? b >> 1 : b) * g.fstride;
  const bool bf = g.bfields != nullptr;
  const int si_b = bf ? field_sign(g.bfields, fchain + i) : 1;
  // element k of the row: X[k][i] (constant on the left) or X[i][k]
  auto elem = [&](int k) -> df2 { return CONST_A ? X[(long long)k * ldx + i] : X[(long long)i * ldx + k]; };
  auto fmul = [&](int k) -> int {   // field multiple m in e^{m lam} of element k
    if (!bf) return 0;
    const int sk = field_sign(g.bfields, fchain + k);
    // X's (row, col) = (k, i) or (i, k)
    return CONST_A ? sg * (g.br * sk + g.bc * si_b) : sg * (g.br * si_b + g.bc * sk);
  };

  // pass 1: row maximum after the field scaling -> exponent
  int xexp = 0;
  if (valid) {
    float mx = 0.f;
    for (int k = 0; k < N; ++k) {
      const df2 v = elem(k);
      const int m = fmul(k);
      mx = fmaxf(mx, fabsf(v.hi) * (m ? g.e[m + 2].hi : 1.f));
    }
    xexp = row_exponent(mx);
  }
  const float xs = p2(-xexp);
  const uint32_t idesc = idesc_bf16(kM, NT);
  const uint32_t lbo = 128, sbo = (uint32_t)(KC / 8) * 128;
  const uint32_t a_base = smem_u32(As), b_base = smem_u32(Bs);
  const int box_rows = kS * (NT / 8) * (KC / 8);
  bool ok = true;

  for (int kc = 0; kc < geo.n_chunks; ++kc) {
    if (kc > 0) ok = mbar_wait(&bar_mma, (kc - 1) & 1, geo.err, 1) && ok;   // stage free
    if (tid == 0 && ok) {
      mbar_expect_tx(&bar_tma, (uint32_t)b_bytes(NT, KC));
      tma_load_2d(Bs, &tmap, 0, (n_tile * geo.n_chunks + kc) * box_rows, &bar_tma);
    }
    // slice this thread's row, K range [kc KC, kc KC + KC), 8 at a time
    for (int kg = 0; kg < KC / 8; ++kg) {
      df2 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = kc * KC + kg * 8 + j;
        df2 x = df_zero();
        if (valid && k < N) {
          x = elem(k);
          const int m = fmul(k);
          if (m) x = df_mul(x, g.e[m + 2]);
          x.hi *= xs;
          x.lo *= xs;
        }
        v[j] = x;
      }
      uint4 sl[kS];
      slice8(v, sl);
      uint8_t* dst = As + (tid >> 3) * (KC / 8) * 128 + kg * 128 + (tid & 7) * 16;
#pragma unroll
      for (int s = 0; s < kS; ++s) *reinterpret_cast<uint4*>(dst + s * (kM * KC * 2)) = sl[s];
    }
    fence_proxy_async();   // the slices, written by threads, are read by the tensor core
    __syncthreads();
    if (tid == 0 && ok) {
      ok = mbar_wait(&bar_tma, kc & 1, geo.err, 2);
      tc_fence_after();
      if (ok) {
        for (int ks = 0; ks < KC / 16; ++ks) {
#pragma unroll 1
          for (int s = 0; s < kS; ++s) {
            const uint64_t ad = smem_desc(a_base + s * (kM * KC * 2) + ks * 256, lbo, sbo);
            for (int t = 0; s + t < kS; ++t) {
              const int grp = s + t < 3 ? s + t : 3;
              const uint64_t bd = smem_desc(b_base + t * (NT * KC * 2) + ks * 256, lbo, sbo);
              // the first product into each accumulator overwrites it
              const bool first = kc == 0 && ks == 0 && (grp < 3 ? s == 0 : (s == 0 && t == 3));
              mma_bf16_ss(tmem + (uint32_t)(grp * NT), ad, bd, idesc, first ? 0u : 1u);
            }
          }
        }
      }
      mma_commit(&bar_mma);   // arrives when the MMAs above have completed
    }
    __syncthreads();
  }
  ok = mbar_wait(&bar_mma, (geo.n_chunks - 1) & 1, geo.err, 3) && ok;
  tc_fence_after();

  // epilogue: this thread's lane of the four accumulators, 16 columns at a time
  const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
  const bool cf = g.cfields != nullptr;
  const int si_c = cf ? field_sign(g.cfields, fchain + i) : 1;
  for (int c0 = 0; c0 < NT; c0 += 16) {
    float acc[kAcc][16];
#pragma unroll
    for (int q = 0; q < kAcc; ++q) tmem_ld16(lane_addr + (uint32_t)(q * NT + c0), acc[q]);
    tmem_wait_ld();
    if (!valid || !ok) continue;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = n_tile * NT + c0 + j;
      if (n >= N) continue;
      // groups 0 and 1 as an exact pair, then add groups 2 and 3..6
      const float s01 = __fadd_rn(acc[0][j], acc[1][j]);
      const float bb = __fsub_rn(s01, acc[0][j]);
      const float e01 = __fadd_rn(__fsub_rn(acc[0][j], __fsub_rn(s01, bb)), __fsub_rn(acc[1][j], bb));
      df2 sum = df_norm(s01, e01);
      sum = df_add(sum, df2{acc[2][j], 0.f});
      sum = df_add(sum, df2{acc[3][j], 0.f});
      const int ex = xexp + fexp[c0 + j];
      const float se = (ex >= -126 && ex <= 127) ? p2(ex) : ldexpf(1.f, ex);
      df2 out{sum.hi * se, sum.lo * se};
      // output element C[r][c]: (n, i) when the constant is on the left, else (i, n)
      const int r = CONST_A ? n : i, c = CONST_A ? i : n;
      if (cf) {
        const int sn = field_sign(g.cfields, fchain + n);
        const int m = CONST_A ? sg * (g.cr * sn + g.cc * si_c) : sg * (g.cr * si_c + g.cc * sn);
        if (m) out = df_mul(out, g.e[m + 2]);
      }
      const long long idx = (long long)b * g.sC + (long long)r * g.ldc + c;
      if (g.Cd) {
        double d = df_to_double(out);
        if (g.colscale) d *= g.colscale[(long long)b * g.sColscale + c];
        g.Cd[idx] = d;
      } else {
        g.C[idx] = out;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
}

// Slices of a constant N x N FP64 matrix as the B operand: row n of B is row n of M
// (as_b = 0: the constant on the left, C = M X) or column n of M (as_b = 1: C = X M),
// scaled by 2^-f_n (f_n over the row of B), cut into kS pre-scaled slices, written in the
// per-(column tile, K chunk) blocks the kernel's TMA copies: [n_tile][chunk][slice]
// [NT/8][KC/8][8][8] bf16, zero-padded to n_tiles NT x KP.
__global__ void k_tc_slice_const(const double* M, int N, int as_b, int NT, int KC, int KP,
                                 int n_tiles, __nv_bfloat16* out, int* exps) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_tiles * NT) return;
  auto elem = [&](int k) -> double {
    if (n >= N || k >= N) return 0.0;
    return as_b ? M[(long long)k * N + n] : M[(long long)n * N + k];
  };
  float mx = 0.f;
  for (int k = 0; k < N; ++k) mx = fmaxf(mx, fabsf(__double2float_rn(elem(k))));
  const int f = row_exponent(mx);
  if (n < N) exps[n] = f;
  const float fs = p2(-f);
  const int n_chunks = KP / KC, nt = n / NT, nn = n % NT;
  for (int k0 = 0; k0 < KP; k0 += 8) {
    df2 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      df2 x = df_from_double(elem(k0 + j));
      v[j] = df2{x.hi * fs, x.lo * fs};
    }
    uint4 sl[kS];
    slice8(v, sl);
    const int kc = k0 / KC, kg = (k0 % KC) / 8;
    const long long blk = (long long)nt * n_chunks + kc;
    const long long off = blk * kS * NT * KC + (long long)(nn >> 3) * (KC / 8) * 64 + kg * 64 +
                          (nn & 7) * 8;
#pragma unroll
    for (int s = 0; s < kS; ++s)
      *reinterpret_cast<uint4*>(out + off + (long long)s * NT * KC) = sl[s];
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  });
  return fn;
}

}  // namespace

TcShape tc_shape(int N) {
  TcShape s{};
  s.N = N;
  s.KC = N <= 16 ? 16 : 32;
  s.KP = (N + s.KC - 1) / s.KC * s.KC;
  s.n_chunks = s.KP / s.KC;
  // column tile: the multiple of 16 up to 64 that pads N least (ties: the larger tile)
  int best = 64, best_cols = 1 << 30;
  for (int nt = 64; nt >= 16; nt -= 16) {
    const int cols = (N + nt - 1) / nt * nt;
    if (cols < best_cols) best = nt, best_cols = cols;
  }
  s.NT = best;
  s.n_tiles = (N + best - 1) / best;
  return s;
}

bool gemm_tc_supported(int N) { return N >= 2 && N <= kMaxTcN && encode_fn() != nullptr; }

size_t tc_const_elems(int N) {
  const TcShape s = tc_shape(N);
  return (size_t)s.n_tiles * s.NT * s.KP * kS;
}

bool tc_prepare_const(const double* M, int N, int as_b, void* slices, int* exps, void* tmap,
                      cudaStream_t st) {
  const TcShape s = tc_shape(N);
  const int rows = s.n_tiles * s.NT;
  k_tc_slice_const<<<(rows + 63) / 64, 64, 0, st>>>(M, N, as_b, s.NT, s.KC, s.KP, s.n_tiles,
                                                     (__nv_bfloat16*)slices, exps);
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t cms = (cuuint64_t)s.n_tiles * s.n_chunks * kS * (s.NT / 8) * (s.KC / 8);
  const cuuint64_t dims[2] = {64, cms};
  const cuuint64_t strides[1] = {128};
  const cuuint32_t box[2] = {64, (cuuint32_t)(kS * (s.NT / 8) * (s.KC / 8))};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn((CUtensorMap*)tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, slices, dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

void gemm_tc(const DfGemmArgs& g, bool const_is_a, const void* tmap, int* err,
             cudaStream_t st) {
  if (g.batch <= 0) return;
  const TcShape s = tc_shape(g.N);
  TcGeom geo{s.NT, s.KC, s.KP, s.n_chunks, s.n_tiles, (long long)g.batch * g.N, err};
  // Tensor memory holds 512 columns per SM: request enough shared memory that no more CTAs
  // share an SM than their accumulators fit (228 KB per SM, 1 KB reserved per CTA).
  const int cols = kAcc * s.NT <= 64 ? 64 : kAcc * s.NT <= 128 ? 128 : 256;
  const size_t fit = 233472 / (512 / cols + 1) - 1024 + 16;
  size_t smem = (size_t)a_bytes(s.KC) + b_bytes(s.NT, s.KC) + 1024;
  if (smem < fit) smem = fit;
  const dim3 grid((unsigned)((geo.rows + kM - 1) / kM), (unsigned)s.n_tiles);
  const CUtensorMap& m = *(const CUtensorMap*)tmap;
  if (const_is_a) {
    allow_max_dynamic_smem((const void*)k_gemm_tc<true>);
    k_gemm_tc<true><<<grid, kThreads, smem, st>>>(g, geo, m);
  } else {
    allow_max_dynamic_smem((const void*)k_gemm_tc<false>);
    k_gemm_tc<false><<<grid, kThreads, smem, st>>>(g, geo, m);
  }
}

}  // namespace nmc
