// FP64-class products on the Blackwell tensor cores (tcgen05, accumulators in tensor memory,
// operands staged in shared memory, the constant operand brought in by TMA), by exact
// integer slicing (Ozaki-style error-free splitting; Ozaki, Ogita, Oishi, Rump, Numer.
// Algorithms 2012).
//
// Every propagation product of the sweep has one constant operand (e^{-+dtau K},
// e^{-+dtau K/2}, shared by all chains) and one chain operand X (an FP32-pair matrix of one
// chain and spin). The kernel forms D = A B^T with A = rows of the chain operand and
// B = rows of the constant, each row scaled by a power of two 2^-e so that its entries lie
// in (-1/2, 1/2) and cut into 7 slices c_s, multiples of q_s = 2^{-8(s+1)} with
// |c_s| <= 256 q_s, each exact in BF16 (stored pre-scaled, so a slice product c_s d_t
// carries its own weight):
//     x 2^-e = sum_s c_s   (hi part: slices 0..6; lo part, |lo| < 2^-25: slices 3..6;
//                           what is left is below 2^-57).
// Slice products are exact in FP32. The tensor core accumulates the 28 slice pairs with
// s + t <= 6 into seven accumulators, one per group g = s + t (groups 0..2 exact for
// K <= 340, group 3 for K <= 160; the dropped pairs weigh < 2^-56 of the row and column
// maxima). The epilogue adds groups 4..6 in FP32, then groups 0..3 and that sum in FP32
// pairs, and scales by 2^{e_row + f_col}.
//
// Matrix shapes: all batch x N rows of the chain operand are one long M dimension (the
// constant is shared), cut into tiles of at most 128 rows (one tensor-memory lane per row;
// fewer when that fills every wave of a multi-wave grid, balanced_rows_per_tile); the
// output columns are cut into tiles of NT <= 64 (seven accumulators x NT columns of tensor
// memory), K into chunks of KC = 32 (16 for N <= 16). One CTA of 544 threads per (row
// tile, column tile), one CTA per SM: 16 warps slice the chain operand's rows into two
// shared-memory stages and later read the accumulators, and one warp issues the TMA copies
// of the constant's slices and the MMAs. (A persistent variant with separate slicing,
// MMA and epilogue warps overlapping consecutive tiles, the constant resident in shared
// memory and two accumulator buffers, measured the same time per launch at N = 64: the
// kernel is bound by its slicing and combining instructions, not by the order of its
// phases.)
//
// C = Cst X (constant on the left) is computed transposed: C^T = X^T Cst^T, so the rows of
// the chain operand are the columns of X, and the epilogue writes C^T's rows as C's columns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "nmc_internal.cuh"

namespace nmc {

namespace {

NMC_DEBUG_FLAG

constexpr int kS = 7;            // slices per operand
constexpr int kLoFirst = 3;      // first slice of the lo part of an FP32 pair
constexpr int kAcc = kS;         // one accumulator per group g = s + t = 0..6
constexpr int kM = 128;          // tile rows = tensor-memory lanes
// SL = 512 slicing/epilogue threads (16 warps), column tiles up to 64, one CTA per SM (7 x 64
// accumulator columns), plus one warp that issues the TMA copies and the MMAs. (A variant with
// 256 slicing threads, column tiles of 32 and two CTAs per SM slices every row twice at N = 64;
// it measured 44 us per launch against 35.)
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Test the phase; while it is incomplete the thread is suspended (it issues nothing) until
// the phase completes or about kSuspendNs nanoseconds pass, so waiting threads do not take
// issue slots from the working ones.
constexpr uint32_t kSuspendNs = 20000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// exact sum of two floats as a normalized pair (Knuth's TwoSum)
__device__ __forceinline__ df2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df2{s, e};
}

// pair + float: TwoSum of the high parts, the low part added, then renormalized
__device__ __forceinline__ df2 df_add_f(df2 a, float x) {
  const df2 t = two_sum(a.hi, x);
  return df_norm(t.hi, __fadd_rn(t.lo, a.lo));
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
// store each slice's 8 values as BF16 (exact: integers <= 256 times a power of two), 16
// bytes per slice at dst + s * stride.
__device__ __forceinline__ void slice8_store(const df2 (&v)[8], uint8_t* dst, int stride) {
  float r[8], q[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) r[j] = v[j].hi, q[j] = v[j].lo;
#pragma unroll
  for (int s = 0; s < kS; ++s) {
    float c[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c[j] = round_to_slice(r[j], s);
      r[j] = __fsub_rn(r[j], c[j]);   // exact
      if (s >= kLoFirst) {            // |lo| < 2^-25: its first slice is s = 3
        const float cl = round_to_slice(q[j], s);
        q[j] = __fsub_rn(q[j], cl);
        c[j] = __fadd_rn(c[j], cl);   // exact: both multiples of q_s, sum <= 256 q_s
      }
    }
    // every slice is exact in BF16, so its BF16 pattern is the upper half of its FP32 one:
    // pack two with one byte permutation (low half = the even element)
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h)
      w[h] = __byte_perm(__float_as_uint(c[2 * h]), __float_as_uint(c[2 * h + 1]), 0x7632);
    *reinterpret_cast<uint4*>(dst + s * stride) = make_uint4(w[0], w[1], w[2], w[3]);
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
  int rpt;            // rows of the chain operand per tile (<= 128; the rest of the tile is zero)
};

// Shared memory (bytes, from a 1024-aligned base): two stages of A slices
// [kS][kM/8][KC/8][8][8] bf16, then two stages of B slices [kS][NT/8][KC/8][8][8] bf16.
__host__ __device__ inline int a_bytes(int KC) { return kS * kM * KC * 2; }
__host__ __device__ inline int b_bytes(int NT, int KC) { return kS * NT * KC * 2; }
__host__ __device__ inline uint32_t tmem_columns(int cols) {
  return cols <= 64 ? 64u : cols <= 128 ? 128u : cols <= 256 ? 256u : 512u;
}

constexpr int kCache = 2;                // chunks of a row kept in registers

// One (row tile, column tile) of D = A B^T. Slicing thread t (< 512) handles row
// r = t % 128 of the tile and, in every K chunk, the 8-wide K group t / 128 (of KC / 8): it
// scans, field-scales and slices those entries into the chunk's stage, then its warp signals
// the stage full. The last warp issues the TMA copies of the constant's slices and the MMAs
// of each full stage, and releases the stage when they complete. In the epilogue slicing
// warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its permitted quarter) and 16
// columns starting at 16 (w / 4).
template <bool CONST_A, int SL>
__global__ void __launch_bounds__(SL + 32, SL == 512 ? 1 : 2)
    k_gemm_tc(const DfGemmArgs g, const TcGeom geo, const __grid_constant__ CUtensorMap tmap) {
  constexpr int kKParts = SL / kM;   // slicing threads per row of the tile (4 or 2)
  extern __shared__ uint8_t smraw[];
  __shared__ uint64_t bar_tma[2], bar_mma[2], bar_full[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int fexp[64];
  __shared__ int rexp[kM];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = g.N, NT = geo.NT, KC = geo.KC, n_chunks = geo.n_chunks;
  const int n_tile = blockIdx.y;
  const bool mma_warp = warp == SL / 32;
  uint8_t* base = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  // stage st: A slices at base + st * a_bytes, B slices at base + 2 a_bytes + st * b_bytes
  auto As = [&](int st) { return base + st * a_bytes(KC); };
  auto Bs = [&](int st) { return base + 2 * a_bytes(KC) + st * b_bytes(NT, KC); };
  const uint32_t tmem_cols = tmem_columns(kAcc * NT);

  if (tid == 0) {
    for (int k = 0; k < 2; ++k) {
      mbar_init(&bar_tma[k], 1);
      mbar_init(&bar_mma[k], 1);
      mbar_init(&bar_full[k], SL / 32);   // one arrival per slicing warp
    }
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

  // this thread's row of the chain operand: matrix b, index i (a row of X, or a column of X
  // when the constant is on the left), and its K group within each chunk
  // kKParts consecutive lanes share a row (one 8-wide K group each), so a warp reads
  // contiguous runs of its rows and writes their 16-byte slice pieces contiguously
  const int r = (warp * (32 / kKParts) + lane / kKParts) & (kM - 1), kp = lane & (kKParts - 1);
  const bool kpart = !mma_warp && kp * 8 < KC;   // KC = 16: only two K groups per chunk
  const long long grow = (long long)blockIdx.x * geo.rpt + r;
  const bool valid = r < geo.rpt && grow < geo.rows;
  const int b = valid ? (int)(grow / N) : 0;
  const int i = valid ? (int)(grow % N) : 0;
  const df2* X = CONST_A ? g.B + (long long)b * g.sB : g.A + (long long)b * g.sA;
  const int ldx = CONST_A ? g.ldb : g.lda;
  const int sg = (g.ns == 2 && (b & 1)) ? -1 : 1;
  const long long fchain = (long long)(g.ns == 2 ? b >> 1 : b) * g.fstride;
  const bool bf = g.bfields != nullptr;
  const int si_b = bf && valid ? field_sign(g.bfields, fchain + i) : 1;
  // 8 entries k0 .. k0 + 7 of the row (X[k][i] or X[i][k]) with their field factors: the
  // loads are issued together, then scaled
  auto load8 = [&](int k0, df2 (&v)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + j;
      v[j] = (valid && k < N) ? (CONST_A ? X[(long long)k * ldx + i] : X[(long long)i * ldx + k])
                              : df_zero();
    }
    if (bf) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int k = k0 + j;
        if (!valid || k >= N) continue;
        const int sk = field_sign(g.bfields, fchain + k);
        const int m = CONST_A ? sg * (g.br * sk + g.bc * si_b) : sg * (g.br * si_b + g.bc * sk);
        if (m) v[j] = df_mul(v[j], g.e[m + 2]);
      }
    }
  };

  // pass 1: this thread's share of the row maximum (its entries kept when N <= 64)
  const bool cache = n_chunks <= kCache;
  df2 keep[kCache][8];
  float mx = 0.f;
  if (kpart) {
    if (cache) {
      load8(kp * 8, keep[0]);
      if (n_chunks > 1) load8(KC + kp * 8, keep[1]);
#pragma unroll
      for (int c = 0; c < kCache; ++c)
#pragma unroll
        for (int j = 0; j < 8; ++j) mx = fmaxf(mx, (c < n_chunks) ? fabsf(keep[c][j].hi) : 0.f);
    } else {
      for (int c = 0; c < n_chunks; ++c) {
        df2 v[8];
        load8(c * KC + kp * 8, v);
#pragma unroll
        for (int j = 0; j < 8; ++j) mx = fmaxf(mx, fabsf(v[j].hi));
      }
    }
  }
  // the row maximum over the row's lanes
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  if (kKParts == 4) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
  if (!mma_warp && kp == 0) rexp[r] = row_exponent(mx);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  bool ok = true;

  if (mma_warp) {
    // ---------------------------------------------------------------- TMA + MMA warp
    if (lane == 0) {
      const uint32_t lbo = 128, sbo = (uint32_t)(KC / 8) * 128;
      const int box_rows = kS * (NT / 8) * (KC / 8);
      // the constant's first two chunks: both stages are free
      for (int c = 0; c < 2 && c < n_chunks; ++c) {
        mbar_expect_tx(&bar_tma[c], (uint32_t)b_bytes(NT, KC));
        tma_load_2d(Bs(c), &tmap, 0, (n_tile * n_chunks + c) * box_rows, &bar_tma[c]);
      }
      for (int kc = 0; kc < n_chunks && ok; ++kc) {
        const int st = kc & 1, use = kc >> 1;
        ok = mbar_wait(&bar_full[st], use & 1, geo.err, 3) && ok;   // A slices written
        ok = mbar_wait(&bar_tma[st], use & 1, geo.err, 4) && ok;    // B slices landed
        if (!ok) break;
        tc_fence_after();
        const uint32_t a_base = smem_u32(As(st)), b_base = smem_u32(Bs(st));
        // One instruction multiplies A slice s by up to four consecutive B slices t0..t0+3,
        // stacked along N: its D columns (s + t) NT are exactly group s + t's accumulator.
        for (int ks = 0; ks < KC / 16; ++ks) {
#pragma unroll 1
          for (int s = 0; s < kS; ++s) {
            const uint64_t ad = smem_desc(a_base + s * (kM * KC * 2) + ks * 256, lbo, sbo);
            for (int t0 = 0; s + t0 < kS; t0 += 4) {
              const int m = kS - s - t0 < 4 ? kS - s - t0 : 4;
              const uint64_t bd = smem_desc(b_base + t0 * (NT * KC * 2) + ks * 256, lbo, sbo);
              // the first instructions (s = 0) write every accumulator once: overwrite
              const bool first = kc == 0 && ks == 0 && s == 0;
              mma_bf16_ss(tmem + (uint32_t)((s + t0) * NT), ad, bd, idesc_bf16(kM, m * NT),
                          first ? 0u : 1u);
            }
          }
        }
        mma_commit(&bar_mma[st]);   // arrives when this chunk's MMAs have completed
        // with this chunk's MMAs queued, wait for the previous chunk's and refill its stage
        // with the constant's chunk kc + 1
        if (kc >= 1 && kc + 1 < n_chunks) {
          const int pst = (kc - 1) & 1;
          ok = mbar_wait(&bar_mma[pst], ((kc - 1) >> 1) & 1, geo.err, 2) && ok;
          if (!ok) break;
          mbar_expect_tx(&bar_tma[pst], (uint32_t)b_bytes(NT, KC));
          tma_load_2d(Bs(pst), &tmap, 0, (n_tile * n_chunks + kc + 1) * box_rows, &bar_tma[pst]);
        }
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- slicing warps
    const float xs = p2(-rexp[r]);
    for (int kc = 0; kc < n_chunks; ++kc) {
      const int st = kc & 1, use = kc >> 1;
      if (kc >= 2)   // this stage's previous MMAs (chunk kc - 2) have completed
        ok = mbar_wait(&bar_mma[st], (use - 1) & 1, geo.err, 1) && ok;
      // rows past the tile's (or the operand's) end are left unsliced: each output row of the
      // MMA depends on its own A row only, and the epilogue discards those rows
      if (kpart && valid) {
        df2 v[8];
        if (cache) {
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = kc == 0 ? keep[0][j] : keep[1][j];
        } else {
          load8(kc * KC + kp * 8, v);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = df2{v[j].hi * xs, v[j].lo * xs};
        const int off = (r >> 3) * (KC / 8) * 128 + kp * 128 + (r & 7) * 16;
        if (NMC_DCHECK(off + 16 <= kM * KC * 2 && r < kM, 301))
          slice8_store(v, As(st) + off, kM * KC * 2);
      }
      fence_proxy_async();   // the slices, written by threads, are read by the tensor core
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_full[st]);
    }
    {
      const int last = n_chunks - 1;
      ok = mbar_wait(&bar_mma[last & 1], (last >> 1) & 1, geo.err, 5) && ok;
    }
    tc_fence_after();

    // ------------------------------------------------------------ epilogue (slicing warps)
    const int lq = warp & 3, cq = warp >> 2;
    const int c0 = cq * 16;
    if (c0 < NT) {
      const int re = lq * 32 + lane;   // the tile row of this lane
      const long long grow_e = (long long)blockIdx.x * geo.rpt + re;
      const bool valid_e = re < geo.rpt && grow_e < geo.rows;
      const int be = valid_e ? (int)(grow_e / N) : 0;
      const int ie = valid_e ? (int)(grow_e % N) : 0;
      const int sge = (g.ns == 2 && (be & 1)) ? -1 : 1;
      const long long fch = (long long)(g.ns == 2 ? be >> 1 : be) * g.fstride;
      const uint32_t lane_addr = tmem + ((uint32_t)(lq * 32) << 16);
      const int xe = rexp[re];
      const bool cf = g.cfields != nullptr;
      const int si_c = cf && valid_e ? field_sign(g.cfields, fch + ie) : 1;
      for (int h = 0; h < 16; h += 8) {
        // groups 0 and 1 as exact pairs, then the other accumulators added in FP32 pairs
        float a[kAcc][8];
#pragma unroll
        for (int q = 0; q < kAcc; ++q) tmem_ld8(lane_addr + (uint32_t)(q * NT + c0 + h), a[q]);
        tmem_wait_ld();
        if (!valid_e || !ok) continue;
        if (!NMC_DCHECK((kAcc - 1) * NT + c0 + h + 8 <= (int)tmem_cols && be < g.batch, 302)) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int n = n_tile * NT + c0 + h + j;
          if (n >= N) continue;
          // groups 4..6 (below 2^-32 of the product) summed in FP32, smallest first; groups
          // 0 and 1 as an exact pair, then groups 2, 3 and that sum added in FP32 pairs
          const float t = __fadd_rn(__fadd_rn(a[6][j], a[5][j]), a[4][j]);
          df2 sum = two_sum(a[0][j], a[1][j]);
          sum = df_add_f(sum, a[2][j]);
          sum = df_add_f(sum, a[3][j]);
          sum = df_add_f(sum, t);
          const int ex = xe + fexp[c0 + h + j];
          const float se = (ex >= -126 && ex <= 127) ? p2(ex) : ldexpf(1.f, ex);
          df2 out{sum.hi * se, sum.lo * se};
          // output element C[rr][cc]: (n, i) when the constant is on the left, else (i, n)
          const int rr = CONST_A ? n : ie, cc = CONST_A ? ie : n;
          if (cf) {
            const int sn = field_sign(g.cfields, fch + n);
            const int m =
                CONST_A ? sge * (g.cr * sn + g.cc * si_c) : sge * (g.cr * si_c + g.cc * sn);
            if (m) out = df_mul(out, g.e[m + 2]);
          }
          const long long idx = (long long)be * g.sC + (long long)rr * g.ldc + cc;
          if (g.Cd) {
            double d = df_to_double(out);
            if (g.colscale) d *= g.colscale[(long long)be * g.sColscale + cc];
            g.Cd[idx] = d;
          } else {
            g.C[idx] = out;
          }
        }
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
    const int kc = k0 / KC, kg = (k0 % KC) / 8;
    const long long blk = (long long)nt * n_chunks + kc;
    const long long off = blk * kS * NT * KC + (long long)(nn >> 3) * (KC / 8) * 64 + kg * 64 +
                          (nn & 7) * 8;
    slice8_store(v, (uint8_t*)(out + off), NT * KC * 2);
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
  s.SL = 512;
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

// Rows per tile: kM, unless the grid takes several waves of `slots` resident CTAs; then the
// fewest rows that still fill those waves, so that the last wave is not a partial one (the
// slicing and the epilogue, which bound the kernel, scale with a tile's rows).
static int balanced_rows_per_tile(long long rows, int n_col_tiles, int slots) {
  const long long tiles = ((rows + kM - 1) / kM) * n_col_tiles;
  const long long waves = (tiles + slots - 1) / slots;
  if (waves < 2 || slots < 1) return kM;
  const long long row_tiles = waves * slots / n_col_tiles;
  const long long rpt = (rows + row_tiles - 1) / row_tiles;
  return (int)(rpt < 1 ? 1 : rpt > kM ? kM : rpt);
}

void gemm_tc(const DfGemmArgs& g, bool const_is_a, const void* tmap, int* err,
             cudaStream_t st) {
  if (g.batch <= 0) return;
  const TcShape s = tc_shape(g.N);
  TcGeom geo{s.NT, s.KC, s.KP, s.n_chunks, s.n_tiles, (long long)g.batch * g.N, err, kM};
  // Tensor memory holds 512 columns per SM: request enough shared memory that no more CTAs
  // share an SM than their accumulators fit (228 KB per SM, 1 KB reserved per CTA).
  const int cols = (int)tmem_columns(kAcc * s.NT);
  const size_t fit = 233472 / (512 / cols + 1) - 1024 + 16;
  size_t smem = (size_t)2 * (a_bytes(s.KC) + b_bytes(s.NT, s.KC)) + 1024;
  if (smem < fit) smem = fit;
  geo.rpt = balanced_rows_per_tile(geo.rows, s.n_tiles, sm_count() * (512 / cols));
  const dim3 grid((unsigned)((geo.rows + geo.rpt - 1) / geo.rpt), (unsigned)s.n_tiles);
  const CUtensorMap& m = *(const CUtensorMap*)tmap;
  auto run = [&](auto kernel, int threads) {
    allow_max_dynamic_smem((const void*)kernel);
    kernel<<<grid, threads, smem, st>>>(g, geo, m);
  };
  if (const_is_a) run(k_gemm_tc<true, 512>, 512 + 32);
  else run(k_gemm_tc<false, 512>, 512 + 32);
}

NMC_DEBUG_READER(debug_fail_gemm_tc)

}  // namespace nmc
