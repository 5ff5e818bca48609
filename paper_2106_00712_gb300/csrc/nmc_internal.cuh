// Internal declarations shared by the libnmc translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"

namespace nmc {

// Sublattice of site i on a bipartite lattice (0 or 1); P = diag((-1)^parity) gives
// P K P = -K. Square (lattice 0, i = x + Lx y): (x + y) mod 2. Honeycomb (lattice 1,
// i = 2 (x + Lx y) + sub): sub, i.e. 1 on the B site of each cell.
__host__ __device__ inline int site_parity(int i, int Lx, int lattice) {
  return lattice == 1 ? (i & 1) : (((i % Lx) + (i / Lx)) & 1);
}

// ---------------------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 multiplies with the
// published multipliers, key bumped by the Weyl constants between rounds.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
// Index checks of the NMC_DEBUG build (a bounds-checked variant of the library, built
// beside it as libnmc_debug.so): a failed check records its id in its translation unit's
// device flag (the first failure wins) and the kernel skips the guarded access; the
// library reads the flags after each call that runs kernels. Without NMC_DEBUG a check is
// the constant true and the flags do not exist.
#ifdef NMC_DEBUG
#define NMC_DEBUG_FLAG static __device__ unsigned int g_dbg_fail = 0u;
#define NMC_DCHECK(cond, id) \
  ((cond) ? true : (atomicCAS(&g_dbg_fail, 0u, (unsigned int)(id)), false))
#define NMC_DEBUG_READER(fn)                                     \
  unsigned int fn() {                                            \
    unsigned int v = 0u;                                         \
    if (cudaMemcpyFromSymbol(&v, g_dbg_fail, sizeof v) != cudaSuccess) { \
      cudaGetLastError();                                        \
      return 0xffffffffu;                                        \
    }                                                            \
    return v;                                                    \
  }
#else
#define NMC_DEBUG_FLAG
#define NMC_DCHECK(cond, id) true
#define NMC_DEBUG_READER(fn) \
  unsigned int fn() { return 0u; }
#endif
// the first failed check id of each translation unit with checks (0: none)
unsigned int debug_fail_flip();
unsigned int debug_fail_stab();
unsigned int debug_fail_gemm();
unsigned int debug_fail_gemm_tc();
unsigned int debug_fail_misc();

constexpr uint32_t kTagFlip = 0u;
constexpr uint32_t kTagInit = 1u;

__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c[0];
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
}

// ---------------------------------------------------------------------------- scaling
// Diagonal scale vectors applied inside the batched GEMMs. Batch index b = 2*chain + spin.
enum ScaleKind : int {
  SC_NONE = 0,
  SC_VEC = 1,        // v[i]
  SC_INV_MAX1 = 2,   // 1 / max(v[i], 1)      (D_big^{-1} of a UDT split)
  SC_MIN1 = 3,       // min(v[i], 1)          (D_small of a UDT split)
  SC_FIELD = 4,      // e^{ sigma lam s(i,l)}
  SC_FIELD_INV = 5   // e^{-sigma lam s(i,l)}
};

struct ScaleDesc {
  int kind = SC_NONE;
  int ns = 2;                      // spins per chain in the batch (2, or 1 = spin up only)
  const double* vec = nullptr;   // SC_VEC/INV_MAX1/MIN1: v + b*vstride
  long long vstride = 0;
  const int8_t* fields = nullptr;  // SC_FIELD*: fields + chain*fstride (already + l*N)
  long long fstride = 0;
  double e_lam = 1.0, e_mlam = 1.0;  // e^{lam}, e^{-lam}
};

__device__ __forceinline__ double scale_at(const ScaleDesc& d, int b, int i) {
  switch (d.kind) {
    case SC_VEC: return d.vec[b * d.vstride + i];
    case SC_INV_MAX1: return 1.0 / fmax(d.vec[b * d.vstride + i], 1.0);
    case SC_MIN1: return fmin(d.vec[b * d.vstride + i], 1.0);
    case SC_FIELD:
    case SC_FIELD_INV: {
      const int s = d.fields[(long long)(d.ns == 2 ? b >> 1 : b) * d.fstride + i];
      const bool up = d.ns == 1 || (b & 1) == 0;
      bool pos = (s > 0) == up;          // sigma * s > 0
      if (d.kind == SC_FIELD_INV) pos = !pos;
      return pos ? d.e_lam : d.e_mlam;
    }
    default: return 1.0;
  }
}

// ---------------------------------------------------------------------------- GEMM
// C[b] = crow .* (op(A[b]) * (brow .* op(B[b]) .* bcol)) .* ccol + beta * Cin[b]
// op(A): M x K, op(B): K x N. Optional: write a float copy (Cf), record per-chain
// max |C - ref| (drift) into an array of doubles (as ordered bit patterns).
template <typename T>
struct GemmArgs {
  int M = 0, N = 0, K = 0, batch = 0;
  const T* A = nullptr; long long sA = 0; int lda = 0; int transA = 0;
  const T* B = nullptr; long long sB = 0; int ldb = 0; int transB = 0;
  T* C = nullptr; long long sC = 0; int ldc = 0;
  const T* Cin = nullptr; long long sCin = 0; int ldcin = 0; double beta = 0.0;
  ScaleDesc brow, bcol, crow, ccol;
  float* Cf = nullptr; long long sCf = 0;           // float copy, ld = ldc
  const void* ref = nullptr; int ref_is_float = 0;  // drift reference, ld = ldc, stride sC
  long long sRef = 0;                               // (ref_is_float: 1 = float, 2 = df2)
  unsigned long long* drift = nullptr;              // per chain: bits of max |C - ref|
  df2* Cdf = nullptr; long long sCdf = 0;           // double-float copy, ld = ldc
  int ns = 2;                                       // spins per chain (drift index)
};

void gemm(const GemmArgs<double>& g, cudaStream_t st);
void gemm(const GemmArgs<float>& g, cudaStream_t st);
// The same FP64-in, FP64-out product with the sums accumulated in FP32 pairs on the FP32
// pipe (error-free products and sums, ~2^-44 relative to the sum of |a_ik b_kj|)
void gemm_pair(const GemmArgs<double>& g, cudaStream_t st);

// Double-float GEMM (compensated FP32 pairs): C[b] = e^{V_c} (A[b] (e^{V_b} B[b])) e^{V_c'}
// where the optional diagonal factors are field exponentials e^{m lam}, m = sigma *
// (r * s(row) + c * s(col)) in {-2..2}, applied while staging B (br, bc) or in the
// epilogue (cr, cc). Output either double-float (C) or FP64 (Cd, optionally times a
// per-column FP64 scale colscale[b][n]).
struct DfGemmArgs {
  int M = 0, N = 0, K = 0, batch = 0;
  const df2* A = nullptr; long long sA = 0; int lda = 0;
  const df2* B = nullptr; long long sB = 0; int ldb = 0;
  df2* C = nullptr; double* Cd = nullptr; long long sC = 0; int ldc = 0;
  const double* colscale = nullptr; long long sColscale = 0;
  const int8_t* bfields = nullptr; int br = 0, bc = 0;
  const int8_t* cfields = nullptr; int cr = 0, cc = 0;
  long long fstride = 0;
  int ns = 2;  // spins per chain in the batch
  df2 e[5];    // e^{m lam}, m = -2..2
  // tensor-core path: BF16 slices of the constant operand and the exponents of its rows
  // (constant on the left) or columns (constant on the right)
  const void* oz_const = nullptr;
  const int* oz_const_exp = nullptr;
};
void gemm_df(const DfGemmArgs& g, cudaStream_t st);
// The same products on the tcgen05 tensor cores (accumulators in tensor memory, the constant's
// slices copied by TMA), any N <= 320. Geometry of the tiling for a given N:
struct TcShape { int N, NT, KC, KP, n_chunks, n_tiles, SL; };
TcShape tc_shape(int N);
bool gemm_tc_supported(int N);
size_t tc_const_elems(int N);   // bf16 elements of one sliced constant (one orientation)
// Slice the constant M (as_b = 0: C = M X, rows of M; as_b = 1: C = X M, columns of M) into
// `slices` (device, tc_const_elems(N) bf16), its exponents into `exps` (device, N ints), and
// encode the TMA tensor map over the slices into `tmap` (host, 128 bytes, 64-aligned).
// Returns false if the tensor map cannot be encoded.
bool tc_prepare_const(const double* M, int N, int as_b, void* slices, int* exps, void* tmap,
                      cudaStream_t st);
// g.oz_const_exp = the constant's exponents; err: device int, set on a bounded-wait expiry.
void gemm_tc(const DfGemmArgs& g, bool const_is_a, const void* tmap, int* err, cudaStream_t st);
void split_to_df(const double* x, df2* y, long long n, cudaStream_t st);

// ---------------------------------------------------------------------------- UDT
// Column-pivoted Householder QR of X[b] (N x N row-major): X P = Q R. Writes Q (U),
// D = |diag R| and Tp = D^{-1} R P^T. ws: per-matrix global workspace of 2*N*N doubles
// (used when the matrix does not fit in shared memory).
void qrp_udt(const double* X, double* U, double* D, double* Tp, double* ws, int N, int batch,
             cudaStream_t st);

// Y[b] = X[b]^{-1} * (diag(1/max(DR,1)) * UR[b]^T) by Gauss-Jordan with partial pivoting.
void solve_stab(const double* X, const double* UR, long long sUR, const double* DR,
                long long sDR, double* Y, double* ws, int N, int batch, cudaStream_t st);

// ---------------------------------------------------------------------------- flips
template <typename T>
struct FlipArgs {
  T* G;                      // [chain][spin][N][N]
  int8_t* fields;            // [chain][L][N]
  int N, L, l;               // slice l
  int kk;                    // delay
  int g_in_smem;
  uint32_t key0, key1, sweep;
  long long chain_offset;
  double dm, dp;             // e^{-2 lam} - 1, e^{2 lam} - 1
  double* sign;              // per chain
  unsigned long long* counts;  // per chain: attempts, accepts, disagreements
  const uint8_t* replay;     // [chain][L][N] or null
  T* panels_g;               // unused (panels live in shared memory)
  df2 dm2, dp2;              // dm, dp as FP32 pairs (compensated mode)
  int ns;                    // 2 spins, or 1: spin up only, G_dn = I - P G_up^T P
  const long long* ctr;      // device counters (ctr[0] = sweep counter) or null: use sweep
  int tc_fold = 0;           // compensated mode: 1 = rank-k fold may use the tensor cores
  const long long* chain_id = nullptr;    // per chain: global index (Philox word 2), or null
  const long long* sweep_base = nullptr;  // per chain: sweep counter at its start, or null
};
template <typename T> void flip_slice(const FlipArgs<T>& f, int n_chains, cudaStream_t st);
size_t flip_smem_bytes(int N, int kk, size_t elem, int g_in_smem, int ns);

// ---------------------------------------------------------------------------- misc
// Raise a kernel's dynamic shared-memory limit to the device maximum (once per device).
void allow_max_dynamic_smem(const void* func);
// The SMs of the current device (cached per device; 1 if the query fails)
int sm_count();
// Fill of the last round of CTAs when `ctas` equal CTAs share `sms` SMs: each SM's time grows
// with the CTAs it is given (they share its pipes), so the grid takes ceil(ctas / sms)
// CTA-times while the average SM needs ctas / sms.
inline double sm_fill(long long ctas, int sms) {
  const long long per = (ctas + sms - 1) / sms;
  return per > 0 ? (double)ctas / ((double)per * sms) : 1.0;
}
// 64 x 64 output tiles for an M x N product batch, unless 32 x 32 tiles fill the SMs markedly
// better (many small products: 512 products of 64 x 64 are 512 CTAs, 3.4 per SM, so a quarter
// of the SMs hold one more than the rest and set the time; 2048 CTAs of 32 x 32 spread to
// within one small CTA)
inline bool prefer_tiles_64(int M, int N, int batch) {
  const int sms = sm_count();
  const long long c64 = (long long)((N + 63) / 64) * ((M + 63) / 64) * batch;
  const long long c32 = (long long)((N + 31) / 32) * ((M + 31) / 32) * batch;
  return sm_fill(c32, sms) < sm_fill(c64, sms) + 0.05;
}
// Prefer the largest shared-memory carveout for a kernel (once per device), so that several
// of its CTAs fit on an SM.
void prefer_max_shared_carveout(const void* func);
void init_fields(int8_t* s, int n_chains, int L, int N, uint32_t k0, uint32_t k1,
                 long long chain_offset, cudaStream_t st);
// Philox initial fields (tag 1) of the listed chains only: chain list[j] gets global index
// ids[j] (both device arrays of n entries).
void init_fields_list(int8_t* s, int L, int N, uint32_t k0, uint32_t k1, const int* list,
                      const long long* ids, int n, cudaStream_t st);
// Start the listed chains afresh: chain_id = ids, sweep_base = sweep, sign = +1, counts and
// drift cleared (device arrays of n entries; sign/counts/drift indexed by chain).
void restart_chain_state(const int* list, const long long* ids, int n, int n_chains, long long sweep,
                         long long* chain_id, long long* sweep_base, double* sign,
                         unsigned long long* counts, unsigned long long* drift,
                         cudaStream_t st);
// chain_id[c] = offset + c, sweep_base[c] = 0 for every chain.
void default_chain_ids(long long* chain_id, long long* sweep_base, int n_chains,
                       long long offset, cudaStream_t st);
void set_identity_batch(double* U, double* D, double* T, int N, int batch, cudaStream_t st);
void copy_to_float(const double* x, float* y, long long n, cudaStream_t st);
void copy_to_double(const float* x, double* y, long long n, cudaStream_t st);
void fields_normalize(int8_t* s, long long n, cudaStream_t st);
void philox_batch(const uint32_t* c0, int n, uint32_t c1, uint32_t c2, uint32_t c3,
                  uint32_t k0, uint32_t k1, uint32_t* out, cudaStream_t st);

// Per-stabilization drift (bits of non-negative doubles): fold into the per-chain maximum,
// write the maximum over chains to hist[*hist_idx] while *hist_idx < hist_cap, then advance
// *hist_idx (a device counter, so the launch does not depend on host state).
void fold_drift(const unsigned long long* stab, unsigned long long* cumulative,
                unsigned long long* hist, long long hist_cap, long long* hist_idx, int n_chains,
                cudaStream_t st);
// End of a sweep: ctr[0] (sweep counter) += 1, ctr[1] (measured sweeps) += meas.
void advance_counters(long long* ctr, int meas, cudaStream_t st);

// Measurement on Gt = e^{dtau K/2} G e^{-dtau K/2}: adds per-chain sums of
// (energy, ekin, double_occ, s_pipi, density) * sign and sign into acc[chain][8].
constexpr int kNumObs = 6;   // energy, ekin, docc, s_pipi, density, sign
// ns = 1: only G~up is given and G~dn = I - P G~up^T P (particle-hole symmetry).
// series_idx (device, may be null): accumulate into acc + (*series_idx) * n_chains * 8.
void measure(const double* Gt, const double* K, const double* sign, int N, int Lx, int lattice,
             double U, double* acc, int n_chains, int ns, cudaStream_t st,
             const long long* series_idx = nullptr);

}  // namespace nmc
