// FP64 numerical stabilization of the DQMC sweep: UDV (here U D T) decompositions of the
// B-matrix products and the stable recompute of G = (I + R L)^{-1}.
//
// k_qrp: Householder QR with column pivoting (Businger-Golub): at step p the remaining
//   column of largest norm (lowest index on ties) is swapped into place, a reflector
//   H_p = I - tau v v^T (v_p = 1) zeroes it below the diagonal, and the trailing columns
//   are updated; squared column norms are downdated with the usual safeguard (recomputed
//   when the downdated value has lost more than half its digits). Outputs U = Q (formed in
//   place by backward accumulation of the reflectors), D = |diag R| and T = D^{-1} R P^T.
// k_solve: Y = X^{-1} (Db_R^{-1} U_R^T) by Gauss-Jordan elimination with partial pivoting
//   on the augmented matrix [X | RHS]; X is the well-scaled middle factor of the
//   stabilized inverse, so partial pivoting is sufficient.
//
// One CTA per matrix (batch = 2 * chains); the working matrix lives in shared memory
// when it fits and in a per-matrix global workspace otherwise.
#include <cfloat>

#include "nmc_internal.cuh"

namespace nmc {

namespace {

NMC_DEBUG_FLAG

constexpr int kThreads = 256;
// Gauss-Jordan: 16 warps (rows over warps, columns over lanes), so a matrix alone on an SM
// (the tail of a batch that does not fill the GPU in one wave) still has the warps to hide
// the FP64 latency
constexpr int kSolveThreads = 512;
constexpr int kSolveWarps = kSolveThreads / 32;
constexpr size_t kSmemLimit = 200 * 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// argmax over lanes: larger key wins, lower index on ties. Keys are the bit patterns of
// non-negative doubles (|x|, squared norms), which order like the values, so the search
// runs on the integer pipes instead of the narrow FP64 pipe; a lane with no candidate
// holds key -1.
__device__ __forceinline__ void warp_argmax(long long& key, int& idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ok = __shfl_xor_sync(0xffffffffu, key, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ok > key || (ok == key && oi < idx)) { key = ok; idx = oi; }
  }
}

// key of a non-negative double (a NaN, with its sign bit cleared, orders above +inf)
__device__ __forceinline__ long long nonneg_key(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffll;
}

__host__ __device__ inline size_t qrp_small_bytes(int N) {
  return (size_t)N * (3 * sizeof(double) + sizeof(int)) + 64;
}

// Four threads per column (a "quad", lanes 4q..4q+3 of a warp) for the trailing updates:
// one warp covers 8 columns, so per-column scalar work costs one warp instruction per
// 8 columns. Column norms are kept squared (n1 = current, n2 = at last recompute); the
// LAPACK downdate safeguard "1 - (r/n1)^2 scaled by (n1/n2)^2 <= sqrt(eps)" is the same test
// as n1^2 - r^2 <= sqrt(eps) n2^2, which needs no division or square root.
constexpr int kQuad = 4;
constexpr int kColsPerPass = kThreads / kQuad;

__device__ __forceinline__ double quad_sum(double v, unsigned mask) {
  v += __shfl_xor_sync(mask, v, 1);
  v += __shfl_xor_sync(mask, v, 2);
  return v;
}

__global__ void __launch_bounds__(kThreads)
k_qrp(const double* __restrict__ X, double* __restrict__ U, double* __restrict__ D,
      double* __restrict__ Tp, double* __restrict__ ws, int N, int use_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int b = blockIdx.x;
  const long long NN = (long long)N * N;
  double* n1 = (double*)smraw;   // squared norms
  double* n2 = n1 + N;
  double* tau = n2 + N;
  int* perm = (int*)(tau + N);
  // column-major with leading dimension N + 1 (W[c*ldw + r]): the 32 columns of a warp fall
  // on different banks when each thread walks its own column; W becomes Q at the end
  const int ldw = N + 1;
  double* W;
  if (use_smem)
    W = (double*)(smraw + ((qrp_small_bytes(N) + 15) & ~(size_t)15));
  else
    W = ws + (long long)b * 2 * NN;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int pw = blockIdx.x & 3;
  const int sub = tid & (kQuad - 1);
  const unsigned qmask = 0xFu << (lane & ~(kQuad - 1));
  const double* Xb = X + (long long)b * NN;

  for (int e = tid; e < (int)NN; e += kThreads) {
    const int r = e / N, c = e - r * N;
    W[(long long)c * ldw + r] = Xb[e];
  }
  for (int c = tid; c < N; c += kThreads) perm[c] = c;
  __syncthreads();
  for (int c0 = 0; c0 < N; c0 += kColsPerPass) {
    const int c = c0 + tid / kQuad;
    if (c < N) {
      double s = 0.0;
      for (int r = sub; r < N; r += kQuad) { const double v = W[(long long)c * ldw + r]; s += v * v; }
      s = quad_sum(s, qmask);
      if (sub == 0) { n1[c] = s; n2[c] = s; }
    }
  }
  __syncthreads();

  const double tol3z = sqrt(DBL_EPSILON);
  for (int p = 0; p < N; ++p) {
    // warp pw: pivot (largest remaining norm, lowest index on ties), swap, reflector
    // H_p = I - tau v v^T (v_p = 1) zeroing W[p+1:, p]; the other warps wait at the barrier.
    // pw = blockIdx % 4: the CTAs sharing an SM run this serial FP64 step on different
    // sub-partitions (warp w issues on sub-partition w % 4) instead of all on the first.
    if (warp == pw) {
      long long best = -1;
      int bi = p;
      for (int c = p + lane; c < N; c += 32) {
        const long long kc = nonneg_key(n1[c]);
        if (kc > best) { best = kc; bi = c; }
      }
      warp_argmax(best, bi);
      const int piv = NMC_DCHECK(bi >= p && bi < N, 201) ? bi : p;
      if (piv != p) {
        for (int r = lane; r < N; r += 32) {
          const double t0 = W[(long long)p * ldw + r];
          W[(long long)p * ldw + r] = W[(long long)piv * ldw + r];
          W[(long long)piv * ldw + r] = t0;
        }
        if (lane == 0) {
          double t1 = n1[p]; n1[p] = n1[piv]; n1[piv] = t1;
          t1 = n2[p]; n2[p] = n2[piv]; n2[piv] = t1;
          const int ti = perm[p]; perm[p] = perm[piv]; perm[piv] = ti;
        }
      }
      __syncwarp();
      double* col = W + (long long)p * ldw;
      const double alpha = col[p];
      double xn2 = 0.0;
      for (int r = p + 1 + lane; r < N; r += 32) xn2 += col[r] * col[r];
      xn2 = warp_sum(xn2);
      double t = 0.0;
      if (xn2 > 0.0) {   // (xn2 is the same in every lane after the butterfly sum)
        // the square root and the two divisions on lane 0 only, then broadcast
        double beta = 0.0, scal = 0.0;
        if (lane == 0) {
          beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
          t = (beta - alpha) / beta;
          scal = 1.0 / (alpha - beta);
        }
        scal = __shfl_sync(0xffffffffu, scal, 0);
        for (int r = p + 1 + lane; r < N; r += 32) col[r] *= scal;
        __syncwarp();
        if (lane == 0) col[p] = beta;
      }
      if (lane == 0) tau[p] = t;
    }
    __syncthreads();
    const double tp = tau[p];
    const double* v = W + (long long)p * ldw;
    // one thread per trailing column: each FP64 warp instruction then carries 32 columns'
    // work, with no partial sums to combine (the FP64 pipe costs the same per warp
    // instruction however many lanes are active)
    for (int c = p + 1 + tid; c < N; c += kThreads) {
      double* col = W + (long long)c * ldw;
      double rp = col[p];
      if (tp != 0.0) {
        double dot = rp;   // v_p = 1
        for (int r = p + 1; r < N; ++r) dot = fma(v[r], col[r], dot);
        const double f = tp * dot;
        for (int r = p + 1; r < N; ++r) col[r] = fma(-f, v[r], col[r]);
        rp -= f;
        col[p] = rp;
      }
      const double a1 = n1[c];
      if (a1 != 0.0) {
        const double d = fma(-rp, rp, a1);
        if (d <= tol3z * n2[c]) {
          double s = 0.0;
          for (int r = p + 1; r < N; ++r) s = fma(col[r], col[r], s);
          n1[c] = s;
          n2[c] = s;
        } else {
          n1[c] = d;
        }
      }
    }
    __syncthreads();
  }

  // outputs D and T = D^{-1} R P^T
  double* Db = D + (long long)b * N;
  for (int r = tid; r < N; r += kThreads) Db[r] = fabs(W[(long long)r * ldw + r]);
  double* Tb = Tp + (long long)b * NN;
  for (int e = tid; e < (int)NN; e += kThreads) {
    const int r = e / N, c = e - r * N;
    const double d = fabs(W[(long long)r * ldw + r]);
    Tb[r * N + perm[c]] = (c >= r) ? W[(long long)c * ldw + r] / d : 0.0;
  }
  __syncthreads();   // T and D are out: W's upper triangle is free
  // Q = H_0 H_1 ... H_{N-1} in place over W (column-major), by backward accumulation:
  // before step p, columns > p hold H_{p+1} ... H_{N-1} in rows > p (rows <= p still hold R
  // and are treated as zero); step p applies H_p to those columns, writing their row p, and
  // then turns column p (the reflector v, v_p = 1) into H_p e_p.
  for (int p = N - 1; p >= 0; --p) {
    const double tp = tau[p];
    const double* v = W + (long long)p * ldw;
    for (int c = p + 1 + tid; c < N; c += kThreads) {   // one thread per column, as above
      double* col = W + (long long)c * ldw;
      double dot = 0.0;
      for (int r = p + 1; r < N; ++r) dot = fma(v[r], col[r], dot);
      const double f = tp * dot;
      if (f != 0.0)
        for (int r = p + 1; r < N; ++r) col[r] = fma(-f, v[r], col[r]);
      col[p] = -f;
    }
    __syncthreads();
    double* cp = W + (long long)p * ldw;
    for (int r = tid; r < N; r += kThreads)
      cp[r] = r < p ? 0.0 : r == p ? 1.0 - tp : -tp * cp[r];
    __syncthreads();
  }
  double* Q = W;
  double* Ub = U + (long long)b * NN;
  for (int e = tid; e < (int)NN; e += kThreads) {
    const int r = e / N, c = e - r * N;
    Ub[e] = Q[(long long)c * ldw + r];
  }
}

__global__ void __launch_bounds__(kSolveThreads)
k_solve(const double* __restrict__ X, const double* __restrict__ UR, long long sUR,
        const double* __restrict__ DR, long long sDR, double* __restrict__ Y,
        double* __restrict__ ws, int N, int use_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_piv;
  __shared__ double s_inv;
  const int b = blockIdx.x;
  const long long NN = (long long)N * N;
  const int ld = 2 * N;
  double* Aug = use_smem ? (double*)smraw : ws + (long long)b * 2 * NN;  // row-major N x 2N
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* Xb = X + (long long)b * NN;
  const double* Ub = UR + (long long)b * sUR;
  const double* Dv = DR + (long long)b * sDR;
  for (int e = tid; e < 2 * (int)NN; e += kSolveThreads) {
    const int r = e / ld, c = e - r * ld;
    double v;
    if (c < N) v = Xb[r * N + c];
    else v = Ub[(c - N) * N + r] / fmax(Dv[r], 1.0);  // (Db_R^{-1} U_R^T)[r][c-N]
    Aug[e] = v;
  }
  __syncthreads();
  const int pw = blockIdx.x & 3;   // the pivot-search warp (see k_qrp)
  for (int p = 0; p < N; ++p) {
    if (warp == pw) {
      long long best = -1;
      int bi = p;
      for (int r = p + lane; r < N; r += 32) {
        const long long kr = nonneg_key(Aug[(long long)r * ld + p]);   // |entry|
        if (kr > best) { best = kr; bi = r; }
      }
      warp_argmax(best, bi);
      // the pivot's reciprocal, once: a division on every warp would cost the narrow FP64
      // pipe about as much as the elimination step itself
      if (lane == 0) {
        if (!NMC_DCHECK(bi >= p && bi < N, 202)) bi = p;
        s_piv = bi;
        s_inv = 1.0 / Aug[(long long)bi * ld + p];
      }
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != p) {
      for (int c = p + tid; c < ld; c += kSolveThreads) {
        const double t = Aug[(long long)p * ld + c];
        Aug[(long long)p * ld + c] = Aug[(long long)piv * ld + c];
        Aug[(long long)piv * ld + c] = t;
      }
      __syncthreads();
    }
    const double inv = s_inv;
    for (int c = p + 1 + tid; c < ld; c += kSolveThreads) Aug[p * ld + c] *= inv;
    __syncthreads();
    // rows over warps, columns over lanes (32-bit indices)
    for (int r = warp; r < N; r += kSolveWarps) {
      if (r == p) continue;
      const double mlt = Aug[r * ld + p];
      for (int c = p + 1 + lane; c < ld; c += 32) Aug[r * ld + c] -= mlt * Aug[p * ld + c];
    }
    __syncthreads();
  }
  double* Yb = Y + (long long)b * NN;
  for (int e = tid; e < (int)NN; e += kSolveThreads) {
    const int r = e / N, c = e - r * N;
    Yb[e] = Aug[r * ld + N + c];
  }
}

}  // namespace

void qrp_udt(const double* X, double* U, double* D, double* Tp, double* ws, int N, int batch,
             cudaStream_t st) {
  const size_t small = (qrp_small_bytes(N) + 15) & ~(size_t)15;
  const size_t big = small + (size_t)N * (N + 1) * sizeof(double);   // W, ld N + 1
  const int use_smem = big <= kSmemLimit;
  const size_t bytes = use_smem ? big : small;
  allow_max_dynamic_smem((const void*)k_qrp);
  k_qrp<<<batch, kThreads, bytes, st>>>(X, U, D, Tp, ws, N, use_smem);
}

void solve_stab(const double* X, const double* UR, long long sUR, const double* DR,
                long long sDR, double* Y, double* ws, int N, int batch, cudaStream_t st) {
  const size_t big = 2 * (size_t)N * N * sizeof(double);
  const int use_smem = big <= kSmemLimit;
  const size_t bytes = use_smem ? big : 0;
  allow_max_dynamic_smem((const void*)k_solve);
  k_solve<<<batch, kSolveThreads, bytes, st>>>(X, UR, sUR, DR, sDR, Y, ws, N, use_smem);
}

bool stab_needs_workspace(int N) {
  const size_t small = (qrp_small_bytes(N) + 15) & ~(size_t)15;
  return small + 2 * (size_t)N * N * sizeof(double) > kSmemLimit;
}

NMC_DEBUG_READER(debug_fail_stab)

}  // namespace nmc
