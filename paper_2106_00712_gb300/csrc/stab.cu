// FP64 numerical stabilization of the DQMC sweep: UDV (here U D T) decompositions of the
// B-matrix products and the stable recompute of G = (I + R L)^{-1}.
//
// k_qrp: Householder QR with column pivoting (Businger-Golub): at step p the remaining
//   column of largest norm (lowest index on ties) is swapped into place, a reflector
//   H_p = I - tau v v^T (v_p = 1) zeroes it below the diagonal, and the trailing columns
//   are updated; column norms are downdated with the usual safeguard (recomputed when
//   the downdated value has lost more than half its digits). Outputs U = Q (formed by
//   backward accumulation of the reflectors), D = |diag R| and T = D^{-1} R P^T.
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

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr size_t kSmemLimit = 200 * 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// argmax over lanes: larger value wins, lower index on ties
__device__ __forceinline__ void warp_argmax(double& v, int& idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
}

__host__ __device__ inline size_t qrp_small_bytes(int N) { return (size_t)N * (3 * sizeof(double) + sizeof(int)) + 64; }

__global__ void __launch_bounds__(kThreads)
k_qrp(const double* __restrict__ X, double* __restrict__ U, double* __restrict__ D,
      double* __restrict__ Tp, double* __restrict__ ws, int N, int use_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int b = blockIdx.x;
  const long long NN = (long long)N * N;
  double* vn1 = (double*)smraw;
  double* vn2 = vn1 + N;
  double* tau = vn2 + N;
  int* perm = (int*)(tau + N);
  __shared__ int s_piv;
  double* W;  // column-major: W[c*N + r]
  double* Q;  // column-major
  if (use_smem) {
    W = (double*)(smraw + ((qrp_small_bytes(N) + 15) & ~(size_t)15));
    Q = W + NN;
  } else {
    W = ws + (long long)b * 2 * NN;
    Q = W + NN;
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* Xb = X + (long long)b * NN;

  for (long long e = tid; e < NN; e += kThreads) {
    const int r = (int)(e / N), c = (int)(e % N);
    W[(long long)c * N + r] = Xb[e];
  }
  for (int c = tid; c < N; c += kThreads) perm[c] = c;
  __syncthreads();
  for (int c = warp; c < N; c += kWarps) {
    double s = 0.0;
    for (int r = lane; r < N; r += 32) { const double v = W[(long long)c * N + r]; s += v * v; }
    s = warp_sum(s);
    if (lane == 0) { vn1[c] = sqrt(s); vn2[c] = vn1[c]; }
  }
  __syncthreads();

  const double tol3z = sqrt(DBL_EPSILON);
  for (int p = 0; p < N; ++p) {
    if (warp == 0) {
      double best = -1.0;
      int bi = N;
      for (int c = p + lane; c < N; c += 32)
        if (vn1[c] > best) { best = vn1[c]; bi = c; }
      warp_argmax(best, bi);
      if (lane == 0) s_piv = bi;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != p) {
      for (int r = tid; r < N; r += kThreads) {
        const double t0 = W[(long long)p * N + r];
        W[(long long)p * N + r] = W[(long long)piv * N + r];
        W[(long long)piv * N + r] = t0;
      }
      if (tid == 0) {
        double t1 = vn1[p]; vn1[p] = vn1[piv]; vn1[piv] = t1;
        t1 = vn2[p]; vn2[p] = vn2[piv]; vn2[piv] = t1;
        const int ti = perm[p]; perm[p] = perm[piv]; perm[piv] = ti;
      }
    }
    __syncthreads();
    if (warp == 0) {
      double* col = W + (long long)p * N;
      const double alpha = col[p];
      double xn2 = 0.0;
      for (int r = p + 1 + lane; r < N; r += 32) xn2 += col[r] * col[r];
      xn2 = warp_sum(xn2);
      double t = 0.0;
      if (xn2 > 0.0) {
        const double beta = -copysign(sqrt(alpha * alpha + xn2), alpha);
        t = (beta - alpha) / beta;
        const double scal = 1.0 / (alpha - beta);
        for (int r = p + 1 + lane; r < N; r += 32) col[r] *= scal;
        __syncwarp();
        if (lane == 0) col[p] = beta;
      }
      if (lane == 0) tau[p] = t;
    }
    __syncthreads();
    const double tp = tau[p];
    const double* v = W + (long long)p * N;
    for (int c = p + 1 + warp; c < N; c += kWarps) {
      double* col = W + (long long)c * N;
      if (tp != 0.0) {
        double dot = 0.0;
        for (int r = p + 1 + lane; r < N; r += 32) dot += v[r] * col[r];
        dot = warp_sum(dot) + col[p];
        const double f = tp * dot;
        for (int r = p + 1 + lane; r < N; r += 32) col[r] -= f * v[r];
        __syncwarp();
        if (lane == 0) col[p] -= f;
        __syncwarp();
      }
      const double n1 = vn1[c];
      if (n1 != 0.0) {
        double temp = fabs(col[p]) / n1;
        temp = fmax(0.0, 1.0 - temp * temp);
        const double r12 = n1 / vn2[c];
        const double temp2 = temp * r12 * r12;
        double nv;
        if (temp2 <= tol3z) {
          double s = 0.0;
          for (int r = p + 1 + lane; r < N; r += 32) s += col[r] * col[r];
          s = warp_sum(s);
          nv = sqrt(s);
          if (lane == 0) { vn1[c] = nv; vn2[c] = nv; }
        } else if (lane == 0) {
          vn1[c] = n1 * sqrt(temp);
        }
      }
      __syncwarp();
    }
    __syncthreads();
  }

  // outputs D and T = D^{-1} R P^T
  double* Db = D + (long long)b * N;
  for (int r = tid; r < N; r += kThreads) Db[r] = fabs(W[(long long)r * N + r]);
  double* Tb = Tp + (long long)b * NN;
  for (long long e = tid; e < NN; e += kThreads) {
    const int r = (int)(e / N), c = (int)(e % N);
    const double d = fabs(W[(long long)r * N + r]);
    Tb[(long long)r * N + perm[c]] = (c >= r) ? W[(long long)c * N + r] / d : 0.0;
  }
  // Q = H_0 H_1 ... H_{N-1} by backward accumulation (column-major)
  for (long long e = tid; e < NN; e += kThreads) {
    const int c = (int)(e / N), r = (int)(e % N);
    Q[e] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int p = N - 1; p >= 0; --p) {
    const double tp = tau[p];
    if (tp != 0.0) {
      const double* v = W + (long long)p * N;
      for (int c = p + warp; c < N; c += kWarps) {
        double* col = Q + (long long)c * N;
        double dot = 0.0;
        for (int r = p + 1 + lane; r < N; r += 32) dot += v[r] * col[r];
        dot = warp_sum(dot) + col[p];
        const double f = tp * dot;
        for (int r = p + 1 + lane; r < N; r += 32) col[r] -= f * v[r];
        __syncwarp();
        if (lane == 0) col[p] -= f;
        __syncwarp();
      }
    }
    __syncthreads();
  }
  double* Ub = U + (long long)b * NN;
  for (long long e = tid; e < NN; e += kThreads) {
    const int r = (int)(e / N), c = (int)(e % N);
    Ub[e] = Q[(long long)c * N + r];
  }
}

__global__ void __launch_bounds__(kThreads)
k_solve(const double* __restrict__ X, const double* __restrict__ UR, long long sUR,
        const double* __restrict__ DR, long long sDR, double* __restrict__ Y,
        double* __restrict__ ws, int N, int use_smem) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_piv;
  const int b = blockIdx.x;
  const long long NN = (long long)N * N;
  const int ld = 2 * N;
  double* Aug = use_smem ? (double*)smraw : ws + (long long)b * 2 * NN;  // row-major N x 2N
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* Xb = X + (long long)b * NN;
  const double* Ub = UR + (long long)b * sUR;
  const double* Dv = DR + (long long)b * sDR;
  for (long long e = tid; e < 2 * NN; e += kThreads) {
    const int r = (int)(e / ld), c = (int)(e % ld);
    double v;
    if (c < N) v = Xb[(long long)r * N + c];
    else v = Ub[(long long)(c - N) * N + r] / fmax(Dv[r], 1.0);  // (Db_R^{-1} U_R^T)[r][c-N]
    Aug[e] = v;
  }
  __syncthreads();
  for (int p = 0; p < N; ++p) {
    if (warp == 0) {
      double best = -1.0;
      int bi = N;
      for (int r = p + lane; r < N; r += 32) {
        const double a = fabs(Aug[(long long)r * ld + p]);
        if (a > best) { best = a; bi = r; }
      }
      warp_argmax(best, bi);
      if (lane == 0) s_piv = bi;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != p) {
      for (int c = p + tid; c < ld; c += kThreads) {
        const double t = Aug[(long long)p * ld + c];
        Aug[(long long)p * ld + c] = Aug[(long long)piv * ld + c];
        Aug[(long long)piv * ld + c] = t;
      }
      __syncthreads();
    }
    const double inv = 1.0 / Aug[(long long)p * ld + p];
    for (int c = p + 1 + tid; c < ld; c += kThreads) Aug[(long long)p * ld + c] *= inv;
    __syncthreads();
    const int width = ld - p - 1;
    for (long long e = tid; e < (long long)N * width; e += kThreads) {
      const int r = (int)(e / width);
      if (r == p) continue;
      const int c = p + 1 + (int)(e % width);
      Aug[(long long)r * ld + c] -= Aug[(long long)r * ld + p] * Aug[(long long)p * ld + c];
    }
    __syncthreads();
  }
  double* Yb = Y + (long long)b * NN;
  for (long long e = tid; e < NN; e += kThreads) {
    const int r = (int)(e / N), c = (int)(e % N);
    Yb[e] = Aug[(long long)r * ld + N + c];
  }
}

}  // namespace

void qrp_udt(const double* X, double* U, double* D, double* Tp, double* ws, int N, int batch,
             cudaStream_t st) {
  const size_t small = (qrp_small_bytes(N) + 15) & ~(size_t)15;
  const size_t big = small + 2 * (size_t)N * N * sizeof(double);
  const int use_smem = big <= kSmemLimit;
  const size_t bytes = use_smem ? big : small;
  cudaFuncSetAttribute(k_qrp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  k_qrp<<<batch, kThreads, bytes, st>>>(X, U, D, Tp, ws, N, use_smem);
}

void solve_stab(const double* X, const double* UR, long long sUR, const double* DR,
                long long sDR, double* Y, double* ws, int N, int batch, cudaStream_t st) {
  const size_t big = 2 * (size_t)N * N * sizeof(double);
  const int use_smem = big <= kSmemLimit;
  const size_t bytes = use_smem ? big : 0;
  if (use_smem)
    cudaFuncSetAttribute(k_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  k_solve<<<batch, kThreads, bytes, st>>>(X, UR, sUR, DR, sDR, Y, ws, N, use_smem);
}

bool stab_needs_workspace(int N) {
  const size_t small = (qrp_small_bytes(N) + 15) & ~(size_t)15;
  return small + 2 * (size_t)N * N * sizeof(double) > kSmemLimit;
}

}  // namespace nmc
