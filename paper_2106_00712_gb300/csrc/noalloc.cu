// nmc_green_noalloc: equal-time Green's functions from caller-given fields, with every
// temporary in a fixed device array compiled into the library -- no cudaMalloc/cudaFree.
//
// Some callers cannot allocate device memory at the point where they need G: code running
// under a memory pool or arena that owns the whole device budget, an embedding runtime
// that forbids allocator calls after start-up, or a caller between two phases of its own
// work that must not perturb the allocator. This entry point serves them: the caller
// passes inputs and outputs, and the scratch comes from `g_scratch` below.
//
// It computes what nmc_set_fields computes for G (left UDV stack over all blocks, then the
// stabilized G_0 = (I + B_{L-1}...B_0)^{-1} per chain and spin) with the same kernels in the
// same order, so for the same inputs it returns the same values.
#include <cmath>
#include <mutex>

#include "../../include/nmc.h"
#include "nmc_internal.cuh"

namespace nmc {
bool stab_needs_workspace(int N);
}

using namespace nmc;

namespace {

// 4,194,304 doubles (32 MiB), held by every GPU that loads the library until exit.
constexpr size_t kScratchDoubles = (size_t)4 << 20;
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch in the current device's context. In host code the symbol name
// is only a host-side stand-in, never a usable device address. The address belongs to the
// context that loaded the library's module: a device reset (cudaDeviceReset) or another
// context on the same device loads it again, possibly elsewhere. So every call made outside
// stream capture looks the address up again (cheap once the module is loaded) and caches
// it per device; a call made while `st` is being captured uses the cached address, which a
// call outside capture must have set after the last reset.
cudaError_t scratch_on_current_device(cudaStream_t st, double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = (double*)p;
  } else if (!g_scratch_addr[dev]) {
    return cudaErrorStreamCaptureUnsupported;  // no address looked up outside capture yet
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t round256(size_t doubles) { return (doubles + 31) & ~(size_t)31; }

struct View {
  const double* U; long long sU;
  const double* D; long long sD;
  const double* T; long long sT;
};

GemmArgs<double> base(int N, int batch, const double* A, long long sA, const double* B,
                      long long sB, double* C) {
  GemmArgs<double> g;
  g.M = g.N = g.K = N;
  g.batch = batch;
  g.A = A; g.sA = sA; g.lda = N;
  g.B = B; g.sB = sB; g.ldb = N;
  g.C = C; g.sC = (long long)N * N; g.ldc = N;
  return g;
}

ScaleDesc fscale(const int8_t* fields, int l, int N, int L, double lam) {
  ScaleDesc d;
  d.kind = SC_FIELD;
  d.fields = fields + (long long)l * N;
  d.fstride = (long long)L * N;
  d.e_lam = std::exp(lam);
  d.e_mlam = std::exp(-lam);
  return d;
}

ScaleDesc vscale(const double* v, long long stride, int kind) {
  ScaleDesc d;
  d.kind = kind;
  d.vec = v;
  d.vstride = stride;
  return d;
}

}  // namespace

extern "C" nmc_status nmc_green_noalloc(int N, int L_tau, int n_wrap, double lam,
                                        const double* d_expK_m, const int8_t* d_fields,
                                        int n_chains, double* d_G, void* cuda_stream) {
  if (N < 2 || N > 1024 || L_tau < 1 || n_wrap < 1 || L_tau % n_wrap || n_chains < 1 ||
      !(lam >= 0.0) || !std::isfinite(lam) || !d_expK_m || !d_fields || !d_G)
    return NMC_EINVAL;
  const long long NN = (long long)N * N;
  const bool ws_needed = stab_needs_workspace(N);
  // per chain (2 matrices): X, X2, Tp, U x2, T x2, M1, Xs, Y (10 N^2), D x2 (2 N), and the
  // QR / solve workspace (2 N^2) when a matrix does not fit in shared memory.
  const size_t per_chain = 2 * (10 * (size_t)NN + 2 * (size_t)N + (ws_needed ? 2 * (size_t)NN : 0));
  const size_t shared = round256(NN) + round256(N) + 16 * 32;  // I, ones, alignment slack
  if (shared + per_chain > kScratchDoubles) return NMC_EINVAL;  // one chain does not fit
  const int chunk = (int)((kScratchDoubles - shared) / per_chain);

  // An error left pending by earlier work (not ours) is reported, not consumed.
  if (cudaPeekAtLastError() != cudaSuccess) return NMC_ECUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* base_ptr = nullptr;
  if (scratch_on_current_device(st, &base_ptr) != cudaSuccess) return NMC_ECUDA;
  const int nb = L_tau / n_wrap;

  double* I = base_ptr;
  double* ones = I + round256(NN);
  double* p = ones + round256(N);
  set_identity_batch(I, ones, nullptr, N, 1, st);

  for (int c0 = 0; c0 < n_chains; c0 += chunk) {
    const int cc = (n_chains - c0 < chunk) ? n_chains - c0 : chunk;
    const int B = 2 * cc;
    const size_t m = round256((size_t)NN * B);  // one batch of matrices, stride N^2
    const size_t v = round256((size_t)N * B);   // one batch of vectors, stride N
    double* q = p;
    double* X = q; q += m;
    double* X2 = q; q += m;
    double* Tp = q; q += m;
    double* Ub[2] = {q, q + m}; q += 2 * m;
    double* Tb[2] = {q, q + m}; q += 2 * m;
    double* M1 = q; q += m;
    double* Xs = q; q += m;
    double* Y = q; q += m;
    double* Db[2] = {q, q + v}; q += 2 * v;
    double* ws = ws_needed ? q : nullptr;
    const int8_t* f = d_fields + (long long)c0 * L_tau * N;

    // left stack L_j, j = nb-1..0, starting from L_nb = I (identity, batch stride 0)
    View src{I, 0, ones, 0, I, 0};
    int out = 0;
    for (int j = nb - 1; j >= 0; --j) {
      const int lt = (j + 1) * n_wrap - 1;
      GemmArgs<double> g = base(N, B, d_expK_m, 0, src.U, src.sU, X);
      g.bcol = vscale(src.D, src.sD, SC_VEC);
      g.crow = fscale(f, lt, N, L_tau, lam);
      gemm(g, st);
      double* x = X;
      double* x2 = X2;
      for (int l = lt - 1; l >= j * n_wrap; --l) {
        GemmArgs<double> h = base(N, B, d_expK_m, 0, x, NN, x2);
        h.crow = fscale(f, l, N, L_tau, lam);
        gemm(h, st);
        double* t = x; x = x2; x2 = t;
      }
      qrp_udt(x, Ub[out], Db[out], Tp, ws, N, B, st);
      GemmArgs<double> gt = base(N, B, Tp, NN, src.T, src.sT, Tb[out]);
      gemm(gt, st);
      src = View{Ub[out], NN, Db[out], N, Tb[out], NN};
      out ^= 1;
    }
    // G = (I + R L_0)^{-1} with R = I
    const View R{I, 0, ones, 0, I, 0};
    GemmArgs<double> g1 = base(N, B, R.U, R.sU, src.U, src.sU, M1);
    g1.transA = 1;
    g1.crow = vscale(R.D, R.sD, SC_INV_MAX1);
    g1.ccol = vscale(src.D, src.sD, SC_INV_MAX1);
    gemm(g1, st);
    GemmArgs<double> g2 = base(N, B, R.T, R.sT, src.T, src.sT, Xs);
    g2.transB = 1;
    g2.crow = vscale(R.D, R.sD, SC_MIN1);
    g2.ccol = vscale(src.D, src.sD, SC_MIN1);
    g2.Cin = M1; g2.sCin = NN; g2.ldcin = N; g2.beta = 1.0;
    gemm(g2, st);
    solve_stab(Xs, R.U, R.sU, R.D, R.sD, Y, ws, N, B, st);
    GemmArgs<double> g3 = base(N, B, src.U, src.sU, Y, NN, d_G + (long long)c0 * 2 * NN);
    g3.brow = vscale(src.D, src.sD, SC_INV_MAX1);
    gemm(g3, st);
    // stop at the first failed launch instead of queueing later chunks behind it
    if (cudaGetLastError() != cudaSuccess) return NMC_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? NMC_OK : NMC_ECUDA;
}
