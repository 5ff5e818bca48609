// libnmc C ABI (include/nmc.h): context, device memory, and the sweep schedule.
//
// Schedule of one sweep over all chains (every step a batched kernel over chains x spins):
//  up sweep (even phase), blocks j = 0..nb-1 of n_wrap slices:
//    for l in block: flip slice l (k_flip), wrap G <- B_l G B_l^{-1}
//    right stack R_{j+1} = B_block R_j (n_wrap GEMMs, column-pivoted QR, T <- T' T)
//    recompute G = (I + R_{j+1} L_{j+1})^{-1} in FP64, record drift, replace G; measure
//  down sweep (odd phase), blocks j = nb-1..0:
//    for l in block, descending: wrap G <- B_l^{-1} G B_l, flip slice l
//    left stack L_j = L_{j+1} B_block (held as L^T = U D T), recompute (I + R_j L_j)^{-1}
// Stack slots 1..nb-1 hold R_j or L_j; slot 0 (R_0) and slot nb (L_nb) are the identity.
// A sweep ends with an update of three device counters (Philox sweep counter, measurement
// slot, drift-history slot) that the kernels read, so a sweep of each direction can be
// recorded once as a CUDA graph and replayed (sweep_graph).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/nmc.h"
#include "../../include/nmc_gen.h"
#include "nmc_internal.cuh"

// nimc.cu: Bernoulli fields from a generator (stream 1, samples n0..n0+n-1), synchronised
nmc_status nmc_gen_fill_fields(nmc_gen* g, int N, int Lt, long long n0, int n, int8_t* d_fields,
                               cudaStream_t st);

namespace nmc_host {
void hopping(int lattice, int Lx, int Ly, double t, std::vector<double>& K);
void jacobi_eigh(int n, std::vector<double>& A, std::vector<double>& w, std::vector<double>& V);
void expk_from_eig(int n, const std::vector<double>& w, const std::vector<double>& V, double c,
                   std::vector<double>& out);
}  // namespace nmc_host

namespace nmc {
bool stab_needs_workspace(int N);
}

using namespace nmc;

namespace {

struct UDTBuf {
  double* U = nullptr;
  double* D = nullptr;
  double* T = nullptr;
};

// A view of a batch of U D T factors (stride 0 = one shared matrix, e.g. the identity).
struct UDTView {
  const double* U;
  long long sU;
  const double* D;
  long long sD;
  const double* T;
  long long sT;
};

constexpr uint64_t kCkptMagic = 0x4e4d43434b505432ull;  // "NMCCKPT2"
constexpr int kNumClasses = 16;   // capacity of the per-class counters (>= KC_COUNT)

// One sweep direction (and measuring or not) recorded as a CUDA graph. The recorded launches
// name the UDV stack buffers by pointer, and a sweep permutes those buffers, so a graph is
// replayed only from the buffer arrangement it was recorded at (`ptrs`).
struct SweepGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> ptrs;
  long long launches[kNumClasses] = {};
};

}  // namespace

struct nmc_ctx {
  int lattice = NMC_SQUARE, Lx = 0, Ly = 0, N = 0, Lt = 0, w = 0, nb = 0;
  double t = 0, U = 0, beta = 0, dtau = 0, lam = 0;
  uint64_t seed = 0;
  nmc_options opt{};
  int kk = 16, g_in_smem = 0;
  int device = -1;
  bool configured = false, have_fields = false;
  bool dry = false;          // size-only allocation pass (nmc_footprint)
  size_t dry_bytes = 0;
  long long sweep_counter = 0;  // Philox counter word 1
  long long phase = 0;          // sweeps since the fields were set (parity = direction)
  std::string err;

  std::vector<double> hK, hEm, hEp, hEmh, hEph;

  // device memory
  double *dK = nullptr, *dEm = nullptr, *dEp = nullptr, *dEmh = nullptr, *dEph = nullptr;
  double *dI = nullptr, *dOnes = nullptr;
  float *dEmf = nullptr, *dEpf = nullptr;
  int8_t* dS = nullptr;
  double *dG = nullptr, *dT1 = nullptr, *dX = nullptr, *dX2 = nullptr, *dTp = nullptr;
  double *dM1 = nullptr, *dXs = nullptr, *dY = nullptr, *dWS = nullptr;
  float *dGf = nullptr, *dT1f = nullptr;
  df2 *dG2 = nullptr, *dT12 = nullptr, *dEm2 = nullptr, *dEp2 = nullptr;
  df2 *dXa = nullptr, *dXb = nullptr, *dEmh2 = nullptr, *dEph2 = nullptr;
  // tensor-core slices of e^{-dtau K}, e^{+dtau K}, e^{-dtau K/2}, e^{+dtau K/2} as A / as B
  // slices of e^{-dtau K}, e^{+dtau K}, e^{-dtau K/2}, e^{+dtau K/2} for the tcgen05 products,
  // [constant][0: on the left, 1: on the right], their exponents and TMA tensor maps
  void* dOz[4][2] = {};
  int* dOzExp[4][2] = {};
  alignas(64) unsigned char tmap[4][2][128] = {};
  bool oz = false;
  int* dErr = nullptr;   // device flag: a bounded device-side wait expired (NMC_ETIMEOUT)
  std::vector<UDTBuf> slot;  // size nb + 1; entries 1..nb-1 allocated
  UDTBuf spare;
  double* dSign = nullptr;
  unsigned long long* dCounts = nullptr;  // [chain][3]: attempts, accepts, disagreements
  unsigned long long* dDrift = nullptr;   // [chain]: bits of max drift
  unsigned long long* dDriftStab = nullptr;  // [chain]: drift of the current recompute
  unsigned long long* dHist = nullptr;    // [stabilization]: max over chains
  long long hist_cap = 0, n_hist = 0;
  double* dSeries = nullptr;              // [slot][chain][8]
  long long series_cap = 0, n_series = 0;
  uint8_t* dReplay = nullptr;
  long long* dCtr = nullptr;   // device mirrors: [0] sweep_counter, [1] n_series, [2] n_hist
  // per chain: global index (Philox word 2) and the sweep counter at its start (word 1 counts
  // sweeps since then); staging for the chain lists of nmc_restart_chains
  long long *dChainId = nullptr, *dSweepBase = nullptr, *dIds = nullptr;
  int* dList = nullptr;
  std::vector<void*> allocs;

  // sweeps replayed as CUDA graphs: [up, down][warm-up, measuring]
  SweepGraph graphs[2][2];
  bool use_graphs = true;
  bool cap = false;                    // recording: launches go to cap_stream
  cudaStream_t cap_stream = nullptr;
  int direct_since_build = 0;          // direct sweeps since the stacks were last built
  long long graphs_recorded = 0, graphs_replayed = 0;

  // per-kernel accounting: launch counts always, CUDA-event brackets when prof is set
  bool prof = false;
  long long launches[kNumClasses] = {};
  long long timed[kNumClasses] = {};
  double total_ms[kNumClasses] = {};
  struct Rec { int cls; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> event_pool;

  cudaStream_t st() const { return cap ? cap_stream : (cudaStream_t)opt.cuda_stream; }
  int chains() const { return opt.n_chains; }
  int ns() const { return opt.ph_symmetric ? 1 : 2; }
  int batch() const { return ns() * opt.n_chains; }
  long long NN() const { return (long long)N * N; }
  bool fp32() const { return opt.precision == NMC_FP32; }
  // compensated FP32-pair propagation: products on the tensor cores (SPLIT_BF16) or SIMT
  bool dfp() const { return opt.precision == NMC_SPLIT_BF16 || opt.precision == NMC_FP32X2; }
  bool tc() const { return opt.precision == NMC_SPLIT_BF16; }
};

namespace {

nmc_status fail(nmc_ctx* x, nmc_status s, const std::string& msg) {
  if (x) x->err = msg;
  return s;
}

#define NMC_CUDA(x, call)                                                                   \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail((x), NMC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
  } while (0)

#define NMC_TRY(expr)              \
  do {                             \
    nmc_status s_ = (expr);        \
    if (s_ != NMC_OK) return s_;   \
  } while (0)

enum KernelClass {
  KC_GEMM = 0, KC_FLIP, KC_QRP, KC_SOLVE, KC_MEASURE, KC_OTHER, KC_GEMM_DF, KC_GEMM_TC,
  KC_GEMM_PAIR, KC_COUNT
};
const char* const kKernelClassNames[KC_COUNT] = {"gemm", "flip", "qrp", "solve", "measure",
                                                 "other", "gemm_df", "gemm_tc", "gemm_pair"};
static_assert(KC_COUNT <= kNumClasses, "per-class counters too small");

cudaEvent_t pool_event(nmc_ctx* x) {
  if (!x->event_pool.empty()) {
    cudaEvent_t e = x->event_pool.back();
    x->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch through the accounting wrapper: count, and bracket with events when profiling.
template <class F>
void launch(nmc_ctx* x, int cls, F&& f) {
  ++x->launches[cls];
  if (!x->prof) {
    f();
    return;
  }
  cudaEvent_t a = pool_event(x), b = pool_event(x);
  cudaEventRecord(a, x->st());
  f();
  cudaEventRecord(b, x->st());
  x->recs.push_back({cls, a, b});
}

void resolve_events(nmc_ctx* x) {
  for (auto& r : x->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      x->total_ms[r.cls] += ms;
      ++x->timed[r.cls];
    }
    x->event_pool.push_back(r.a);
    x->event_pool.push_back(r.b);
  }
  x->recs.clear();
}

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the context stream):
// creating or destroying one context does not synchronise the device, so other contexts'
// work on other streams keeps running (the serving loop depends on this).
void drop_graphs(nmc_ctx* x) {
  for (auto& d : x->graphs)
    for (auto& g : d) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
      g.ptrs.clear();
    }
}

void free_all(nmc_ctx* x) {
  drop_graphs(x);
  for (void* p : x->allocs) cudaFreeAsync(p, x->st());
  x->allocs.clear();
  x->dK = x->dEm = x->dEp = x->dEmh = x->dEph = x->dI = x->dOnes = nullptr;
  x->dEmf = x->dEpf = nullptr;
  x->dS = nullptr;
  x->dG = x->dT1 = x->dX = x->dX2 = x->dTp = x->dM1 = x->dXs = x->dY = x->dWS = nullptr;
  x->dGf = x->dT1f = nullptr;
  x->dG2 = x->dT12 = x->dEm2 = x->dEp2 = x->dXa = x->dXb = x->dEmh2 = x->dEph2 = nullptr;
  for (int a = 0; a < 4; ++a)
    for (int r = 0; r < 2; ++r) x->dOz[a][r] = nullptr, x->dOzExp[a][r] = nullptr;
  x->oz = false;
  x->dErr = nullptr;
  x->slot.clear();
  x->spare = UDTBuf{};
  x->dSign = nullptr;
  x->dCounts = nullptr;
  x->dDrift = nullptr;
  x->dDriftStab = nullptr;
  x->dHist = nullptr;
  x->hist_cap = x->n_hist = 0;
  x->dSeries = nullptr;
  x->series_cap = x->n_series = 0;
  x->dReplay = nullptr;
  x->dCtr = nullptr;
  x->dChainId = x->dSweepBase = x->dIds = nullptr;
  x->dList = nullptr;
  x->configured = false;
  x->have_fields = false;
}

// Allocation-failure injection (nmc_debug_fail_alloc): the n-th device allocation from the
// moment it is armed fails as if the allocator had run out of memory; 0 = off.
std::atomic<long long> g_fail_alloc_in{0};

bool injected_alloc_failure() {
  long long n = g_fail_alloc_in.load();
  while (n > 0) {
    if (g_fail_alloc_in.compare_exchange_weak(n, n - 1)) return n == 1;
  }
  return false;
}

template <typename T>
nmc_status dalloc(nmc_ctx* x, T** p, size_t count) {
  if (x->dry) {
    x->dry_bytes += ((std::max<size_t>(count, 1) * sizeof(T) + 511) / 512) * 512;
    *p = nullptr;
    return NMC_OK;
  }
  if (injected_alloc_failure())
    return fail(x, NMC_ENOMEM, "cudaMallocAsync: out of memory (injected by nmc_debug_fail_alloc)");
  void* q = nullptr;
  const cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(count, 1) * sizeof(T), x->st());
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(x, NMC_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  }
  x->allocs.push_back(q);
  *p = (T*)q;
  return NMC_OK;
}

nmc_status alloc_all(nmc_ctx* x) {
  if (!x->dry) {
    free_all(x);
    NMC_CUDA(x, cudaGetDevice(&x->device));
  }
  const long long NN = x->NN();
  const int B = x->batch();
  const size_t mats = (size_t)B * NN;
  NMC_TRY(dalloc(x, &x->dK, NN));
  NMC_TRY(dalloc(x, &x->dEm, NN));
  NMC_TRY(dalloc(x, &x->dEp, NN));
  NMC_TRY(dalloc(x, &x->dEmh, NN));
  NMC_TRY(dalloc(x, &x->dEph, NN));
  NMC_TRY(dalloc(x, &x->dI, NN));
  NMC_TRY(dalloc(x, &x->dOnes, x->N));
  NMC_TRY(dalloc(x, &x->dS, (size_t)x->chains() * x->Lt * x->N));
  NMC_TRY(dalloc(x, &x->dG, mats));
  NMC_TRY(dalloc(x, &x->dT1, mats));
  NMC_TRY(dalloc(x, &x->dX, mats));
  NMC_TRY(dalloc(x, &x->dX2, mats));
  NMC_TRY(dalloc(x, &x->dTp, mats));
  NMC_TRY(dalloc(x, &x->dM1, mats));
  NMC_TRY(dalloc(x, &x->dXs, mats));
  NMC_TRY(dalloc(x, &x->dY, mats));
  if (stab_needs_workspace(x->N)) NMC_TRY(dalloc(x, &x->dWS, 2 * mats));
  if (x->fp32()) {
    NMC_TRY(dalloc(x, &x->dEmf, NN));
    NMC_TRY(dalloc(x, &x->dEpf, NN));
    NMC_TRY(dalloc(x, &x->dGf, mats));
    NMC_TRY(dalloc(x, &x->dT1f, mats));
  }
  if (x->dfp()) {
    NMC_TRY(dalloc(x, &x->dEm2, NN));
    NMC_TRY(dalloc(x, &x->dEp2, NN));
    NMC_TRY(dalloc(x, &x->dG2, mats));
    NMC_TRY(dalloc(x, &x->dT12, mats));
    NMC_TRY(dalloc(x, &x->dXa, mats));
    NMC_TRY(dalloc(x, &x->dXb, mats));
    NMC_TRY(dalloc(x, &x->dEmh2, NN));
    NMC_TRY(dalloc(x, &x->dEph2, NN));
    x->oz = x->tc();
    if (x->oz && !x->dry && !gemm_tc_supported(x->N))
      return fail(x, NMC_EINVAL, "NMC_SPLIT_BF16 needs N <= 320 and the TMA tensor-map encoder");
    if (x->oz)
      for (int a = 0; a < 4; ++a)
        for (int r = 0; r < 2; ++r) {
          uint16_t* p = nullptr;
          NMC_TRY(dalloc(x, &p, tc_const_elems(x->N)));
          x->dOz[a][r] = p;
          NMC_TRY(dalloc(x, &x->dOzExp[a][r], x->N));
        }
  }
  x->slot.assign(x->nb + 1, UDTBuf{});
  auto alloc_udt = [&](UDTBuf& u) -> nmc_status {
    NMC_TRY(dalloc(x, &u.U, mats));
    NMC_TRY(dalloc(x, &u.D, (size_t)B * x->N));
    NMC_TRY(dalloc(x, &u.T, mats));
    return NMC_OK;
  };
  for (int j = 1; j < x->nb; ++j) NMC_TRY(alloc_udt(x->slot[j]));
  NMC_TRY(alloc_udt(x->spare));
  NMC_TRY(dalloc(x, &x->dSign, x->chains()));
  NMC_TRY(dalloc(x, &x->dCounts, 3 * (size_t)x->chains()));
  NMC_TRY(dalloc(x, &x->dDrift, x->chains()));
  NMC_TRY(dalloc(x, &x->dDriftStab, x->chains()));
  x->hist_cap = 4096;
  NMC_TRY(dalloc(x, &x->dHist, x->hist_cap));
  NMC_TRY(dalloc(x, &x->dCtr, 3));
  NMC_TRY(dalloc(x, &x->dErr, 1));
  NMC_TRY(dalloc(x, &x->dChainId, x->chains()));
  NMC_TRY(dalloc(x, &x->dSweepBase, x->chains()));
  NMC_TRY(dalloc(x, &x->dIds, x->chains()));
  NMC_TRY(dalloc(x, &x->dList, x->chains()));
  if (x->dry) return NMC_OK;

  cudaStream_t st = x->st();
  NMC_CUDA(x, cudaMemsetAsync(x->dCtr, 0, 3 * sizeof(long long), st));
  NMC_CUDA(x, cudaMemsetAsync(x->dErr, 0, sizeof(int), st));
  const size_t mb = NN * sizeof(double);
  NMC_CUDA(x, cudaMemcpyAsync(x->dK, x->hK.data(), mb, cudaMemcpyHostToDevice, st));
  NMC_CUDA(x, cudaMemcpyAsync(x->dEm, x->hEm.data(), mb, cudaMemcpyHostToDevice, st));
  NMC_CUDA(x, cudaMemcpyAsync(x->dEp, x->hEp.data(), mb, cudaMemcpyHostToDevice, st));
  NMC_CUDA(x, cudaMemcpyAsync(x->dEmh, x->hEmh.data(), mb, cudaMemcpyHostToDevice, st));
  NMC_CUDA(x, cudaMemcpyAsync(x->dEph, x->hEph.data(), mb, cudaMemcpyHostToDevice, st));
  set_identity_batch(x->dI, x->dOnes, nullptr, x->N, 1, st);
  if (x->fp32()) {
    copy_to_float(x->dEm, x->dEmf, NN, st);
    copy_to_float(x->dEp, x->dEpf, NN, st);
  }
  if (x->dfp()) {
    split_to_df(x->dEm, x->dEm2, NN, st);
    split_to_df(x->dEp, x->dEp2, NN, st);
    split_to_df(x->dEmh, x->dEmh2, NN, st);
    split_to_df(x->dEph, x->dEph2, NN, st);
    if (x->oz) {
      const double* src[4] = {x->dEm, x->dEp, x->dEmh, x->dEph};
      for (int a = 0; a < 4; ++a)
        for (int r = 0; r < 2; ++r)
          if (!tc_prepare_const(src[a], x->N, r, x->dOz[a][r], x->dOzExp[a][r], x->tmap[a][r], st))
            return fail(x, NMC_ECUDA, "cuTensorMapEncodeTiled failed for the constant's slices");
    }
  }
  NMC_CUDA(x, cudaGetLastError());
  NMC_CUDA(x, cudaStreamSynchronize(st));
  x->configured = true;
  return NMC_OK;
}

nmc_status ensure_configured(nmc_ctx* x) {
  if (x->configured) {
    NMC_CUDA(x, cudaSetDevice(x->device));
    return NMC_OK;
  }
  return alloc_all(x);
}

void clamp_delay(nmc_ctx* x) {
  const size_t elem = x->fp32() ? sizeof(float) : sizeof(double);
  const size_t limit = 200 * 1024;
  int kk = std::max(1, std::min(x->opt.delay_k, x->N));
  const int ns = x->opt.ph_symmetric ? 1 : 2;
  x->g_in_smem = flip_smem_bytes(x->N, kk, elem, 1, ns) <= limit ? 1 : 0;
  while (kk > 1 && flip_smem_bytes(x->N, kk, elem, x->g_in_smem, ns) > limit) --kk;
  x->kk = kk;
}

// ---------------------------------------------------------------------------- GEMM helpers
ScaleDesc field_scale(const nmc_ctx* x, int l, bool inv) {
  ScaleDesc d;
  d.kind = inv ? SC_FIELD_INV : SC_FIELD;
  d.ns = x->ns();
  d.fields = x->dS + (long long)l * x->N;
  d.fstride = (long long)x->Lt * x->N;
  d.e_lam = std::exp(x->lam);
  d.e_mlam = std::exp(-x->lam);
  return d;
}

ScaleDesc vec_scale(const double* v, long long stride, int kind) {
  ScaleDesc d;
  d.kind = kind;
  d.vec = v;
  d.vstride = stride;
  return d;
}

template <typename T>
GemmArgs<T> gemm_base(const nmc_ctx* x, const T* A, long long sA, const T* B, long long sB,
                      T* C) {
  GemmArgs<T> g;
  g.M = g.N = g.K = x->N;
  g.batch = x->batch();
  g.A = A; g.sA = sA; g.lda = x->N;
  g.B = B; g.sB = sB; g.ldb = x->N;
  g.C = C; g.sC = x->NN(); g.ldc = x->N;
  g.ns = x->ns();
  return g;
}

DfGemmArgs df_base(const nmc_ctx* x, const df2* A, long long sA, const df2* B, long long sB) {
  DfGemmArgs g;
  g.M = g.N = g.K = x->N;
  g.batch = x->batch();
  g.A = A; g.sA = sA; g.lda = x->N;
  g.B = B; g.sB = sB; g.ldb = x->N;
  g.sC = x->NN(); g.ldc = x->N;
  g.fstride = (long long)x->Lt * x->N;
  g.ns = x->ns();
  for (int m = -2; m <= 2; ++m) {
    const double v = std::exp(m * x->lam);
    const float hi = (float)v;
    g.e[m + 2].hi = hi;
    g.e[m + 2].lo = (float)(v - (double)hi);
  }
  return g;
}

enum ConstId { OZ_EM = 0, OZ_EP = 1, OZ_EMH = 2, OZ_EPH = 3 };

// Double-float product with one constant operand: tensor cores (exact BF16 slicing) when
// available for this N, else the SIMT double-float kernel.
void df_gemm(nmc_ctx* x, DfGemmArgs& g, int const_id, bool const_is_a) {
  cudaStream_t st = x->st();
  if (x->oz) {
    const int r = const_is_a ? 0 : 1;
    g.oz_const = x->dOz[const_id][r];
    g.oz_const_exp = x->dOzExp[const_id][r];
    launch(x, KC_GEMM_TC, [&] { gemm_tc(g, const_is_a, x->tmap[const_id][r], x->dErr, st); });
  } else {
    launch(x, KC_GEMM_DF, [&] { gemm_df(g, st); });
  }
}

UDTView identity_view(const nmc_ctx* x) { return UDTView{x->dI, 0, x->dOnes, 0, x->dI, 0}; }
UDTView view_of(const nmc_ctx* x, const UDTBuf& b) {
  return UDTView{b.U, x->NN(), b.D, x->N, b.T, x->NN()};
}

// ---------------------------------------------------------------------------- steps
void wrap(nmc_ctx* x, int l, bool up) {
  cudaStream_t st = x->st();
  const long long NN = x->NN();
  if (x->dfp()) {
    const int8_t* fl = x->dS + (long long)l * x->N;
    if (up) {  // T1 = Em (e^V G e^-V); G = T1 Ep
      DfGemmArgs g = df_base(x, x->dEm2, 0, x->dG2, NN);
      g.C = x->dT12;
      g.bfields = fl; g.br = 1; g.bc = -1;
      df_gemm(x, g, OZ_EM, true);
      DfGemmArgs h = df_base(x, x->dT12, NN, x->dEp2, 0);
      h.C = x->dG2;
      df_gemm(x, h, OZ_EP, false);
    } else {   // T1 = Ep G; G = e^-V (T1 Em) e^V
      DfGemmArgs g = df_base(x, x->dEp2, 0, x->dG2, NN);
      g.C = x->dT12;
      df_gemm(x, g, OZ_EP, true);
      DfGemmArgs h = df_base(x, x->dT12, NN, x->dEm2, 0);
      h.C = x->dG2;
      h.cfields = fl; h.cr = -1; h.cc = 1;
      df_gemm(x, h, OZ_EM, false);
    }
    return;
  }
  if (x->fp32()) {
    if (up) {  // T1 = Em (e^V G e^-V); G = T1 Ep
      auto g = gemm_base<float>(x, x->dEmf, 0, x->dGf, NN, x->dT1f);
      g.brow = field_scale(x, l, false);
      g.bcol = field_scale(x, l, true);
      launch(x, KC_GEMM, [&] { gemm(g, st); });
      launch(x, KC_GEMM, [&] { gemm(gemm_base<float>(x, x->dT1f, NN, x->dEpf, 0, x->dGf), st); });
    } else {   // T1 = Ep G; G = e^-V (T1 Em) e^V
      launch(x, KC_GEMM, [&] { gemm(gemm_base<float>(x, x->dEpf, 0, x->dGf, NN, x->dT1f), st); });
      auto g = gemm_base<float>(x, x->dT1f, NN, x->dEmf, 0, x->dGf);
      g.crow = field_scale(x, l, true);
      g.ccol = field_scale(x, l, false);
      launch(x, KC_GEMM, [&] { gemm(g, st); });
    }
  } else {
    if (up) {
      auto g = gemm_base<double>(x, x->dEm, 0, x->dG, NN, x->dT1);
      g.brow = field_scale(x, l, false);
      g.bcol = field_scale(x, l, true);
      launch(x, KC_GEMM, [&] { gemm(g, st); });
      launch(x, KC_GEMM, [&] { gemm(gemm_base<double>(x, x->dT1, NN, x->dEp, 0, x->dG), st); });
    } else {
      launch(x, KC_GEMM, [&] { gemm(gemm_base<double>(x, x->dEp, 0, x->dG, NN, x->dT1), st); });
      auto g = gemm_base<double>(x, x->dT1, NN, x->dEm, 0, x->dG);
      g.crow = field_scale(x, l, true);
      g.ccol = field_scale(x, l, false);
      launch(x, KC_GEMM, [&] { gemm(g, st); });
    }
  }
}

void flip(nmc_ctx* x, int l, const uint8_t* replay) {
  const uint32_t k0 = (uint32_t)(x->seed & 0xffffffffu), k1 = (uint32_t)(x->seed >> 32);
  const double dm = std::exp(-2.0 * x->lam) - 1.0, dp = std::exp(2.0 * x->lam) - 1.0;
  if (x->dfp()) {
    auto split = [](double v) {
      df2 r;
      r.hi = (float)v;
      r.lo = (float)(v - (double)r.hi);
      return r;
    };
    FlipArgs<df2> f{x->dG2, x->dS, x->N, x->Lt, l, x->kk, x->g_in_smem, k0, k1,
                    (uint32_t)x->sweep_counter, x->opt.chain_offset, dm, dp, x->dSign,
                    x->dCounts, replay, nullptr, split(dm), split(dp), x->ns(), x->dCtr};
    f.tc_fold = x->tc() ? 1 : 0;
    f.chain_id = x->dChainId;
    f.sweep_base = x->dSweepBase;
    launch(x, KC_FLIP, [&] { flip_slice(f, x->chains(), x->st()); });
  } else if (x->fp32()) {
    FlipArgs<float> f{x->dGf, x->dS, x->N, x->Lt, l, x->kk, x->g_in_smem, k0, k1,
                      (uint32_t)x->sweep_counter, x->opt.chain_offset, dm, dp, x->dSign,
                      x->dCounts, replay, nullptr, df2{0.f, 0.f}, df2{0.f, 0.f}, x->ns(), x->dCtr};
    f.chain_id = x->dChainId;
    f.sweep_base = x->dSweepBase;
    launch(x, KC_FLIP, [&] { flip_slice(f, x->chains(), x->st()); });
  } else {
    FlipArgs<double> f{x->dG, x->dS, x->N, x->Lt, l, x->kk, x->g_in_smem, k0, k1,
                       (uint32_t)x->sweep_counter, x->opt.chain_offset, dm, dp, x->dSign,
                       x->dCounts, replay, nullptr, df2{0.f, 0.f}, df2{0.f, 0.f}, x->ns(), x->dCtr};
    f.chain_id = x->dChainId;
    f.sweep_base = x->dSweepBase;
    launch(x, KC_FLIP, [&] { flip_slice(f, x->chains(), x->st()); });
  }
}

// The FP64 products of the stabilization (T updates, recompute): k_gemm on the FP64 pipe,
// or, with nmc_options.stab_pairs, the same products accumulated in FP32 pairs
void stab_gemm(nmc_ctx* x, const GemmArgs<double>& g) {
  cudaStream_t st = x->st();
  if (x->opt.stab_pairs) launch(x, KC_GEMM_PAIR, [&] { gemm_pair(g, st); });
  else launch(x, KC_GEMM, [&] { gemm(g, st); });
}

// dst = QRP-UDT of (product of block j's B matrices) applied to src; right: B_block src,
// left (transposed stack): B_block^T src.
void stack_update(nmc_ctx* x, int j, const UDTView& src, const UDTBuf& dst, bool right) {
  cudaStream_t st = x->st();
  const long long NN = x->NN();
  const int w = x->w;
  double* X = x->dX;
  double* X2 = x->dX2;
  if (x->dfp()) {
    // (B_block U) in double-float, then X = (B_block U) D in FP64 for the QR:
    // right: B_block = B_{(j+1)w-1} ... B_{jw}; left (transposed): B_{jw}^T ... B_{(j+1)w-1}^T
    const long long nsplit = src.sU ? NN * x->batch() : NN;
    launch(x, KC_OTHER, [&] { split_to_df(src.U, x->dXa, nsplit, st); });
    const df2* cur = x->dXa;
    long long scur = src.sU ? NN : 0;
    df2* bufs[2] = {x->dXb, x->dXa};
    for (int k = 0; k < w; ++k) {
      const int l = right ? j * w + k : (j + 1) * w - 1 - k;
      const bool last = k == w - 1;
      DfGemmArgs g = df_base(x, x->dEm2, 0, cur, scur);
      const int8_t* fl = x->dS + (long long)l * x->N;
      if (right) { g.bfields = fl; g.br = 1; }
      else { g.cfields = fl; g.cr = 1; }
      if (last) {
        g.Cd = X;
        g.colscale = src.D;
        g.sColscale = src.sD;
      } else {
        g.C = bufs[k & 1];
      }
      df_gemm(x, g, OZ_EM, true);
      cur = bufs[k & 1];
      scur = NN;
    }
    launch(x, KC_QRP, [&] { qrp_udt(X, dst.U, dst.D, x->dTp, x->dWS, x->N, x->batch(), st); });
    stab_gemm(x, gemm_base<double>(x, x->dTp, NN, src.T, src.sT, dst.T));
    return;
  }
  if (right) {
    const int l0 = j * w;
    auto g = gemm_base<double>(x, x->dEm, 0, src.U, src.sU, X);
    g.brow = field_scale(x, l0, false);
    g.bcol = vec_scale(src.D, src.sD, SC_VEC);
    launch(x, KC_GEMM, [&] { gemm(g, st); });
    for (int l = l0 + 1; l < l0 + w; ++l) {
      auto h = gemm_base<double>(x, x->dEm, 0, X, NN, X2);
      h.brow = field_scale(x, l, false);
      launch(x, KC_GEMM, [&] { gemm(h, st); });
      std::swap(X, X2);
    }
  } else {
    const int lt = (j + 1) * w - 1;
    auto g = gemm_base<double>(x, x->dEm, 0, src.U, src.sU, X);
    g.bcol = vec_scale(src.D, src.sD, SC_VEC);
    g.crow = field_scale(x, lt, false);
    launch(x, KC_GEMM, [&] { gemm(g, st); });
    for (int l = lt - 1; l >= j * w; --l) {
      auto h = gemm_base<double>(x, x->dEm, 0, X, NN, X2);
      h.crow = field_scale(x, l, false);
      launch(x, KC_GEMM, [&] { gemm(h, st); });
      std::swap(X, X2);
    }
  }
  launch(x, KC_QRP, [&] { qrp_udt(X, dst.U, dst.D, x->dTp, x->dWS, x->N, x->batch(), st); });
  launch(x, KC_GEMM, [&] { gemm(gemm_base<double>(x, x->dTp, NN, src.T, src.sT, dst.T), st); });
}

// G = (I + R L)^{-1} with R = U_R D_R T_R, L^T = U_L D_L T_L:
//   X = Db_R^{-1} (U_R^T U_L) Db_L^{-1} + Ds_R (T_R T_L^T) Ds_L
//   G = U_L Db_L^{-1} X^{-1} Db_R^{-1} U_R^T
void recompute(nmc_ctx* x, const UDTView& R, const UDTView& L, bool drift) {
  cudaStream_t st = x->st();
  const long long NN = x->NN();
  auto g1 = gemm_base<double>(x, R.U, R.sU, L.U, L.sU, x->dM1);
  g1.transA = 1;
  g1.crow = vec_scale(R.D, R.sD, SC_INV_MAX1);
  g1.ccol = vec_scale(L.D, L.sD, SC_INV_MAX1);
  stab_gemm(x, g1);
  auto g2 = gemm_base<double>(x, R.T, R.sT, L.T, L.sT, x->dXs);
  g2.transB = 1;
  g2.crow = vec_scale(R.D, R.sD, SC_MIN1);
  g2.ccol = vec_scale(L.D, L.sD, SC_MIN1);
  g2.Cin = x->dM1; g2.sCin = NN; g2.ldcin = x->N; g2.beta = 1.0;
  stab_gemm(x, g2);
  launch(x, KC_SOLVE, [&] { solve_stab(x->dXs, R.U, R.sU, R.D, R.sD, x->dY, x->dWS, x->N, x->batch(), st); });
  auto g3 = gemm_base<double>(x, L.U, L.sU, x->dY, NN, x->dG);
  g3.brow = vec_scale(L.D, L.sD, SC_INV_MAX1);
  if (drift) {
    g3.ref = x->fp32() ? (const void*)x->dGf : x->dfp() ? (const void*)x->dG2 : (const void*)x->dG;
    g3.ref_is_float = x->fp32() ? 1 : x->dfp() ? 2 : 0;
    g3.sRef = NN;
    g3.drift = x->dDriftStab;
    cudaMemsetAsync(x->dDriftStab, 0, sizeof(unsigned long long) * x->chains(), st);
  }
  if (x->fp32()) { g3.Cf = x->dGf; g3.sCf = NN; }
  if (x->dfp()) { g3.Cdf = x->dG2; g3.sCdf = NN; }
  stab_gemm(x, g3);
  if (drift) {
    launch(x, KC_OTHER, [&] {
      fold_drift(x->dDriftStab, x->dDrift, x->dHist, x->hist_cap, x->dCtr + 2, x->chains(), st);
    });
    ++x->n_hist;
  }
}

void measure_now(nmc_ctx* x) {
  cudaStream_t st = x->st();
  const long long NN = x->NN();
  double* acc = x->dSeries;   // + (device series index) * chains * 8
  if (x->dfp()) {  // G~ = e^{dtau K/2} G e^{-dtau K/2} from the pair copy of the recomputed G
    DfGemmArgs g = df_base(x, x->dEph2, 0, x->dG2, NN);
    g.C = x->dT12;
    df_gemm(x, g, OZ_EPH, true);
    DfGemmArgs h = df_base(x, x->dT12, NN, x->dEmh2, 0);
    h.Cd = x->dM1;
    df_gemm(x, h, OZ_EMH, false);
    launch(x, KC_MEASURE, [&] { nmc::measure(x->dM1, x->dK, x->dSign, x->N, x->Lx, x->lattice, x->U, acc, x->chains(), x->ns(), st, x->dCtr + 1); });
    return;
  }
  launch(x, KC_GEMM, [&] { gemm(gemm_base<double>(x, x->dEph, 0, x->dG, NN, x->dT1), st); });   // e^{dtau K/2} G
  launch(x, KC_GEMM, [&] { gemm(gemm_base<double>(x, x->dT1, NN, x->dEmh, 0, x->dM1), st); });  // ... e^{-dtau K/2}
  launch(x, KC_MEASURE, [&] { nmc::measure(x->dM1, x->dK, x->dSign, x->N, x->Lx, x->lattice, x->U, acc, x->chains(), x->ns(), st, x->dCtr + 1); });
}

void sweep_up(nmc_ctx* x, bool meas, const uint8_t* replay) {
  const int nb = x->nb, w = x->w;
  for (int j = 0; j < nb; ++j) {
    for (int l = j * w; l < (j + 1) * w; ++l) {
      flip(x, l, replay);
      wrap(x, l, true);
    }
    const UDTView src = (j == 0) ? identity_view(x) : view_of(x, x->slot[j]);
    stack_update(x, j, src, x->spare, true);
    const UDTView Lv = (j + 1 == nb) ? identity_view(x) : view_of(x, x->slot[j + 1]);
    recompute(x, view_of(x, x->spare), Lv, true);
    if (j + 1 < nb) std::swap(x->spare, x->slot[j + 1]);
    if (meas) measure_now(x);
  }
}

void sweep_down(nmc_ctx* x, bool meas, const uint8_t* replay) {
  const int nb = x->nb, w = x->w;
  for (int j = nb - 1; j >= 0; --j) {
    for (int l = (j + 1) * w - 1; l >= j * w; --l) {
      wrap(x, l, false);
      flip(x, l, replay);
    }
    const UDTView src = (j + 1 == nb) ? identity_view(x) : view_of(x, x->slot[j + 1]);
    stack_update(x, j, src, x->spare, false);
    const UDTView Rv = (j == 0) ? identity_view(x) : view_of(x, x->slot[j]);
    recompute(x, Rv, view_of(x, x->spare), true);
    if (j >= 1) std::swap(x->spare, x->slot[j]);
    if (meas) measure_now(x);
  }
}

// Build the stacks a sweep of the given direction needs, and G, from the fields alone.
void build_stacks(nmc_ctx* x, bool for_up) {
  const int nb = x->nb;
  if (for_up) {  // left stacks L_j, j = nb-1..1; G_0 = (I + L_0)^{-1}
    for (int j = nb - 1; j >= 0; --j) {
      const UDTView src = (j + 1 == nb) ? identity_view(x) : view_of(x, x->slot[j + 1]);
      stack_update(x, j, src, x->spare, false);
      if (j >= 1) std::swap(x->spare, x->slot[j]);
    }
    recompute(x, identity_view(x), view_of(x, x->spare), false);
  } else {       // right stacks R_j, j = 1..nb-1; G_L = (I + R_nb)^{-1}
    for (int j = 0; j < nb; ++j) {
      const UDTView src = (j == 0) ? identity_view(x) : view_of(x, x->slot[j]);
      stack_update(x, j, src, x->spare, true);
      if (j + 1 < nb) std::swap(x->spare, x->slot[j + 1]);
    }
    recompute(x, view_of(x, x->spare), identity_view(x), false);
  }
}

// Copy the host counters to their device mirrors (the kernels read the device copies).
nmc_status push_counters(nmc_ctx* x) {
  const long long h[3] = {x->sweep_counter, x->n_series, x->n_hist};
  NMC_CUDA(x, cudaMemcpyAsync(x->dCtr, h, sizeof h, cudaMemcpyHostToDevice, x->st()));
  NMC_CUDA(x, cudaStreamSynchronize(x->st()));
  return NMC_OK;
}

nmc_status reset_chain_state(nmc_ctx* x) {
  cudaStream_t st = x->st();
  std::vector<double> ones(x->chains(), 1.0);
  NMC_CUDA(x, cudaMemcpyAsync(x->dSign, ones.data(), ones.size() * sizeof(double),
                              cudaMemcpyHostToDevice, st));
  NMC_CUDA(x, cudaMemsetAsync(x->dCounts, 0, 3 * sizeof(unsigned long long) * x->chains(), st));
  NMC_CUDA(x, cudaMemsetAsync(x->dDrift, 0, sizeof(unsigned long long) * x->chains(), st));
  NMC_CUDA(x, cudaMemsetAsync(x->dHist, 0, sizeof(unsigned long long) * x->hist_cap, st));
  default_chain_ids(x->dChainId, x->dSweepBase, x->chains(), x->opt.chain_offset, st);
  x->n_hist = 0;
  x->n_series = 0;
  NMC_TRY(push_counters(x));
  x->phase = 0;
  NMC_CUDA(x, cudaStreamSynchronize(st));
  return NMC_OK;
}

nmc_status after_fields(nmc_ctx* x) {
  NMC_TRY(reset_chain_state(x));
  build_stacks(x, true);
  x->direct_since_build = 0;
  NMC_CUDA(x, cudaGetLastError());
  NMC_CUDA(x, cudaStreamSynchronize(x->st()));
  x->have_fields = true;
  return NMC_OK;
}

nmc_status ensure_series(nmc_ctx* x, long long need) {
  if (need <= x->series_cap) return NMC_OK;
  long long cap = std::max<long long>(need, 2 * x->series_cap);
  cap = std::max<long long>(cap, 64);
  double* p = nullptr;
  const size_t bytes = (size_t)cap * x->chains() * 8 * sizeof(double);
  const cudaError_t e = cudaMallocAsync((void**)&p, bytes, x->st());
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(x, NMC_ENOMEM, "series buffer: cudaMallocAsync failed");
  }
  NMC_CUDA(x, cudaMemsetAsync(p, 0, bytes, x->st()));
  if (x->dSeries && x->n_series > 0)
    NMC_CUDA(x, cudaMemcpyAsync(p, x->dSeries, (size_t)x->n_series * x->chains() * 8 * sizeof(double),
                                cudaMemcpyDeviceToDevice, x->st()));
  if (x->dSeries) {  // stream-ordered: freed after the copy above
    x->allocs.erase(std::remove(x->allocs.begin(), x->allocs.end(), (void*)x->dSeries),
                    x->allocs.end());
    cudaFreeAsync(x->dSeries, x->st());
  }
  x->dSeries = p;
  x->allocs.push_back(p);
  x->series_cap = cap;
  drop_graphs(x);   // recorded measurements address the old buffer
  return NMC_OK;
}

// first failed index check of the NMC_DEBUG build (0: none, or not a debug build)
unsigned int debug_failed() {
  unsigned int (*const readers[])() = {debug_fail_flip, debug_fail_stab, debug_fail_gemm,
                                       debug_fail_gemm_tc, debug_fail_misc};
  for (auto r : readers)
    if (const unsigned int id = r()) return id;
  return 0u;
}

nmc_status check_drift(nmc_ctx* x) {
  if (const unsigned int id = debug_failed()) {
    char buf[96];
    std::snprintf(buf, sizeof buf, "index check %u failed (bounds-checked build)", id);
    return fail(x, NMC_ECUDA, buf);
  }
  std::vector<unsigned long long> bits(x->chains());
  int err = 0;
  NMC_CUDA(x, cudaMemcpyAsync(bits.data(), x->dDrift, bits.size() * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, x->st()));
  NMC_CUDA(x, cudaMemcpyAsync(&err, x->dErr, sizeof(int), cudaMemcpyDeviceToHost, x->st()));
  NMC_CUDA(x, cudaStreamSynchronize(x->st()));
  if (err) {
    char buf[120];
    std::snprintf(buf, sizeof buf, "a bounded device-side wait expired (tensor-core product, "
                  "stage %d); results of this call are not valid", err);
    return fail(x, NMC_ETIMEOUT, buf);
  }
  double tol = x->opt.drift_tol;
  if (tol <= 0) tol = x->fp32() ? 1e-3 : x->dfp() ? 1e-5 : 1e-6;
  for (size_t c = 0; c < bits.size(); ++c) {
    double d;
    std::memcpy(&d, &bits[c], sizeof d);
    if (!std::isfinite(d) || d > tol) {
      char buf[160];
      std::snprintf(buf, sizeof buf, "chain %zu: stabilization drift %.3e exceeds %.1e", c, d, tol);
      return fail(x, NMC_ENUMERIC, buf);
    }
  }
  return NMC_OK;
}

std::vector<const void*> slot_state(const nmc_ctx* x) {
  std::vector<const void*> v{x->spare.U, x->spare.D, x->spare.T};
  for (const auto& b : x->slot) {
    v.push_back(b.U);
    v.push_back(b.D);
    v.push_back(b.T);
  }
  return v;
}

// The stack-buffer permutation of one sweep (the swaps of sweep_up / sweep_down).
void advance_slots(nmc_ctx* x, bool up) {
  if (up)
    for (int j = 0; j + 1 < x->nb; ++j) std::swap(x->spare, x->slot[j + 1]);
  else
    for (int j = x->nb - 1; j >= 1; --j) std::swap(x->spare, x->slot[j]);
}

// One sweep as a CUDA graph: recorded on first use (on a private stream; nothing runs while
// recording), then replayed on the context stream. Every per-sweep value the kernels need
// (Philox sweep counter, measurement slot, drift-history slot) is read from device
// counters, so one recording serves every later sweep of that direction from the same
// stack-buffer arrangement. Returns false (the caller then launches the sweep directly) when
// graphs are off, while profiling, or if recording fails.
bool sweep_graph(nmc_ctx* x, bool up, bool meas) {
  if (!x->opt.sweep_graphs || !x->use_graphs || x->prof || x->direct_since_build < 2)
    return false;
  SweepGraph& gr = x->graphs[up ? 0 : 1][meas ? 1 : 0];
  const std::vector<const void*> state = slot_state(x);
  if (gr.exec && gr.ptrs != state) {
    cudaGraphExecDestroy(gr.exec);
    gr.exec = nullptr;
  }
  if (!gr.exec) {
    if (!x->cap_stream &&
        cudaStreamCreateWithFlags(&x->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      x->use_graphs = false;
      return false;
    }
    long long before[kNumClasses];
    std::memcpy(before, x->launches, sizeof before);
    const UDTBuf spare0 = x->spare;
    const std::vector<UDTBuf> slot0 = x->slot;
    const long long hist0 = x->n_hist;
    if (cudaStreamBeginCapture(x->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      x->use_graphs = false;
      return false;
    }
    x->cap = true;
    if (up) sweep_up(x, meas, nullptr);
    else sweep_down(x, meas, nullptr);
    launch(x, KC_OTHER, [&] { advance_counters(x->dCtr, meas ? 1 : 0, x->st()); });
    x->cap = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(x->cap_stream, &graph);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    // recording ran the host side of the sweep only: put its host state back
    x->spare = spare0;
    x->slot = slot0;
    x->n_hist = hist0;
    for (int k = 0; k < kNumClasses; ++k) {
      gr.launches[k] = x->launches[k] - before[k];
      x->launches[k] = before[k];
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      x->use_graphs = false;
      return false;
    }
    gr.exec = exec;
    gr.ptrs = state;
    ++x->graphs_recorded;
  }
  if (cudaGraphLaunch(gr.exec, x->st()) != cudaSuccess) {
    cudaGetLastError();
    x->use_graphs = false;
    return false;
  }
  advance_slots(x, up);
  ++x->graphs_replayed;
  x->n_hist += x->nb;   // one drift record per block
  for (int k = 0; k < kNumClasses; ++k) x->launches[k] += gr.launches[k];
  return true;
}

nmc_status run_sweeps(nmc_ctx* x, int n, int meas, const uint8_t* replay, bool wait = true) {
  if (meas) NMC_TRY(ensure_series(x, x->n_series + n));
  for (int s = 0; s < n; ++s) {
    const bool up = x->phase % 2 == 0;
    if (replay || !sweep_graph(x, up, meas != 0)) {
      if (up) sweep_up(x, meas != 0, replay);
      else sweep_down(x, meas != 0, replay);
      launch(x, KC_OTHER, [&] { advance_counters(x->dCtr, meas ? 1 : 0, x->st()); });
      ++x->direct_since_build;
    }
    NMC_CUDA(x, cudaGetLastError());
    ++x->phase;
    ++x->sweep_counter;
    if (meas) ++x->n_series;
  }
  if (!wait) return NMC_OK;
  NMC_CUDA(x, cudaStreamSynchronize(x->st()));
  return check_drift(x);
}

bool valid_fields(const int8_t* s, size_t n) {
  for (size_t e = 0; e < n; ++e)
    if (s[e] != 1 && s[e] != -1) return false;
  return true;
}

void binned(const std::vector<double>& series, int nbins, double& mean, double& err) {
  const size_t n = series.size();
  mean = 0;
  err = 0;
  if (n == 0) return;
  for (double v : series) mean += v;
  mean /= n;
  if ((int)n < nbins || nbins < 2) return;
  const size_t per = n / nbins;
  std::vector<double> b(nbins, 0.0);
  for (int k = 0; k < nbins; ++k) {
    for (size_t e = 0; e < per; ++e) b[k] += series[k * per + e];
    b[k] /= per;
  }
  double m = 0;
  for (double v : b) m += v;
  m /= nbins;
  double var = 0;
  for (double v : b) var += (v - m) * (v - m);
  err = std::sqrt(var / (nbins - 1) / nbins);
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

void nmc_default_options(nmc_options* o) {
  if (!o) return;
  o->n_chains = 1;
  o->delay_k = 16;
  o->precision = NMC_FP64;
  o->drift_tol = 0.0;
  o->chain_offset = 0;
  o->cuda_stream = nullptr;
  o->ph_symmetric = 0;
  o->sweep_graphs = 1;
  o->stab_pairs = 0;
}

// Sites of a lattice, or 0 if the lattice and sizes are not accepted: square needs even
// lengths (bipartite) or length 1; honeycomb is bipartite for any cell counts.
static int lattice_sites(int lattice, int Lx, int Ly) {
  if (Lx < 1 || Ly < 1 || Lx > 1024 || Ly > 1024) return 0;
  int N = 0;
  if (lattice == NMC_SQUARE) {
    if ((Lx > 1 && Lx % 2) || (Ly > 1 && Ly % 2)) return 0;
    N = Lx * Ly;
  } else if (lattice == NMC_HONEYCOMB) {
    N = 2 * Lx * Ly;
  }
  return (N >= 2 && N <= 1024) ? N : 0;
}

nmc_status nmc_create(int lattice, int Lx, int Ly, double t, double U, double beta, double dtau,
                      int n_wrap, uint64_t seed, nmc_ctx** out) {
  if (!out) return NMC_EINVAL;
  *out = nullptr;
  const int N = lattice_sites(lattice, Lx, Ly);
  if (!N) return NMC_EINVAL;
  if (!(t > 0) || !(U >= 0) || !(beta > 0) || !(dtau > 0) || n_wrap < 1) return NMC_EINVAL;
  const double ratio = beta / dtau;
  const double Ltd = std::round(ratio);
  if (Ltd < 1 || std::fabs(ratio - Ltd) > 1e-9 * ratio || Ltd > 1e6) return NMC_EINVAL;
  const int Lt = (int)Ltd;
  if (Lt % n_wrap) return NMC_EINVAL;
  nmc_ctx* x = new (std::nothrow) nmc_ctx();
  if (!x) return NMC_ENOMEM;
  x->lattice = lattice; x->Lx = Lx; x->Ly = Ly; x->N = N; x->Lt = Lt; x->w = n_wrap; x->nb = Lt / n_wrap;
  x->t = t; x->U = U; x->beta = beta; x->dtau = dtau; x->seed = seed;
  x->lam = std::acosh(std::exp(dtau * U / 2.0));
  nmc_default_options(&x->opt);
  nmc_host::hopping(lattice, Lx, Ly, t, x->hK);
  std::vector<double> A = x->hK, wv, V;
  nmc_host::jacobi_eigh(x->N, A, wv, V);
  nmc_host::expk_from_eig(x->N, wv, V, -dtau, x->hEm);
  nmc_host::expk_from_eig(x->N, wv, V, +dtau, x->hEp);
  nmc_host::expk_from_eig(x->N, wv, V, -dtau / 2, x->hEmh);
  nmc_host::expk_from_eig(x->N, wv, V, +dtau / 2, x->hEph);
  clamp_delay(x);
  *out = x;
  return NMC_OK;
}

nmc_status nmc_configure(nmc_ctx* x, const nmc_options* o) {
  if (!x) return NMC_EINVAL;
  if (x->have_fields) return fail(x, NMC_ESTATE, "nmc_configure after fields were set");
  nmc_options n;
  nmc_default_options(&n);
  if (o) n = *o;
  if (n.precision == NMC_TF32X3)
    return fail(x, NMC_EINVAL,
                "NMC_TF32X3 is not built: three TF32 products with FP32 accumulation give "
                "FP32-class products, which cannot hold the 1e-5 drift bar of this model");
  if (n.n_chains < 1 || n.delay_k < 1 ||
      (n.precision != NMC_FP64 && n.precision != NMC_FP32 && n.precision != NMC_SPLIT_BF16 &&
       n.precision != NMC_FP32X2) ||
      n.chain_offset < 0 || n.n_chains > (1 << 20) || (n.ph_symmetric != 0 && n.ph_symmetric != 1) ||
      (n.sweep_graphs != 0 && n.sweep_graphs != 1) || (n.stab_pairs != 0 && n.stab_pairs != 1))
    return fail(x, NMC_EINVAL, "invalid nmc_options");
  if (n.stab_pairs && n.precision != NMC_SPLIT_BF16 && n.precision != NMC_FP32X2)
    return fail(x, NMC_EINVAL, "stab_pairs applies to the compensated precisions only");
  x->opt = n;
  clamp_delay(x);
  return alloc_all(x);
}

nmc_status nmc_set_fields(nmc_ctx* x, const int8_t* s, size_t n) {
  if (!x || !s) return NMC_EINVAL;
  const size_t need = (size_t)x->opt.n_chains * x->Lt * x->N;
  if (n != need) return fail(x, NMC_EINVAL, "nmc_set_fields: size mismatch");
  if (!valid_fields(s, n)) return fail(x, NMC_EINVAL, "nmc_set_fields: values must be +1 or -1");
  NMC_TRY(ensure_configured(x));
  NMC_CUDA(x, cudaMemcpyAsync(x->dS, s, n, cudaMemcpyHostToDevice, x->st()));
  return after_fields(x);
}

nmc_status nmc_set_fields_device(nmc_ctx* x, const int8_t* d_s, size_t n) {
  if (!x || !d_s) return NMC_EINVAL;
  const size_t need = (size_t)x->opt.n_chains * x->Lt * x->N;
  if (n != need) return fail(x, NMC_EINVAL, "nmc_set_fields_device: size mismatch");
  NMC_TRY(ensure_configured(x));
  NMC_CUDA(x, cudaMemcpyAsync(x->dS, d_s, n, cudaMemcpyDeviceToDevice, x->st()));
  launch(x, KC_OTHER, [&] { fields_normalize(x->dS, (long long)n, x->st()); });
  return after_fields(x);
}

nmc_status nmc_generate(nmc_ctx* x, int mode, const void* model) {
  if (!x) return NMC_EINVAL;
  if (mode != 0 && mode != 1) return fail(x, NMC_EINVAL, "nmc_generate: mode must be 0 or 1");
  if (mode == 1 && !model) return fail(x, NMC_EINVAL, "nmc_generate: mode 1 needs a generator");
  NMC_TRY(ensure_configured(x));
  if (mode == 1) {
    NMC_CUDA(x, cudaStreamSynchronize(x->st()));   // the generator writes on its own stream
    const nmc_status s = nmc_gen_fill_fields((nmc_gen*)const_cast<void*>(model), x->N, x->Lt,
                                             x->opt.chain_offset, x->chains(), x->dS, x->st());
    if (s != NMC_OK) return fail(x, s, std::string("nmc_generate: ") +
                                        nmc_gen_last_error((const nmc_gen*)model));
  } else {
    launch(x, KC_OTHER, [&] {
      init_fields(x->dS, x->chains(), x->Lt, x->N, (uint32_t)(x->seed & 0xffffffffu),
                  (uint32_t)(x->seed >> 32), x->opt.chain_offset, x->st());
    });
  }
  NMC_CUDA(x, cudaGetLastError());
  return after_fields(x);
}

nmc_status nmc_sweep(nmc_ctx* x, int n_sweeps, int measure) {
  if (!x || n_sweeps < 0) return NMC_EINVAL;
  if (!x->have_fields) return fail(x, NMC_ESTATE, "nmc_sweep before fields were set");
  NMC_TRY(ensure_configured(x));
  return run_sweeps(x, n_sweeps, measure, nullptr);
}

nmc_status nmc_sweep_async(nmc_ctx* x, int n_sweeps, int measure) {
  if (!x || n_sweeps < 0) return NMC_EINVAL;
  if (!x->have_fields) return fail(x, NMC_ESTATE, "nmc_sweep_async before fields were set");
  NMC_TRY(ensure_configured(x));
  return run_sweeps(x, n_sweeps, measure, nullptr, false);
}

nmc_status nmc_query(nmc_ctx* x, int* idle) {
  if (!x || !idle) return NMC_EINVAL;
  if (!x->configured) return fail(x, NMC_ESTATE, "nmc_query before configuration");
  NMC_CUDA(x, cudaSetDevice(x->device));
  const cudaError_t e = cudaStreamQuery(x->st());
  if (e == cudaSuccess) { *idle = 1; return NMC_OK; }
  if (e == cudaErrorNotReady) { cudaGetLastError(); *idle = 0; return NMC_OK; }
  return fail(x, NMC_ECUDA, std::string("cudaStreamQuery: ") + cudaGetErrorString(e));
}

nmc_status nmc_sync(nmc_ctx* x) {
  if (!x) return NMC_EINVAL;
  if (!x->configured) return fail(x, NMC_ESTATE, "nmc_sync before configuration");
  NMC_CUDA(x, cudaSetDevice(x->device));
  NMC_CUDA(x, cudaStreamSynchronize(x->st()));
  return check_drift(x);
}

nmc_status nmc_footprint(int lattice, int Lx, int Ly, double t, double U, double beta,
                         double dtau, int n_wrap, const nmc_options* opts, size_t* bytes) {
  if (!bytes) return NMC_EINVAL;
  nmc_ctx* x = nullptr;
  const nmc_status st = nmc_create(lattice, Lx, Ly, t, U, beta, dtau, n_wrap, 0, &x);
  if (st != NMC_OK) return st;
  nmc_options o;
  nmc_default_options(&o);
  if (opts) o = *opts;
  x->opt = o;
  clamp_delay(x);
  x->dry = true;
  alloc_all(x);
  *bytes = x->dry_bytes;
  delete x;
  return NMC_OK;
}

nmc_status nmc_sweep_replay(nmc_ctx* x, const uint8_t* accept, size_t n, int measure) {
  if (!x || !accept) return NMC_EINVAL;
  if (!x->have_fields) return fail(x, NMC_ESTATE, "nmc_sweep_replay before fields were set");
  const size_t need = (size_t)x->opt.n_chains * x->Lt * x->N;
  if (n != need) return fail(x, NMC_EINVAL, "nmc_sweep_replay: size mismatch");
  NMC_TRY(ensure_configured(x));
  if (!x->dReplay) NMC_TRY(dalloc(x, &x->dReplay, need));
  NMC_CUDA(x, cudaMemcpyAsync(x->dReplay, accept, n, cudaMemcpyHostToDevice, x->st()));
  return run_sweeps(x, 1, measure, x->dReplay);
}

nmc_status nmc_series(nmc_ctx* x, double* out, long long max_sweeps, long long* n_sweeps) {
  if (!x || !n_sweeps || max_sweeps < 0 || (max_sweeps > 0 && !out)) return NMC_EINVAL;
  if (!x->configured) return fail(x, NMC_ESTATE, "nmc_series before configuration");
  NMC_CUDA(x, cudaSetDevice(x->device));
  *n_sweeps = x->n_series;
  const long long S = std::min(max_sweeps, x->n_series);
  if (S > 0)
    NMC_CUDA(x, cudaMemcpyAsync(out, x->dSeries, (size_t)S * x->chains() * 8 * sizeof(double),
                                cudaMemcpyDeviceToHost, x->st()));
  NMC_CUDA(x, cudaStreamSynchronize(x->st()));
  return NMC_OK;
}

nmc_status nmc_measure(nmc_ctx* x, nmc_obs* per_chain, nmc_obs* pooled) {
  if (!x) return NMC_EINVAL;
  if (!x->configured) return fail(x, NMC_ESTATE, "nmc_measure before configuration");
  NMC_CUDA(x, cudaSetDevice(x->device));
  const int C = x->chains();
  const long long S = x->n_series;
  std::vector<double> ser((size_t)S * C * 8);
  std::vector<unsigned long long> cnt(3 * (size_t)C), dr(C);
  cudaStream_t st = x->st();
  if (S > 0)
    NMC_CUDA(x, cudaMemcpyAsync(ser.data(), x->dSeries, ser.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
  NMC_CUDA(x, cudaMemcpyAsync(cnt.data(), x->dCounts, cnt.size() * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, st));
  NMC_CUDA(x, cudaMemcpyAsync(dr.data(), x->dDrift, dr.size() * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, st));
  NMC_CUDA(x, cudaStreamSynchronize(st));
  const long long per_sweep = x->nb;
  std::vector<nmc_obs> pc(C);
  // per chain
  for (int c = 0; c < C; ++c) {
    nmc_obs& o = pc[c];
    std::memset(&o, 0, sizeof o);
    nmc_est* est[6] = {&o.energy, &o.ekin, &o.double_occ, &o.s_pipi, &o.density, &o.sign};
    double tot[6] = {0, 0, 0, 0, 0, 0};
    for (long long s = 0; s < S; ++s)
      for (int k = 0; k < 6; ++k) tot[k] += ser[((size_t)s * C + c) * 8 + k];
    for (int k = 0; k < 5; ++k) {
      std::vector<double> seq;
      for (long long s = 0; s < S; ++s) {
        const double* a = &ser[((size_t)s * C + c) * 8];
        seq.push_back(a[5] != 0 ? a[k] / a[5] : 0.0);
      }
      double m, e;
      binned(seq, 10, m, e);
      est[k]->mean = tot[5] != 0 ? tot[k] / tot[5] : 0.0;
      est[k]->err = e;
    }
    {
      std::vector<double> seq;
      for (long long s = 0; s < S; ++s) seq.push_back(ser[((size_t)s * C + c) * 8 + 5] / per_sweep);
      double m, e;
      binned(seq, 10, m, e);
      o.sign.mean = S > 0 ? tot[5] / (S * per_sweep) : 0.0;
      o.sign.err = e;
    }
    o.accept = cnt[3 * c] ? (double)cnt[3 * c + 1] / (double)cnt[3 * c] : 0.0;
    std::memcpy(&o.max_drift, &dr[c], sizeof(double));
    o.n_meas = S * per_sweep;
    o.n_disagree = (long long)cnt[3 * c + 2];
  }
  if (per_chain) std::memcpy(per_chain, pc.data(), C * sizeof(nmc_obs));
  if (pooled) {
    nmc_obs p;
    std::memset(&p, 0, sizeof p);
    auto pool = [&](nmc_est nmc_obs::*fld, nmc_est& dst) {
      double m = 0;
      for (int c = 0; c < C; ++c) m += (pc[c].*fld).mean;
      m /= C;
      double e = 0;
      if (C >= 2) {
        double v = 0;
        for (int c = 0; c < C; ++c) v += ((pc[c].*fld).mean - m) * ((pc[c].*fld).mean - m);
        e = std::sqrt(v / (C - 1) / C);
      } else {
        e = (pc[0].*fld).err;
      }
      dst.mean = m;
      dst.err = e;
    };
    pool(&nmc_obs::energy, p.energy);
    pool(&nmc_obs::ekin, p.ekin);
    pool(&nmc_obs::double_occ, p.double_occ);
    pool(&nmc_obs::s_pipi, p.s_pipi);
    pool(&nmc_obs::density, p.density);
    pool(&nmc_obs::sign, p.sign);
    unsigned long long att = 0, acc = 0, dis = 0;
    for (int c = 0; c < C; ++c) {
      att += cnt[3 * c];
      acc += cnt[3 * c + 1];
      dis += cnt[3 * c + 2];
      p.max_drift = std::max(p.max_drift, pc[c].max_drift);
    }
    p.accept = att ? (double)acc / (double)att : 0.0;
    p.n_meas = S * per_sweep;
    p.n_disagree = (long long)dis;
    *pooled = p;
  }
  return NMC_OK;
}

nmc_status nmc_get_fields(nmc_ctx* x, int8_t* s, size_t n) {
  if (!x || !s) return NMC_EINVAL;
  if (!x->have_fields) return fail(x, NMC_ESTATE, "no fields set");
  const size_t need = (size_t)x->opt.n_chains * x->Lt * x->N;
  if (n != need) return fail(x, NMC_EINVAL, "nmc_get_fields: size mismatch");
  NMC_CUDA(x, cudaSetDevice(x->device));
  NMC_CUDA(x, cudaMemcpyAsync(s, x->dS, n, cudaMemcpyDeviceToHost, x->st()));
  NMC_CUDA(x, cudaStreamSynchronize(x->st()));
  return NMC_OK;
}

nmc_status nmc_get_green(nmc_ctx* x, int chain, int spin, double* G) {
  if (!x || !G || chain < 0 || chain >= x->opt.n_chains || spin < 0 || spin > 1)
    return NMC_EINVAL;
  if (!x->have_fields) return fail(x, NMC_ESTATE, "no fields set");
  NMC_CUDA(x, cudaSetDevice(x->device));
  const long long NN = x->NN();
  const int sp_stored = x->ns() == 2 ? spin : 0;
  const long long off = ((long long)chain * x->ns() + sp_stored) * NN;
  if (x->dfp()) {
    std::vector<df2> tmp(NN);
    NMC_CUDA(x, cudaMemcpyAsync(tmp.data(), x->dG2 + off, NN * sizeof(df2),
                                cudaMemcpyDeviceToHost, x->st()));
    NMC_CUDA(x, cudaStreamSynchronize(x->st()));
    for (long long e = 0; e < NN; ++e) G[e] = (double)tmp[e].hi + (double)tmp[e].lo;
  } else if (x->fp32()) {
    std::vector<float> tmp(NN);
    NMC_CUDA(x, cudaMemcpyAsync(tmp.data(), x->dGf + off, NN * sizeof(float),
                                cudaMemcpyDeviceToHost, x->st()));
    NMC_CUDA(x, cudaStreamSynchronize(x->st()));
    for (long long e = 0; e < NN; ++e) G[e] = tmp[e];
  } else {
    NMC_CUDA(x, cudaMemcpyAsync(G, x->dG + off, NN * sizeof(double), cudaMemcpyDeviceToHost,
                                x->st()));
    NMC_CUDA(x, cudaStreamSynchronize(x->st()));
  }
  if (x->ns() == 1 && spin == 1) {  // G_dn = I - P G_up^T P, P = sublattice signs
    const int N = x->N;
    std::vector<double> up(G, G + NN);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        const int pij = (nmc::site_parity(i, x->Lx, x->lattice) ^
                         nmc::site_parity(j, x->Lx, x->lattice)) ? -1 : 1;
        G[(size_t)i * N + j] = (i == j ? 1.0 : 0.0) - pij * up[(size_t)j * N + i];
      }
  }
  return NMC_OK;
}

nmc_status nmc_get_dims(const nmc_ctx* x, int* N, int* L_tau, int* n_chains, int* delay_k) {
  if (!x) return NMC_EINVAL;
  if (N) *N = x->N;
  if (L_tau) *L_tau = x->Lt;
  if (n_chains) *n_chains = x->opt.n_chains;
  if (delay_k) *delay_k = x->kk;
  return NMC_OK;
}

// checkpoint layout: u64 magic, i64 N, Lt, chains, seed, sweep_counter, phase, n_series,
// precision; then fields (int8), sign (f64), counts (u64 x3), drift (u64), chain ids (i64),
// sweep bases (i64), series (f64)
nmc_status nmc_checkpoint(nmc_ctx* x, void* buf, size_t* n) {
  if (!x || !n) return NMC_EINVAL;
  if (!x->have_fields) return fail(x, NMC_ESTATE, "no fields set");
  const int C = x->chains();
  const size_t nf = (size_t)C * x->Lt * x->N;
  const size_t nser = (size_t)x->n_series * C * 8;
  const size_t hdr = 9 * sizeof(int64_t);
  const size_t total = hdr + nf + C * sizeof(double) + 3 * C * sizeof(uint64_t) +
                       C * sizeof(uint64_t) + 2 * C * sizeof(int64_t) + nser * sizeof(double);
  if (!buf) { *n = total; return NMC_OK; }
  if (*n < total) return fail(x, NMC_EINVAL, "nmc_checkpoint: buffer too small");
  NMC_CUDA(x, cudaSetDevice(x->device));
  char* p = (char*)buf;
  const int64_t h[9] = {(int64_t)kCkptMagic, x->N, x->Lt, C, (int64_t)x->seed, x->sweep_counter,
                        x->phase, x->n_series,
                        x->opt.precision + 16 * x->opt.ph_symmetric + 256 * x->lattice +
                        4096 * x->opt.stab_pairs};
  std::memcpy(p, h, hdr);
  p += hdr;
  cudaStream_t st = x->st();
  NMC_CUDA(x, cudaMemcpyAsync(p, x->dS, nf, cudaMemcpyDeviceToHost, st)); p += nf;
  NMC_CUDA(x, cudaMemcpyAsync(p, x->dSign, C * sizeof(double), cudaMemcpyDeviceToHost, st));
  p += C * sizeof(double);
  NMC_CUDA(x, cudaMemcpyAsync(p, x->dCounts, 3 * C * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  p += 3 * C * sizeof(uint64_t);
  NMC_CUDA(x, cudaMemcpyAsync(p, x->dDrift, C * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  p += C * sizeof(uint64_t);
  NMC_CUDA(x, cudaMemcpyAsync(p, x->dChainId, C * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  p += C * sizeof(int64_t);
  NMC_CUDA(x, cudaMemcpyAsync(p, x->dSweepBase, C * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  p += C * sizeof(int64_t);
  if (nser)
    NMC_CUDA(x, cudaMemcpyAsync(p, x->dSeries, nser * sizeof(double), cudaMemcpyDeviceToHost, st));
  NMC_CUDA(x, cudaStreamSynchronize(st));
  *n = total;
  return NMC_OK;
}

nmc_status nmc_restore(nmc_ctx* x, const void* buf, size_t n) {
  if (!x || !buf) return NMC_EINVAL;
  const size_t hdr = 9 * sizeof(int64_t);
  if (n < hdr) return fail(x, NMC_EINVAL, "nmc_restore: truncated");
  int64_t h[9];
  std::memcpy(h, buf, hdr);
  const int C = x->opt.n_chains;
  if ((uint64_t)h[0] != kCkptMagic || h[1] != x->N || h[2] != x->Lt || h[3] != C ||
      (uint64_t)h[4] != x->seed || h[8] != x->opt.precision + 16 * x->opt.ph_symmetric + 256 * x->lattice +
                        4096 * x->opt.stab_pairs)
    return fail(x, NMC_EINVAL, "nmc_restore: checkpoint does not match this context");
  const size_t nf = (size_t)C * x->Lt * x->N;
  const long long ns = h[7];
  const size_t nser = (size_t)ns * C * 8;
  const size_t total = hdr + nf + C * sizeof(double) + 4 * C * sizeof(uint64_t) +
                       2 * C * sizeof(int64_t) + nser * sizeof(double);
  if (n < total) return fail(x, NMC_EINVAL, "nmc_restore: truncated");
  const char* p = (const char*)buf + hdr;
  if (!valid_fields((const int8_t*)p, nf)) return fail(x, NMC_EINVAL, "nmc_restore: bad fields");
  NMC_TRY(ensure_configured(x));
  cudaStream_t st = x->st();
  NMC_CUDA(x, cudaMemcpyAsync(x->dS, p, nf, cudaMemcpyHostToDevice, st)); p += nf;
  NMC_CUDA(x, cudaStreamSynchronize(st));
  NMC_TRY(reset_chain_state(x));
  NMC_CUDA(x, cudaMemcpyAsync(x->dSign, p, C * sizeof(double), cudaMemcpyHostToDevice, st));
  p += C * sizeof(double);
  NMC_CUDA(x, cudaMemcpyAsync(x->dCounts, p, 3 * C * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  p += 3 * C * sizeof(uint64_t);
  NMC_CUDA(x, cudaMemcpyAsync(x->dDrift, p, C * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  p += C * sizeof(uint64_t);
  NMC_CUDA(x, cudaMemcpyAsync(x->dChainId, p, C * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  p += C * sizeof(int64_t);
  NMC_CUDA(x, cudaMemcpyAsync(x->dSweepBase, p, C * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  p += C * sizeof(int64_t);
  NMC_CUDA(x, cudaStreamSynchronize(st));
  NMC_TRY(ensure_series(x, ns));
  if (nser)
    NMC_CUDA(x, cudaMemcpyAsync(x->dSeries, p, nser * sizeof(double), cudaMemcpyHostToDevice, st));
  x->n_series = ns;
  x->sweep_counter = h[5];
  x->phase = h[6];
  NMC_TRY(push_counters(x));
  build_stacks(x, x->phase % 2 == 0);
  x->direct_since_build = 0;
  NMC_CUDA(x, cudaGetLastError());
  NMC_CUDA(x, cudaStreamSynchronize(st));
  x->have_fields = true;
  return NMC_OK;
}

nmc_status nmc_expk(int lattice, int Lx, int Ly, double t, double c, double* out) {
  const int N = lattice_sites(lattice, Lx, Ly);
  if (!out || !N) return NMC_EINVAL;
  std::vector<double> K, w, V, E;
  nmc_host::hopping(lattice, Lx, Ly, t, K);
  nmc_host::jacobi_eigh(N, K, w, V);
  nmc_host::expk_from_eig(N, w, V, c, E);
  std::memcpy(out, E.data(), E.size() * sizeof(double));
  return NMC_OK;
}

void nmc_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                uint32_t out[4]) {
  uint32_t c[4] = {c0, c1, c2, c3};
  philox4x32_10(c, k0, k1);
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

nmc_status nmc_philox_device(const uint32_t* d_c0, int n, uint32_t c1, uint32_t c2, uint32_t c3,
                             uint32_t k0, uint32_t k1, uint32_t* d_out, void* cuda_stream) {
  if (!d_c0 || !d_out || n < 0) return NMC_EINVAL;
  philox_batch(d_c0, n, c1, c2, c3, k0, k1, d_out, (cudaStream_t)cuda_stream);
  if (cudaGetLastError() != cudaSuccess) return NMC_ECUDA;
  if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) return NMC_ECUDA;
  return NMC_OK;
}

nmc_status nmc_drift_history(nmc_ctx* x, double* out, long long max, long long* n) {
  if (!x || !n || (max > 0 && !out)) return NMC_EINVAL;
  if (!x->configured) return fail(x, NMC_ESTATE, "nmc_drift_history before configuration");
  NMC_CUDA(x, cudaSetDevice(x->device));
  const long long have = std::min(x->n_hist, x->hist_cap);
  *n = x->n_hist;
  const long long m = std::min(have, max);
  if (m > 0) {
    std::vector<unsigned long long> bits(m);
    NMC_CUDA(x, cudaMemcpyAsync(bits.data(), x->dHist, m * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, x->st()));
    NMC_CUDA(x, cudaStreamSynchronize(x->st()));
    for (long long k = 0; k < m; ++k) std::memcpy(&out[k], &bits[k], sizeof(double));
  }
  return NMC_OK;
}

nmc_status nmc_profile(nmc_ctx* x, int enable) {
  if (!x) return NMC_EINVAL;
  x->prof = enable != 0;
  return NMC_OK;
}

nmc_status nmc_kernel_stats(nmc_ctx* x, nmc_kernel_stat* out, int max, int* n, int reset) {
  if (!x || (max > 0 && !out)) return NMC_EINVAL;
  if (x->configured) {
    NMC_CUDA(x, cudaSetDevice(x->device));
    NMC_CUDA(x, cudaStreamSynchronize(x->st()));
  }
  resolve_events(x);
  for (int c = 0; c < KC_COUNT && c < max; ++c) {
    std::memset(out[c].name, 0, sizeof out[c].name);
    std::strncpy(out[c].name, kKernelClassNames[c], sizeof out[c].name - 1);
    out[c].launches = x->launches[c];
    out[c].timed = x->timed[c];
    out[c].total_ms = x->total_ms[c];
  }
  if (n) *n = KC_COUNT;
  if (reset)
    for (int c = 0; c < KC_COUNT; ++c) x->launches[c] = x->timed[c] = 0, x->total_ms[c] = 0;
  return NMC_OK;
}

nmc_status nmc_restart_chains(nmc_ctx* x, const int* chains, const long long* global_ids,
                              int n) {
  if (!x || n < 0 || (n > 0 && (!chains || !global_ids))) return NMC_EINVAL;
  if (!x->have_fields) return fail(x, NMC_ESTATE, "nmc_restart_chains before fields were set");
  if (x->phase % 2) return fail(x, NMC_ESTATE, "nmc_restart_chains between the sweeps of a pair");
  if (n > x->chains()) return fail(x, NMC_EINVAL, "nmc_restart_chains: more chains than held");
  std::vector<char> seen(x->chains(), 0);
  for (int j = 0; j < n; ++j) {
    if (chains[j] < 0 || chains[j] >= x->chains() || seen[chains[j]] || global_ids[j] < 0 ||
        global_ids[j] > 0xffffffffll)
      return fail(x, NMC_EINVAL, "nmc_restart_chains: bad or repeated chain, or id outside 32 bits");
    seen[chains[j]] = 1;
  }
  NMC_TRY(ensure_configured(x));
  cudaStream_t st = x->st();
  if (n > 0) {
    NMC_CUDA(x, cudaMemcpyAsync(x->dList, chains, n * sizeof(int), cudaMemcpyHostToDevice, st));
    NMC_CUDA(x, cudaMemcpyAsync(x->dIds, global_ids, n * sizeof(long long),
                                cudaMemcpyHostToDevice, st));
    launch(x, KC_OTHER, [&] {
      init_fields_list(x->dS, x->Lt, x->N, (uint32_t)(x->seed & 0xffffffffu),
                       (uint32_t)(x->seed >> 32), x->dList, x->dIds, n, st);
    });
    launch(x, KC_OTHER, [&] {
      restart_chain_state(x->dList, x->dIds, n, x->chains(), x->sweep_counter, x->dChainId,
                          x->dSweepBase,
                          x->dSign, x->dCounts, x->dDrift, st);
    });
  }
  // every chain's stacks and G from its fields: at an even phase this is exactly the state
  // the last (descending) sweep left for the chains that keep running
  build_stacks(x, true);
  x->direct_since_build = 0;
  NMC_CUDA(x, cudaGetLastError());
  NMC_CUDA(x, cudaStreamSynchronize(st));
  return NMC_OK;
}

nmc_status nmc_series_range(nmc_ctx* x, long long first, long long count, double* out) {
  if (!x || first < 0 || count < 0 || (count > 0 && !out)) return NMC_EINVAL;
  if (first + count > x->n_series)
    return fail(x, NMC_EINVAL, "nmc_series_range: beyond the measured sweeps");
  if (count == 0) return NMC_OK;
  NMC_CUDA(x, cudaSetDevice(x->device));
  const size_t per = (size_t)x->chains() * 8;
  NMC_CUDA(x, cudaMemcpyAsync(out, x->dSeries + (size_t)first * per,
                              (size_t)count * per * sizeof(double), cudaMemcpyDeviceToHost,
                              x->st()));
  NMC_CUDA(x, cudaStreamSynchronize(x->st()));
  return NMC_OK;
}

void nmc_debug_fail_alloc(long long n) { g_fail_alloc_in.store(n > 0 ? n : 0); }

nmc_status nmc_debug_product(int precision, int N, int batch, int const_is_a, const double* cst,
                             const double* X, const int8_t* fields, int br, int bc, int cr,
                             int cc, double lam, const double* colscale, double* C) {
  if ((precision != NMC_SPLIT_BF16 && precision != NMC_FP32X2) || N < 2 || N > 1024 ||
      batch < 1 || batch % 2 || !cst || !X || !C || !(lam >= 0.0) ||
      std::abs(br) > 1 || std::abs(bc) > 1 || std::abs(cr) > 1 || std::abs(cc) > 1 ||
      (!const_is_a && (br || bc)))
    return NMC_EINVAL;
  const bool tc = precision == NMC_SPLIT_BF16;
  if (tc && !gemm_tc_supported(N)) return NMC_EINVAL;
  const size_t NN = (size_t)N * N, mats = NN * batch;
  std::vector<void*> bufs;
  auto dmalloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return p;
  };
  nmc_status st = NMC_OK;
  double* dC64 = (double*)dmalloc(NN * sizeof(double));
  df2* dC2 = (df2*)dmalloc(NN * sizeof(df2));
  double* dX64 = (double*)dmalloc(mats * sizeof(double));
  df2* dX2 = (df2*)dmalloc(mats * sizeof(df2));
  double* dOut = (double*)dmalloc(mats * sizeof(double));
  int8_t* dF = fields ? (int8_t*)dmalloc((size_t)(batch / 2) * N) : nullptr;
  double* dCol = colscale ? (double*)dmalloc(mats / N * sizeof(double) * 1) : nullptr;
  void* dSl = tc ? dmalloc(tc_const_elems(N) * 2) : nullptr;
  int* dExp = tc ? (int*)dmalloc(N * sizeof(int)) : nullptr;
  int* dErr = (int*)dmalloc(sizeof(int));
  alignas(64) unsigned char tmap[128];
  if (!dC64 || !dC2 || !dX64 || !dX2 || !dOut || (fields && !dF) || (colscale && !dCol) ||
      (tc && (!dSl || !dExp)) || !dErr) {
    cudaGetLastError();
    st = NMC_ENOMEM;
  }
  if (st == NMC_OK) {
    cudaMemcpy(dC64, cst, NN * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(dX64, X, mats * sizeof(double), cudaMemcpyHostToDevice);
    if (fields) cudaMemcpy(dF, fields, (size_t)(batch / 2) * N, cudaMemcpyHostToDevice);
    if (colscale) cudaMemcpy(dCol, colscale, mats / N * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemset(dErr, 0, sizeof(int));
    split_to_df(dC64, dC2, (long long)NN, 0);
    split_to_df(dX64, dX2, (long long)mats, 0);
    DfGemmArgs g;
    g.M = g.N = g.K = N;
    g.batch = batch;
    g.A = const_is_a ? dC2 : dX2; g.sA = const_is_a ? 0 : (long long)NN; g.lda = N;
    g.B = const_is_a ? dX2 : dC2; g.sB = const_is_a ? (long long)NN : 0; g.ldb = N;
    g.Cd = dOut; g.sC = (long long)NN; g.ldc = N;
    g.colscale = dCol; g.sColscale = N;
    g.fstride = N;
    g.ns = 2;
    if (fields) {
      g.bfields = dF; g.br = br; g.bc = bc;
      g.cfields = dF; g.cr = cr; g.cc = cc;
    }
    for (int m = -2; m <= 2; ++m) {
      const double v = std::exp(m * lam);
      g.e[m + 2].hi = (float)v;
      g.e[m + 2].lo = (float)(v - (double)(float)v);
    }
    if (tc) {
      if (!tc_prepare_const(dC64, N, const_is_a ? 0 : 1, dSl, dExp, tmap, 0)) {
        st = NMC_ECUDA;
      } else {
        g.oz_const = dSl;
        g.oz_const_exp = dExp;
        gemm_tc(g, const_is_a != 0, tmap, dErr, 0);
      }
    } else {
      gemm_df(g, 0);
    }
    int err = 0;
    if (st == NMC_OK) {
      if (cudaDeviceSynchronize() != cudaSuccess ||
          cudaMemcpy(&err, dErr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(C, dOut, mats * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        st = NMC_ECUDA;
      } else if (err) {
        st = NMC_ETIMEOUT;
      }
    }
  }
  for (void* p : bufs) cudaFree(p);
  return st;
}

nmc_status nmc_graph_stats(const nmc_ctx* x, long long* recorded, long long* replayed) {
  if (!x) return NMC_EINVAL;
  if (recorded) *recorded = x->graphs_recorded;
  if (replayed) *replayed = x->graphs_replayed;
  return NMC_OK;
}

const char* nmc_last_error(const nmc_ctx* x) { return x ? x->err.c_str() : "null context"; }

const char* nmc_version(void) { return "libnmc 0.1 (sm_103a)"; }

int nmc_debug_build(void) {
#ifdef NMC_DEBUG
  return 1;
#else
  return 0;
#endif
}

unsigned int nmc_debug_checks(void) { return debug_failed(); }

void nmc_destroy(nmc_ctx* x) {
  if (!x) return;
  if (x->device >= 0) cudaSetDevice(x->device);
  if (!x->recs.empty()) {
    cudaStreamSynchronize(x->st());
    resolve_events(x);
  }
  for (cudaEvent_t e : x->event_pool) cudaEventDestroy(e);
  x->event_pool.clear();
  free_all(x);
  if (x->cap_stream) cudaStreamDestroy(x->cap_stream);
  delete x;
}

}  // extern "C"
