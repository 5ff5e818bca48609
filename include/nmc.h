/*
 * nmc.h -- C ABI of libnmc: the determinant quantum Monte Carlo (DQMC) sweep used by
 * network-initialized Monte Carlo (arXiv 2106.00712), run on one NVIDIA GB300 (sm_103a).
 *
 * The operation is the Markov chain over the discrete Hubbard-Stratonovich field s(i,l)
 * of the half-filled Hubbard model (Eq. 3) on a periodic square or honeycomb lattice, with
 * weight prod_sigma Det[I + B^sigma_L ... B^sigma_1] (Supplemental Material Sec. I.2,
 * partition function in determinant form) and B^sigma_l = e^{-dtau K} e^{sigma lam
 * diag s(.,l)}, cosh lam = e^{dtau U/2} (Sec. I.2, discrete HS transform). One sweep gives
 * every s(i,l) one Metropolis flip attempt (Sec. I.3, definition of a sweep); chains are
 * independent, one per initial configuration (Algorithm 1, step 4).
 *
 * Conventions shared by every call
 *  - Every call returns nmc_status; nothing aborts or throws across the ABI. On failure
 *    nmc_last_error(ctx) holds a one-line reason (until the next failing call).
 *  - The caller owns every buffer it passes; the library copies what it needs. The
 *    library owns the context and all device memory it allocates (stream-ordered
 *    cudaMallocAsync on the context stream), except nmc_green_noalloc, which allocates none.
 *  - Lattices: the nmc_lattice enum, square or honeycomb. The generator of network initialization
 *    (Algorithm 1, steps 2-3) has its own header, nmc_gen.h; nmc_generate mode 1 uses it.
 *  - Device work is ordered on the context's CUDA stream (nmc_options.cuda_stream, NULL =
 *    the legacy default stream). Calls that return host data synchronise that stream.
 *  - A context is not thread-safe: serialise calls on one context.
 *  - Layouts: fields are int8 [chain][l][i], l = 0..L_tau-1 the imaginary-time slice,
 *    i = x + Lx*y the site; values +1 or -1. Matrices are row-major N x N doubles.
 *  - Random numbers: Philox4x32-10 keyed by seed (key = low, high 32 bits), counter
 *    (l*N + i, sweep, chain, tag); tag 0 = flip uniform u = x0 * 2^-32, accepted iff
 *    u < |R|; tag 1 = initial field, s = -1 iff the top bit of x0 is set. "chain" is the
 *    global chain index (local index + nmc_options.chain_offset), so results do not
 *    depend on how chains are split over processes.
 */
#ifndef NMC_H
#define NMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nmc_ctx nmc_ctx;

typedef enum {
  NMC_OK = 0,
  NMC_EINVAL = 1,    /* invalid argument or size; nothing changed                        */
  NMC_ENOMEM = 2,    /* device or host allocation failed                                 */
  NMC_ECUDA = 3,     /* a CUDA call failed (no device, launch error, ...)                */
  NMC_ENUMERIC = 4,  /* non-finite G or stabilization drift above nmc_options.drift_tol  */
  NMC_ETIMEOUT = 5,  /* a bounded device-side wait expired                               */
  NMC_ESTATE = 6     /* call out of order (e.g. nmc_sweep before fields are set)         */
} nmc_status;

/* Arithmetic of the propagation steps. Ratios, acceptance, UDV stabilization, the
 * recomputed G and the measurements are always FP64. */
typedef enum {
  NMC_FP64 = 0,       /* flips, delayed updates, wraps and stack products in FP64         */
  NMC_FP32 = 1,       /* flips, delayed updates and wraps in FP32 (FP32 accumulation)     */
  NMC_SPLIT_BF16 = 2, /* compensated: G, flips and delayed-update panels in FP32 pairs
                         (error-free products and sums); every wrap, stack and measurement
                         product on the BF16 tensor cores by exact integer slicing (each
                         operand cut into 7 integer BF16 slices, slice products exact in FP32
                         accumulators, ~2^-49 of the row/column maxima), and the rank-k fold
                         too where that is faster; QR, recompute, ratios, measurement FP64 */
  NMC_TF32X3 = 3,     /* not built (NMC_EINVAL): three TF32 products accumulated in FP32 give
                         FP32-class products, which cannot hold the 1e-5 drift bar here   */
  NMC_FP32X2 = 4      /* compensated as NMC_SPLIT_BF16, with every product and fold in FP32
                         pairs on the FP32 SIMT pipes (no tensor cores)                   */
} nmc_precision;

/* Lattices of Eq. 3 (both periodic and bipartite; K_ij = -t per nearest-neighbour pair,
 * set once, so a length-2 direction has one bond and a length-1 direction none).
 *   NMC_SQUARE:    Lx x Ly sites, i = x + Lx*y; sublattice parity (x + y) mod 2.
 *   NMC_HONEYCOMB: Lx x Ly cells of two sites (the honeycomb lattice of the paper's
 *                  Hubbard runs, "Models" and SM Sec. II.1: L x L cells, 2 L^2 sites),
 *                  i = 2 (x + Lx*y) + sub; the A site (sub 0) of cell (x,y) bonds to the
 *                  B sites (sub 1) of cells (x,y), (x-1,y), (x,y-1); parity = sub.
 * The estimators' staggered sign p_i = (-1)^parity: S(pi,pi) on the square lattice and
 * the antiferromagnetic S(Gamma) (Eq. 4 with opposite signs on A and B) on the honeycomb. */
typedef enum { NMC_SQUARE = 0, NMC_HONEYCOMB = 1 } nmc_lattice;

typedef struct {
  int n_chains;          /* independent chains held by this context (>= 1)       default 1  */
  int delay_k;           /* accepted flips folded per rank-k delayed update (>= 1) def. 16   */
  int precision;         /* nmc_precision                                        default 0  */
  double drift_tol;      /* NMC_ENUMERIC if max|G_wrapped - G_recomputed| exceeds this;
                            <= 0 selects 1e-6 (FP64), 1e-3 (FP32), 1e-5 (SPLIT_BF16,
                            FP32X2)                                              default 0 */
  long long chain_offset;/* global index of local chain 0 (Philox counter word 2) def. 0   */
  void* cuda_stream;     /* cudaStream_t for all device work                     def. NULL */
  int ph_symmetric;      /* 1: propagate spin up only; at half filling on the bipartite
                            lattice G_dn = I - P G_up^T P (P = diag of sublattice signs) exactly,
                            R_dn = 1 + Delta_dn G_up_ii, and G~_dn follows the same way.
                            Same chain, half the work.                           default 0  */
  int sweep_graphs;      /* 1: after the first sweep of each direction, record one sweep as a
                            CUDA graph and replay it (one launch per sweep instead of one per
                            kernel; the same kernels with the same arguments, so the results
                            are identical); not while profiling or replaying decisions.
                            0: launch every kernel directly.                     default 1  */
  int stab_pairs;        /* compensated precisions only (else NMC_EINVAL). 1: the products of
                            the stabilization (the T updates of the UDT stacks and the three
                            products of the recompute) take FP64 operands and give FP64
                            results, but accumulate in FP32 pairs on the FP32 pipe (error-free
                            products and sums, ~2^-44 of the sum of |a_ik b_kj|) instead of FP64
                            FMAs; operands must lie within the FP32 range, which the stacks'
                            D-split keeps them in. The QR and the Gauss-Jordan solve stay FP64.
                            0: FP64 (SIMT FP64 pipe).                            default 0  */
} nmc_options;

typedef struct {
  double mean;
  double err;            /* standard error: across chains (>= 2 chains) or over 10 bins of
                            the per-sweep series (1 chain); 0 when not estimable          */
} nmc_est;

typedef struct {
  nmc_est energy;        /* <H>/N of Eq. 3 (sign-weighted)                                  */
  nmc_est ekin;          /* kinetic part: -(1/N) sum_sigma Tr(K G~^sigma)                   */
  nmc_est double_occ;    /* (1/N) sum_i <n_i,up n_i,dn>                                    */
  nmc_est s_pipi;        /* S(Q) at Q = (pi,pi), S(Q) as defined with Eq. 4               */
  nmc_est density;       /* (1/N) sum_i,sigma <n_i,sigma>                                  */
  nmc_est sign;          /* average configuration sign                                     */
  double accept;         /* accepted / attempted flips                                     */
  double max_drift;      /* max over stabilizations of max|G_wrapped - G_recomputed|       */
  long long n_meas;      /* measurements accumulated (per chain)                           */
  long long n_disagree;  /* replay sweeps: attempts whose own decision differed            */
} nmc_obs;

/* Create a context for the periodic lattice (nmc_lattice, Lx x Ly) with hopping t and
 * interaction U (Eq. 3) at inverse temperature beta, Trotter step dtau (Sec. I.2:
 * L_tau = beta/dtau slices), stabilization every n_wrap slices, Philox seed `seed`.
 * Host-side set-up (K, e^{-+dtau K}, e^{-+dtau K/2} by a Jacobi eigensolver, lam) happens
 * here; device memory is allocated by nmc_configure / the first call that needs it.
 * lattice: nmc_lattice; N = Lx*Ly (square) or 2*Lx*Ly (honeycomb).
 * NMC_EINVAL: unknown lattice, N < 2, square with Lx or Ly odd and > 1 (must be
 * bipartite), t <= 0,
 * U < 0, beta <= 0, dtau <= 0, beta/dtau not an integer to 1e-9 relative,
 * L_tau % n_wrap != 0, n_wrap < 1, N > 1024, out == NULL. *out is NULL on failure. */
nmc_status nmc_create(int lattice, int Lx, int Ly, double t, double U, double beta,
                      double dtau, int n_wrap, uint64_t seed, nmc_ctx** out);

/* Set options (copied). Allowed before the first nmc_set_fields / nmc_generate only
 * (NMC_ESTATE after). opts == NULL restores the defaults. Allocates device memory:
 * NMC_ENOMEM / NMC_ECUDA on failure. */
nmc_status nmc_configure(nmc_ctx* ctx, const nmc_options* opts);

/* Fill `opts` with the defaults listed in nmc_options. */
void nmc_default_options(nmc_options* opts);

/* Set every chain's field from host memory (int8 [n_chains][L_tau][N], n = element
 * count, values +-1: NMC_EINVAL otherwise), then build the left UDV stack and the
 * equal-time G_0 = (I + B_{L-1}...B_0)^{-1} of each spin. Resets acceptance counters,
 * accumulators, drift and the sweep direction (next sweep ascends in l); the sweep
 * counter (Philox word 1) keeps counting. */
nmc_status nmc_set_fields(nmc_ctx* ctx, const int8_t* s, size_t n);

/* As nmc_set_fields with a device pointer (read on the context stream; values are not
 * validated -- entries other than +1 are treated as -1). */
nmc_status nmc_set_fields_device(nmc_ctx* ctx, const int8_t* d_s, size_t n);

/* Generate initial fields on the device. mode 0: uniform random from Philox (tag 1),
 * ignoring `model`. mode 1: configurations from a trained generator (Algorithm 1, step 3),
 * `model` an nmc_gen* (include/nmc_gen.h) for the same N and L_tau; chain c gets the
 * Bernoulli fields of generation sample chain_offset + c. Other modes: NMC_EINVAL.
 * Then as nmc_set_fields. */
nmc_status nmc_generate(nmc_ctx* ctx, int mode, const void* model);

/* Run n_sweeps sweeps on every chain (n_sweeps >= 0). Sweeps alternate direction
 * (ascending l, then descending); within a slice sites go i = 0..N-1. G is recomputed
 * from the UDV stacks every n_wrap slices; if measure != 0 the estimators are
 * accumulated at each recompute on the symmetric-Trotter G~ = e^{dtau K/2} G e^{-dtau K/2}.
 * Returns NMC_ENUMERIC if the drift is non-finite or above drift_tol (state is kept). */
nmc_status nmc_sweep(nmc_ctx* ctx, int n_sweeps, int measure);

/* As nmc_sweep, but only enqueues the work on the context stream and returns; the drift
 * check happens at nmc_sync. Host state (sweep counter, direction) advances immediately,
 * so further calls queue behind. Used by the serving loop to keep many contexts' work in
 * flight on different streams at once. */
nmc_status nmc_sweep_async(nmc_ctx* ctx, int n_sweeps, int measure);

/* *idle = 1 if all work enqueued on the context stream has finished, else 0. */
nmc_status nmc_query(nmc_ctx* ctx, int* idle);

/* Wait for the context stream, then check the drift as nmc_sweep does. */
nmc_status nmc_sync(nmc_ctx* ctx);

/* Host only: device bytes nmc_configure allocates for this problem and these options
 * (opts NULL = defaults), excluding the growable measurement series (8 doubles per chain
 * per measured sweep). For admission control. */
nmc_status nmc_footprint(int lattice, int Lx, int Ly, double t, double U, double beta,
                         double dtau, int n_wrap, const nmc_options* opts, size_t* bytes);

/* One sweep that applies the given accept decisions instead of its own
 * (uint8 [n_chains][L_tau][N], nonzero = flip; n = element count). The library still
 * evaluates its own ratio for every attempt and counts disagreements
 * (nmc_obs.n_disagree). Used to compare precisions on identical trajectories. */
nmc_status nmc_sweep_replay(nmc_ctx* ctx, const uint8_t* accept, size_t n, int measure);

/* Per-sweep accumulators of the measuring sweeps since the last reset (host out, double
 * [n][n_chains][8], n = min(max_sweeps, *n_sweeps)): for each measured sweep and chain the
 * sums over that sweep's L_tau/n_wrap measurements of sign * (energy, ekin, double_occ,
 * s_pipi, density), the sum of the signs, and two zeros; the sweep's estimate of an
 * observable is entry k / entry 5. *n_sweeps receives the number recorded. */
nmc_status nmc_series(nmc_ctx* ctx, double* out, long long max_sweeps, long long* n_sweeps);

/* Per-sweep accumulators of measured sweeps first .. first + count - 1 (host out, double
 * [count][n_chains][8], the layout of nmc_series). NMC_EINVAL beyond the recorded sweeps. */
nmc_status nmc_series_range(nmc_ctx* ctx, long long first, long long count, double* out);

/* Start the listed chains afresh while the others keep running (the admission step of the
 * serving loop, which packs independent requests into one context). chains: n distinct
 * local chain indices; global_ids: their new global indices (Philox counter word 2, < 2^32).
 * Each listed chain gets the Philox initial field of its global index (tag 1), its sweep
 * numbering (Philox counter word 1) restarts at 0 with the next sweep, its sign is set to +1
 * and its acceptance counts and drift are cleared; its per-sweep accumulators are those of
 * the sweeps from then on. Then the UDV stacks and G of every chain are rebuilt from the
 * fields, which reproduces the running chains' state exactly. So a restarted chain follows
 * the same trajectory as the same global chain started alone in a fresh context. Only between
 * sweep pairs: NMC_ESTATE after an odd number of sweeps since the fields were set (the next
 * sweep must ascend), or before any fields; NMC_EINVAL for bad or repeated chains. Device
 * work on the context stream; returns when it is done. */
nmc_status nmc_restart_chains(nmc_ctx* ctx, const int* chains, const long long* global_ids,
                              int n);

/* Reduce the accumulators. per_chain: array of n_chains (or NULL); pooled: one (or
 * NULL). Pooled means are averages of per-chain means; errors as in nmc_est. */
nmc_status nmc_measure(nmc_ctx* ctx, nmc_obs* per_chain, nmc_obs* pooled);

/* Copy every chain's current field to host memory (int8 [n_chains][L_tau][N]). */
nmc_status nmc_get_fields(nmc_ctx* ctx, int8_t* s, size_t n);

/* Copy the current equal-time G of one chain and spin (0 = up, 1 = down) to host
 * memory (N x N row-major). After an even number of sweeps since the fields were set,
 * G sits at slice 0, after an odd number at slice L_tau (equal to slice 0 cyclically).
 * In FP32, SPLIT_BF16 and FP32X2 mode the propagated G is widened to double. */
nmc_status nmc_get_green(nmc_ctx* ctx, int chain, int spin, double* G);

/* Sizes: N, L_tau, n_chains, effective delay (after the shared-memory clamp). */
nmc_status nmc_get_dims(const nmc_ctx* ctx, int* N, int* L_tau, int* n_chains, int* delay_k);

/* Checkpoint: all state needed for an exact resume (fields, sweep counter, direction,
 * accumulators, counters). buf == NULL: *n receives the size. NMC_EINVAL if *n is too
 * small. nmc_restore rebuilds the UDV stacks from the fields. */
nmc_status nmc_checkpoint(nmc_ctx* ctx, void* buf, size_t* n);
nmc_status nmc_restore(nmc_ctx* ctx, const void* buf, size_t n);

/* Host-only helper (no GPU needed): e^{c K} for the hopping matrix K of an nmc_lattice
 * (K_ij = -t on nearest neighbours), by the library's Jacobi eigensolver. out: N x N.
 * NMC_EINVAL for the sizes nmc_create rejects. */
nmc_status nmc_expk(int lattice, int Lx, int Ly, double t, double c, double* out);

/* Host-only helper: Philox4x32-10 block function; out[4] = words of counter
 * (c0,c1,c2,c3) under key (k0,k1). Same code as the device generator's host twin. */
void nmc_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                uint32_t k1, uint32_t out[4]);

/* Device generator check: out[4*j + w] = word w of Philox(counter (c0[j], c1, c2, c3),
 * key (k0, k1)) for j < n, computed by the device code the sweep uses. Device out. */
nmc_status nmc_philox_device(const uint32_t* d_c0, int n, uint32_t c1, uint32_t c2,
                             uint32_t c3, uint32_t k0, uint32_t k1, uint32_t* d_out,
                             void* cuda_stream);

/* Drift history: out[k] = max over chains of max|G_propagated - G_recomputed| at the k-th
 * stabilization since the fields were set (first `max` entries; the library keeps the
 * first 4096). *n receives the number of stabilizations so far. Synchronises the stream. */
nmc_status nmc_drift_history(nmc_ctx* ctx, double* out, long long max, long long* n);

/* Per-kernel accounting (tracing). Every library kernel launch is counted by class
 * ("gemm", "flip", "qrp", "solve", "measure", "other", "gemm_df", "gemm_tc", "gemm_pair"). With
 * profiling enabled, each
 * launch is also bracketed by CUDA events on the context stream, and nmc_kernel_stats
 * reports the summed device time of the bracketed launches. */
typedef struct {
  char name[16];
  long long launches;    /* launches since the last reset                               */
  long long timed;       /* launches bracketed by events                                */
  double total_ms;       /* summed event time of the bracketed launches                 */
} nmc_kernel_stat;

/* Enable (1) or disable (0) event bracketing of launches. */
nmc_status nmc_profile(nmc_ctx* ctx, int enable);

/* Synchronise the stream and write up to `max` entries (one per kernel class) to `out`;
 * *n receives the number of classes. reset != 0 clears the counters afterwards. */
nmc_status nmc_kernel_stats(nmc_ctx* ctx, nmc_kernel_stat* out, int max, int* n, int reset);

/* Sweep graphs (nmc_options.sweep_graphs): *recorded = graphs recorded, *replayed = sweeps
 * run by replaying a recorded graph, since the context was created. Either pointer may be
 * NULL. Host counters only; no device work. */
nmc_status nmc_graph_stats(const nmc_ctx* ctx, long long* recorded, long long* replayed);

/* Equal-time Green's functions G_0 = (I + B_{L-1}...B_0)^{-1} of each chain and spin from
 * caller-given fields, WITHOUT allocating: no cudaMalloc, cudaFree or other allocating
 * call. The paper has no counterpart; this exists for callers that cannot allocate device
 * memory when they need G (a caller whose memory pool or arena owns the device budget, or
 * a runtime that forbids allocator calls after start-up). Computes what nmc_set_fields
 * computes for G, with the same kernels in the same order.
 *   N, L_tau, n_wrap: sites, slices, stabilization interval (L_tau % n_wrap == 0);
 *   lam: HS coupling, cosh(lam) = e^{dtau U / 2};
 *   d_expK_m: device, N x N row-major e^{-dtau K} (e.g. from nmc_expk(..., -dtau, ...));
 *   d_fields: device, int8 [n_chains][L_tau][N], values +-1;
 *   d_G: device output, [n_chains][2][N][N] row-major (spin 0 = up).
 * Work is enqueued on cuda_stream (NULL = legacy default stream); outputs are valid once
 * the stream reaches that point. Scratch: a fixed array of 4,194,304 doubles (32 MiB) in
 * the library, held by every GPU that loads it until exit. Chains are processed in chunks
 * that fit; one chain needs 20 N^2 + 4 N doubles (24 N^2 + 4 N when N > 111), so
 * NMC_EINVAL is returned, before any work is enqueued, when that exceeds the array
 * (N > 409), and for invalid arguments. Each call made outside stream capture looks up
 * the array's device address (cudaGetSymbolAddress) in the current device's context and
 * caches it for that device; a call made while cuda_stream is being captured uses the
 * cached address. A device reset (cudaDeviceReset) invalidates that address, so after a
 * reset, and before the first capture on a device, make one call outside capture (a call
 * under capture with no cached address returns NMC_ECUDA). NMC_ECUDA is also returned,
 * with nothing enqueued, when a CUDA error is already pending on entry, and at the first
 * failed launch. Every call shares the one array and overwrites it: calls whose work
 * overlaps on the GPU (other streams, other threads) race -- serialise them. */
nmc_status nmc_green_noalloc(int N, int L_tau, int n_wrap, double lam, const double* d_expK_m,
                             const int8_t* d_fields, int n_chains, double* d_G,
                             void* cuda_stream);

/* Arithmetic-pipe probe (measurement): launch blocks x threads threads on cuda_stream,
 * each running 8 independent fused multiply-add chains for `iters` rounds in FP64 (kind 0)
 * or FP32 (kind 1), and store one value per thread to d_out (device, blocks * threads
 * elements of that type). Work: blocks * threads * iters * 16 flop. Timed by the caller
 * with events on the same stream, it gives the measured FP64 / FP32 SIMT peak that the
 * roofline of the SIMT kernels is quoted against. Kinds 2 (FP64) and 3 (FP32) run the same
 * loop on one lane per warp only: the same warp instructions with 1/32 of the work, which
 * shows whether a pipe's cost is per warp instruction or per active lane. NMC_EINVAL for
 * bad sizes. */
nmc_status nmc_fma_probe(int kind, int blocks, int threads, int iters, void* d_out,
                         void* cuda_stream);

/* Testing hook (host only): make the n-th device allocation of any context from now on
 * fail as if the device were out of memory (the call that made it returns NMC_ENOMEM and
 * frees what it had allocated when the context is destroyed); n <= 0 disarms. Lets callers
 * test their handling of NMC_ENOMEM without exhausting a shared GPU's memory. */
void nmc_debug_fail_alloc(long long n);

/* Testing hook: one batched product of the compensated modes, as the sweep runs it, on host
 * data (device memory is allocated and freed inside; synchronous). C[b] = cst X[b]
 * (const_is_a = 1) or X[b] cst, for b < batch (even: matrix b belongs to chain b/2, spin
 * b%2, sigma = +1 for spin 0 and -1 for spin 1). cst: N x N; X, C: [batch][N][N] row-major
 * doubles; X is rounded to FP32 pairs first, as the sweep holds G. With `fields`
 * (int8 [batch/2][N], +-1): the chain operand's element (r,c) is multiplied by
 * e^{sigma lam (br s_r + bc s_c)} before the product and output element (r,c) by
 * e^{sigma lam (cr s_r + cc s_c)} after it (br..cc in {-1,0,1}; br, bc only with the
 * constant on the left, the one form the sweep uses). With `colscale`
 * ([batch][N]): output column c of matrix b times colscale[b][c]. precision: NMC_SPLIT_BF16
 * (tcgen05 tensor cores, exact slicing) or NMC_FP32X2 (FP32 pairs on the SIMT pipes).
 * NMC_EINVAL for other arguments, NMC_ETIMEOUT if a bounded device wait expired. */
nmc_status nmc_debug_product(int precision, int N, int batch, int const_is_a, const double* cst,
                             const double* X, const int8_t* fields, int br, int bc, int cr,
                             int cc, double lam, const double* colscale, double* C);

const char* nmc_last_error(const nmc_ctx* ctx);
const char* nmc_version(void);

/* The bounds-checked build (libnmc_debug.so, compiled with NMC_DEBUG): its kernels check
 * their key indices (pivot rows, panel slots, tile offsets, output entries, chain lists)
 * and, on a failed check, skip the access and record the check's id; the calls that run
 * kernels then return NMC_ECUDA naming it. nmc_debug_build: 1 in that build, 0 otherwise.
 * nmc_debug_checks: the first failed check's id since the library was loaded (0: none;
 * always 0 outside that build). Host only, synchronous. */
int nmc_debug_build(void);
unsigned int nmc_debug_checks(void);
void nmc_destroy(nmc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* NMC_H */
