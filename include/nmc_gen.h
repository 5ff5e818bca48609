/*
 * nmc_gen.h -- C ABI of libnmc's network initialization: the generative network of
 * network-initialized Monte Carlo (arXiv 2106.00712, Algorithm 1 steps 2-3), trained on
 * observables of short Markov chains, whose generated configurations start the DQMC
 * chains of nmc.h (Algorithm 1 step 4, nmc_generate mode 1).
 *
 * Network (SM Sec. II, Hubbard model): a random +-1 input configuration z of shape
 * z0 x z1 x z2, then transposed 3D convolutions with stride 1 and valid padding (each axis
 * grows by k - 1), each followed by a sigmoid: c1 filters of size k1, then one filter of
 * size k2. The output p (values in (0,1)) has shape L_tau x A x B with A*B = N, A = 2 Lx
 * (honeycomb) or Lx (square), B = Ly; p[l][a][b] belongs to site i = a + A*b at slice l.
 * The paper's honeycomb network: z 10x2x2, 20 filters 16x6x3, 1 filter 36x6x3, output
 * 60x12x6 (L = 6, beta = 6, dtau = 0.1).
 * Parameter layouts (row-major, float32): W1 [1][c1][k1_0][k1_1][k1_2], b1 [c1],
 * W2 [c1][1][k2_0][k2_1][k2_2], b2 [1]; out[co][o] = b[co] + sum_ci sum_{i+k=o} in[ci][i] W[ci][co][k].
 *
 * Loss (Eq. 4): sum over a batch of w1 (S(G_l) - S_l)^2 + w2 (E_k(G_l) - E_k,l)^2, where the
 * l-th generated configuration enters the determinant weight with continuous fields
 * x = 2p - 1 (the footnote to Algorithm 1: B_l = e^{-dtau K} e^{sigma lam diag x(.,l)}),
 * S = S(Gamma) (honeycomb) or S(pi,pi) (square) and E_k the kinetic energy per site are the
 * sweep's estimators on the symmetric-Trotter G~ at slice 0 (the same estimators as
 * nmc_measure's s_pipi and ekin), and (S_l, E_k,l) are the l-th training sample's values.
 * Its gradient with respect to x is exact: dLoss/dx(i,l) = -lam sum_sigma sigma
 * [H(0,l)^T Gbar G(l,0)^T]_ii with G(l,0) = B_{l-1}...B_0 G_0, H(0,l) = (I - G_0)(B_{l-1}...B_0)^{-1}
 * and Gbar = dLoss/dG_0, all formed from UDV stacks with the split-D recompute (FP64).
 *
 * Random numbers: Philox4x32-10 keyed by the generator's seed. Input z: -1 iff the top bit
 * of word 0 at counter (element, sample, stream, 2); Bernoulli: s = +1 iff word 0 * 2^-32 < p
 * at counter (l*N + i, sample, stream, 3). Training uses stream 0 (sample n of the training
 * set has input z(n, 0)); generation uses stream 1. Initial weights: Glorot uniform from
 * word 0 at counter (index, layer, 0, 4), biases 0. Adam (learning rate lr, beta1 = 0.9,
 * beta2 = 0.999, epsilon = 1e-7; SM Sec. II).
 *
 * Conventions as in nmc.h: every call returns nmc_status; a context is not thread-safe;
 * device work runs on the stream given at creation; device pointers must be valid on the
 * context's device; host buffers are copied.
 */
#ifndef NMC_GEN_H
#define NMC_GEN_H

#include "nmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nmc_gen nmc_gen;

typedef struct {
  int z[3];    /* input shape                                         paper: 10, 2, 2   */
  int c1;      /* filters of the first layer                          paper: 20         */
  int k1[3];   /* first-layer kernel                                  paper: 16, 6, 3   */
  int k2[3];   /* second-layer kernel (one filter)                    paper: 36, 6, 3   */
} nmc_gen_arch;

/* Fill `arch` with the paper's honeycomb network (SM Sec. II). */
void nmc_gen_paper_arch(nmc_gen_arch* arch);

/* Create a generator for the lattice problem of nmc_create (same arguments and checks)
 * with the given architecture, Glorot-initialized from `seed`. max_batch: configurations
 * per loss evaluation (device workspace ~ max_batch * 2 * (2 nb + 10) * N^2 doubles;
 * larger requests are processed in chunks). NMC_EINVAL: lattice arguments as nmc_create,
 * arch sizes < 1, output shape != (L_tau, A, B), max_batch < 1, out == NULL.
 * NMC_ENOMEM / NMC_ECUDA on allocation failure. */
nmc_status nmc_gen_create(int lattice, int Lx, int Ly, double t, double U, double beta,
                          double dtau, int n_wrap, const nmc_gen_arch* arch, uint64_t seed,
                          int max_batch, void* cuda_stream, nmc_gen** out);

/* Host copies of the parameters (float32, layouts above); NULL pointers are skipped. */
nmc_status nmc_gen_get_params(const nmc_gen* g, float* W1, float* b1, float* W2, float* b2);
/* Set the parameters from host arrays (all four required) and reset the Adam state. */
nmc_status nmc_gen_set_params(nmc_gen* g, const float* W1, const float* b1, const float* W2,
                              const float* b2);

/* Generator output for samples n0 .. n0+n-1 of input stream `stream` (0 training,
 * 1 generation): device d_p, float32 [n][L_tau][A][B]. */
nmc_status nmc_gen_probs(nmc_gen* g, long long n0, int n, int stream, float* d_p);

/* Bernoulli +-1 fields from the generator for samples n0 .. n0+n-1 of `stream`: device
 * d_fields, int8 [n][L_tau][N] (the layout of nmc_set_fields_device). */
nmc_status nmc_gen_sample_fields(nmc_gen* g, long long n0, int n, int stream,
                                 int8_t* d_fields);

/* Observables of configurations with fields d_x (device, double [n][L_tau][N], any real
 * values; +-1 for Markov-chain samples): d_obs (device, double [n][2]) = (S, E_k). */
nmc_status nmc_gen_observables(nmc_gen* g, const double* d_x, int n, double* d_obs);

/* Observables measured directly on generated configurations (the footnote to Algorithm 1:
 * x = 2p - 1) for samples n0 .. n0+n-1 of `stream`: d_obs (device, double [n][2]). */
nmc_status nmc_gen_generated_observables(nmc_gen* g, long long n0, int n, int stream,
                                         double* d_obs);

/* Eq. 4 per configuration and its exact gradient: d_targets (device, double [n][2] =
 * (S_l, E_k,l)); outputs d_loss (device, double [n], may be NULL) and d_grad (device,
 * double [n][L_tau][N], may be NULL). */
nmc_status nmc_gen_loss_grad(nmc_gen* g, const double* d_x, int n, const double* d_targets,
                             double w1, double w2, double* d_loss, double* d_grad);

/* One Adam step on the batch of training samples `ids` (host, n entries; sample id picks
 * input z(id, 0)) against targets (host, double [n][2] = (S, E_k)): forward, Eq. 4 loss,
 * backward, update. *loss_out (host, may be NULL) receives the batch loss. */
nmc_status nmc_gen_train_step(nmc_gen* g, const long long* ids, int n, const double* targets,
                              double w1, double w2, double lr, double* loss_out);

/* Train on n samples (targets host [n][2], sample k paired with input z(k, 0)) for
 * `epochs` passes in a random order (Fisher-Yates with Philox uniforms at counter
 * (k, epoch, 0, 5), epoch counted since creation or the last nmc_gen_set_params, so that
 * successive calls continue one schedule), `batch` samples per step (the last step of an
 * epoch may be smaller). NMC_ENUMERIC if a configuration's density departs from 1 by
 * more than 1e-6 (a failed stabilization; the message names the batch), before the
 * update of that step.
 * w1, w2 <= 0 select the inverse variances of the targets. epoch_loss (host, may be NULL):
 * mean loss per sample of each epoch. */
nmc_status nmc_gen_train(nmc_gen* g, const double* targets, int n, int epochs, int batch,
                         double lr, double w1, double w2, double* epoch_loss);

/* Bound the global norm of each step's gradient (over all parameters) by max_norm before
 * the Adam update (0, the default: no bound; the paper states none). Single-configuration
 * estimators are unbounded, and a generator driven into saturation meets configurations
 * whose loss gradient is many orders above the typical one. */
nmc_status nmc_gen_set_clip(nmc_gen* g, double max_norm);

/* Adam steps taken since creation or the last nmc_gen_set_params. */
long long nmc_gen_steps(const nmc_gen* g);

const char* nmc_gen_last_error(const nmc_gen* g);
void nmc_gen_destroy(nmc_gen* g);

#ifdef __cplusplus
}
#endif

#endif /* NMC_GEN_H */
