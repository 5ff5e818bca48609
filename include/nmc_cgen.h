/*
 * nmc_cgen.h -- C ABI of libnmc's convolutional field generator: a second network for the
 * initialization step of network-initialized Monte Carlo (arXiv 2106.00712, Algorithm 1
 * steps 2-3), beside the paper's own network (nmc_gen.h). It maps noise z ~ N(0,1) of the
 * field's shape to independent Bernoulli logits, one per field entry s(i, l), and is
 * trained by maximum likelihood on fields the DQMC itself produces; its samples start DQMC
 * chains through nmc_set_fields_device (Algorithm 1 step 4).
 *
 * Network: four periodic 3D convolutions with 3 x 3 x 3 kernels over the field's shape
 * (L_tau, Ly, Lx) -- x fastest, so entry p = l N + (x + Lx y) is field entry (i, l) of
 * nmc_set_fields -- with channels 1 -> C -> C -> C -> 1 and a ReLU after the first three:
 *     conv(h)[co][p] = b[co] + sum_ci sum_{d in {-1,0,1}^3} W[co][ci][d + 1] h[ci][p + d]
 * (indices periodic in all three axes). Every convolution reads BF16 operands (the noise,
 * the hidden activations, the weights; in the backward pass the gradient flowing in) and
 * accumulates in FP32; master weights, their gradients and Adam's moments are FP32.
 * Loss of fields s given noise z: mean over samples and entries of softplus(l) - y l with
 * y = (1 + s) / 2 (the Bernoulli negative log-likelihood).
 *
 * Parameters, one flat FP32 array in this order: W0 [C][1][3][3][3], b0 [C],
 * W1 [C][C][3][3][3], b1 [C], W2 [C][C][3][3][3], b2 [C], W3 [1][C][3][3][3], b3 [1].
 * Initial weights: Glorot uniform (bound sqrt(6 / (27 (Cin + Cout)))) from word 0 of
 * Philox4x32-10 at counter (index, layer, 0, 7) under the key `seed`, biases 0.
 *
 * Random numbers (Philox4x32-10, key = seed): noise entry p of sample n in stream st is
 * sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller) with u1 = (w0 + 1/2) 2^-32, u2 = w1 2^-32 from the
 * words at counter (p, n, st, 5); a sampled field entry is +1 iff w0 2^-32 < sigmoid(logit),
 * w0 from counter (p, n, st, 6). Training steps draw stream 0, nmc_cgen_sample stream 1.
 *
 * Conventions as in nmc.h: every call returns nmc_status; a generator is not thread-safe;
 * device work runs on the stream given at creation; device pointers must be valid on its
 * device; host buffers are copied.
 */
#ifndef NMC_CGEN_H
#define NMC_CGEN_H

#include "nmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nmc_cgen nmc_cgen;

/* Create a generator for fields of shape (L_tau, Ly, Lx) with C channels (1 <= C <= 64),
 * Glorot-initialized from `seed`; max_batch: samples per call (workspace ~ 10 max_batch C
 * L_tau Lx Ly bytes). NMC_EINVAL: a size < 1, C > 64, out == NULL; NMC_ENOMEM / NMC_ECUDA on
 * allocation failure. */
nmc_status nmc_cgen_create(int Lx, int Ly, int L_tau, int channels, uint64_t seed,
                           int max_batch, void* cuda_stream, nmc_cgen** out);

/* Number of parameters (the length of the flat array above). */
nmc_status nmc_cgen_n_params(const nmc_cgen* g, long long* n);

/* Host copy of the FP32 parameters / set them from a host array (Adam's state is reset). */
nmc_status nmc_cgen_get_params(const nmc_cgen* g, float* theta);
nmc_status nmc_cgen_set_params(nmc_cgen* g, const float* theta);

/* Logits for n (<= max_batch) noise samples: d_z device FP32 [n][L_tau][Ly][Lx] (rounded
 * to BF16 on input), d_logits device FP32, same shape. */
nmc_status nmc_cgen_forward(nmc_cgen* g, const float* d_z, int n, float* d_logits);

/* Loss (host *loss) and its gradient with respect to the parameters (device d_grad, FP32,
 * n_params) for given noise d_z (FP32 [n][...], rounded to BF16) and fields d_fields
 * (int8 [n][L_tau][N], +-1). No update. */
nmc_status nmc_cgen_loss_grad(nmc_cgen* g, const float* d_z, const int8_t* d_fields, int n,
                              double* loss, float* d_grad);

/* One Adam step (learning rate lr, beta1 0.9, beta2 0.999, epsilon 1e-8) on n fields
 * d_fields (int8 [n][L_tau][N]), with the noise of samples sample0 .. sample0 + n - 1 of
 * stream 0; *loss receives the loss before the step. */
nmc_status nmc_cgen_train_step(nmc_cgen* g, const int8_t* d_fields, int n, long long sample0,
                               float lr, double* loss);

/* Fields for samples n0 .. n0 + n - 1 of stream 1 (noise, logits, Bernoulli draws):
 * device d_fields, int8 [n][L_tau][N] (the layout of nmc_set_fields_device); optionally
 * the logits (device FP32, may be NULL). */
nmc_status nmc_cgen_sample(nmc_cgen* g, long long n0, int n, int8_t* d_fields, float* d_logits);

void nmc_cgen_destroy(nmc_cgen* g);

#ifdef __cplusplus
}
#endif

#endif
