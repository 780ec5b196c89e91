/*
 * lpsim_surrogate.h -- C ABI of the link-travel-time surrogate used by the
 * assignment loop: a small MLP (inputs padded to 64 -> 256 -> 256 -> 256 ->
 * 1, GELU, BF16 weights and activations, FP32 accumulation) trained on the
 * simulator's own link statistics with mean-squared error and Adam, with
 * forward and backward passes in hand-written sm_103a tensor-core kernels
 * (tcgen05.mma into tensor memory, operands staged by TMA).
 *
 * The paper has no surrogate: it is the learned extension of the traffic
 * assignment named in the paper's title (dynamic rerouting is its future
 * work, Sec. 5, Conclusion).  The plain simulation still computes every relative gap.
 *
 * Conventions as in lpsim.h: int status codes, lpsim_last_error(), host
 * pointers for all inputs and outputs, the model owns its device memory.
 * Parameter tensors, in order: W1 (256 x 64), b1 (256), W2 (256 x 256),
 * b2, W3 (256 x 256), b3, W4 (1 x 256), b4 (1); W is out x in, row-major,
 * f32.  Columns of W1 beyond n_features multiply zero padding.
 */
#ifndef LPSIM_SURROGATE_H
#define LPSIM_SURROGATE_H

#include <stdint.h>

#include "lpsim.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lpsim_mlp lpsim_mlp;

/* New model with He-initialised weights from `seed`; batch = rows per
 * training step and per forward chunk (multiple of 128); stream as in
 * lpsim_load_network (NULL: the model creates its own). */
int lpsim_mlp_create(lpsim_mlp **out, uint32_t n_features, uint32_t batch, uint64_t seed, void *stream);
int lpsim_mlp_set_params(lpsim_mlp *m, const float *const *tensors);
int lpsim_mlp_get_params(lpsim_mlp *m, float *const *tensors);

/* y[i] = MLP(X[i, :]) for n rows of n_features f32 values (BF16 inside).
 * With more than `batch` rows the outputs gather on the device (4 bytes per
 * row, in whole batches; allocated at the first such call and kept until
 * lpsim_mlp_destroy, LPSIM_E_OOM if it cannot be) and cross back once. */
int lpsim_mlp_forward(lpsim_mlp *m, uint64_t n, const float *X, float *y);

/* Forward and backward of one batch (n <= batch rows): mean squared error
 * against t into *loss (nullable) and its gradient with respect to every
 * parameter tensor into grads[8] (each nullable). */
int lpsim_mlp_grad(lpsim_mlp *m, uint64_t n, const float *X, const float *t, float *loss, float *const *grads);

/* Training pool: samples (n rows of n_features f32 inputs X and targets t,
 * host arrays, copied) appended to a device-resident pool that the model
 * keeps between calls, so a training set that grows with every simulation
 * is uploaded once per row.  lpsim_mlp_pool_clear empties it.  Errors:
 * LPSIM_E_INVALID_ARG (NULL arrays with n > 0), LPSIM_E_OOM. */
int lpsim_mlp_pool_add(lpsim_mlp *m, uint64_t n, const float *X, const float *t);
int lpsim_mlp_pool_clear(lpsim_mlp *m);
uint64_t lpsim_mlp_pool_size(const lpsim_mlp *m);

/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr)
 * on minibatches of min(batch, pool size) rows drawn from shuffled passes
 * over the pool: pass q visits every row once in the order of a seeded
 * pseudo-random permutation (a Feistel network with cycle walking, keyed by
 * shuffle_seed and q), gathered on the device, so no minibatch crosses the
 * host.  losses (nullable, `steps` entries) receives each step's batch loss.
 * Errors: LPSIM_E_INVALID_ARG on an empty pool; LPSIM_E_TIMEOUT (a bounded
 * device wait or permutation walk gave up); LPSIM_E_OOM. */
int lpsim_mlp_train_pool(lpsim_mlp *m, uint32_t steps, float lr, uint64_t shuffle_seed, float *losses);

/* lpsim_mlp_pool_clear, lpsim_mlp_pool_add of the n samples, then
 * lpsim_mlp_train_pool. */
int lpsim_mlp_train(lpsim_mlp *m, uint64_t n, const float *X, const float *t, uint32_t steps, float lr,
                    uint64_t shuffle_seed, float *losses);

/* One Adam step (Kingma and Ba 2015, Algorithm 1; beta1 0.9, beta2 0.999,
 * eps 1e-8, learning rate lr) on the FP32 master weights with gradients
 * given by the caller: grads[8] host tensors in the parameter order above
 * (none NULL), e.g. gradients averaged over several models' lpsim_mlp_grad
 * calls.  The same update lpsim_mlp_train applies after each minibatch; it
 * continues that call's step count t (lpsim_mlp_set_params resets it) and
 * refreshes the BF16 weight copies.  Errors: LPSIM_E_INVALID_ARG on a NULL
 * tensor or a negative or non-finite lr; LPSIM_E_CUDA. */
int lpsim_mlp_apply_grads(lpsim_mlp *m, const float *const *grads, float lr);

/* Diagnostic: D (M x N, f32) = A (M x K) . B (N x K)^T for BF16 bit
 * patterns A, B (row-major) on the tensor-core GEMM kernel the model uses.
 * M % 128 == 0, K % 64 == 0, N == 64 or N % 256 == 0. */
int lpsim_mlp_gemm_test(uint32_t M, uint32_t N, uint32_t K, const uint16_t *A, const uint16_t *B, float *D);

/* Timing on the model's stream with CUDA events, on the batch buffers as they
 * are (device-resident): mean milliseconds of one inference forward pass of
 * `batch` rows (three tensor-core GEMMs with fused epilogues) and, if
 * train_ms is not NULL, of one training forward + backward pass. */
int lpsim_mlp_time(lpsim_mlp *m, uint32_t iters, double *fwd_ms, double *train_ms);

/* Diagnostics: GELU(z) and GELU'(z) of n inputs (host arrays) as the
 * tensor-core epilogues compute them -- z Phi(z) and Phi(z) + z phi(z) with
 * the standard normal CDF as a logistic of a fitted odd polynomial,
 * 1 / (1 + 2^(z q(z^2))) (|error| < 6.8e-6, |z| |error| < 3.1e-6), and the
 * exact density -- so that tests can hold them to their error bound. */
int lpsim_mlp_gelu_eval(uint64_t n, const float *z, float *gelu, float *dgelu);

void lpsim_mlp_destroy(lpsim_mlp *m);

#ifdef __cplusplus
}
#endif
#endif
