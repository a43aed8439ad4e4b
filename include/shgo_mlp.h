/*
 * shgo_mlp.h - learned screening of (shell pair, nucleus) triples for the SHGO nuclear-attraction
 * library (include/shgo.h).
 *
 * The paper has no screening: it computes every term of Eq. 11.  This is an added pattern that
 * leaves what is computed unchanged up to a stated threshold: a small network predicts
 * log10 max_{ma,mb} |Z_C <a ma|1/|r-C||b mb>| for one shell pair (a, b) and one nucleus C, and
 * triples predicted below a threshold (with a safety margin) are left out of the nucleus sum of
 * Eq. 11.  The exact method remains the reference: callers audit a sample of the skipped triples with it.
 *
 * Network: 16 inputs (shgo_screen_features) -> 64 -> 64 -> 1, SiLU activations.  The forward pass
 * uses BF16 weights (rounded from FP32 master weights after every update) with FP32 accumulation;
 * training (forward, backward, Adam) runs in the library's own kernels.  Parameter layout (FP32,
 * SHGO_MLP_NPARAM values): W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3[1].  Inputs are
 * standardised with the mean and standard deviation given at creation.
 */
#ifndef SHGO_MLP_H
#define SHGO_MLP_H

#include <stdint.h>

#include "shgo.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SHGO_MLP_IN 16
#define SHGO_MLP_HIDDEN 64
#define SHGO_MLP_NPARAM (64 * 16 + 64 + 64 * 64 + 64 + 64 + 1)

typedef struct shgo_mlp shgo_mlp;

/* A network on the current device from host arrays: params[SHGO_MLP_NPARAM] and the 16 feature
 * means and standard deviations (sd > 0). */
shgo_status shgo_mlp_create(const float* params, const float* feature_mean, const float* feature_sd,
                            shgo_mlp** out);
void shgo_mlp_free(shgo_mlp* mlp);

/* FP32 master parameters to a host array of SHGO_MLP_NPARAM. */
shgo_status shgo_mlp_get_params(const shgo_mlp* mlp, float* params);

/* Checkpoint of the training state (host arrays of SHGO_MLP_NPARAM): FP32 master parameters, Adam's first
 * and second moments and the step count behind its bias corrections.  Waits for the device.  Restoring
 * it into a network with the same feature normalisation and continuing with the same samples gives the
 * same parameters, bit for bit, as training without the interruption: every training pass sums in a
 * fixed order (see shgo_mlp_train_step). */
shgo_status shgo_mlp_get_state(const shgo_mlp* mlp, float* params, float* adam_m, float* adam_v, int64_t* step);
shgo_status shgo_mlp_set_state(shgo_mlp* mlp, const float* params, const float* adam_m, const float* adam_v,
                               int64_t step);

/* y[s] = network(X[s, :]) for n samples; X [n][16] and y [n] are device arrays.  Asynchronous. */
shgo_status shgo_mlp_forward(const shgo_mlp* mlp, const float* X, int64_t n, float* y, void* stream);

/* Loss sum_s w_s (y_s - T_s)^2 / n with w_s = under_weight where y_s < T_s, 1 otherwise (an
 * under-predicted triple is the one that could be skipped wrongly).  Gradient with respect to the
 * FP32 parameters (host grad[SHGO_MLP_NPARAM]) and the loss (host), without an update.  Blocking. */
shgo_status shgo_mlp_gradients(shgo_mlp* mlp, const float* X, const float* T, int64_t n, float under_weight,
                               float* grad, float* loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on that loss over the n samples; the loss of the
 * pass before the update goes to *loss when loss != NULL (then the call blocks on `stream`).
 * The pass runs on the tensor cores (mma.sync BF16 with FP32 accumulation; FP32 activations and gradient
 * operands split into BF16 high and low parts) in a fixed summation order: per block of 32-sample tiles,
 * then over blocks in block order, the number of blocks depending only on n and the device.  Two runs over
 * the same samples from the same state give the same bits. */
shgo_status shgo_mlp_train_step(shgo_mlp* mlp, const float* X, const float* T, int64_t n, float under_weight,
                                float lr, float* loss, void* stream);

/*
 * Features of n (shell pair, nucleus) triples of a basis or batch, written to X [n][16] (device):
 *   0 la, 1 lb, 2-5 log10 of the smallest and largest exponent of a and of b, 6 |AB|,
 *   7 log10 K_AB of the most diffuse primitive pair, 8 |P - C| and 9 log10(1 + p |P - C|^2) for that
 *   pair, 10 log10 Z_C, 11-12 log10 sum |c~| of a and b (normalised contraction coefficients),
 *   13 |A - C|, 14 |B - C|, 15 log10 sum_ij |c~_i c~_j| K_ij (pi/p_ij)^{3/2} (an overlap scale).
 * triples [n][2] (device, int32) holds (unique shell-pair index, nucleus index into centers).
 * Shell-pair indices run over 0..shgo_basis_npairs-1 in the library's pair order, which
 * shgo_pair_shells reports.
 */
shgo_status shgo_screen_features(const shgo_basis* basis, const double* centers, const double* charges,
                                 const int32_t* triples, int64_t n, float* X, void* stream);

/* Shells (a, b) of the library's pair index q (host arrays of npairs), with a's l >= b's l. */
shgo_status shgo_pair_shells(const shgo_basis* basis, int32_t* shell_a, int32_t* shell_b);

/*
 * Screening of a basis (or batch) for the given nuclei: predicts every (pair, nucleus) triple and
 * keeps those with prediction >= log10_threshold - log10_margin.  The kept nucleus lists are kept
 * in the basis and used by shgo_nuclear_attraction_screened until the next call.  kept/skipped
 * receive the triple counts.  Blocking.
 */
shgo_status shgo_screen_build(shgo_basis* basis, const shgo_mlp* mlp, const double* centers, const double* charges,
                              int64_t n_centers, double log10_threshold, double log10_margin, int64_t* kept,
                              int64_t* skipped);

/* Skip mask of the last shgo_screen_build: for pair q the nuclei of its molecule in order, one
 * byte each (1 = kept), concatenated over pairs (length kept + skipped, host). */
shgo_status shgo_screen_mask(const shgo_basis* basis, uint8_t* mask);

/* V as shgo_nuclear_attraction (or the batched call for a batch), with the nucleus sum of every
 * shell pair restricted to its kept nuclei.  Asynchronous. */
shgo_status shgo_nuclear_attraction_screened(shgo_basis* basis, const double* centers, const double* charges,
                                             int64_t n_centers, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SHGO_MLP_H */
