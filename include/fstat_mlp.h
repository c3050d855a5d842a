/*
 * fstat_mlp.h -- C ABI of the patch-scoring network of the learned-proposal
 * search (part of libfstat.so).
 *
 * The paper has no learned component; this network is the design's learned
 * proposal: it reads a patch of a coarse-grid 2F map (n_in values, e.g. 16 x 16
 * sky points x 32 frequencies = 8192) and scores whether a signal lies in it,
 * so that only the best-scoring patches are refined on the fine grid while the
 * exhaustive fine-grid F-statistic stays the fallback and the judge.
 *
 * Network: n_in -> H ReLU -> H ReLU -> 1 logit s, p = sigmoid(s).
 *   z1 = X W1 + b1, h1 = relu(z1), z2 = h1 W2 + b2, h2 = relu(z2), s = h2 . w3 + b3.
 * Loss: mean over the batch of w_i (softplus(s_i) - y_i s_i), w_i = pos_weight
 * for y_i = 1, else 1.  Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Storage: FP32 master parameters and Adam moments; BF16 copies of W1, W2 and
 * of the activations feed tensor-core matrix products with FP32 accumulation;
 * layer 3 and the loss run in FP32.
 *
 * Conventions as in fstat.h: status codes, inputs copied, outputs to caller
 * buffers, `mem` selects host or device pointers.  Inputs X are BF16 bit
 * patterns (uint16), row-major [B][n_in].
 */
#ifndef FSTAT_MLP_H
#define FSTAT_MLP_H

#include <stdint.h>

#include "fstat.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fstat_mlp fstat_mlp;

/* Create a network on `device` with n_in inputs (multiple of 8), H hidden
 * units (multiple of 8) and batches of up to max_batch rows.  Parameters are
 * zero until fstat_mlp_set_params.  Errors: EINVAL, ECUDA, ENOMEM. */
int fstat_mlp_create(fstat_mlp **out, int device, int32_t n_in, int32_t n_hidden, int32_t max_batch);
void fstat_mlp_destroy(fstat_mlp *m);
const char *fstat_mlp_last_error(const fstat_mlp *m);

/* Set / read the FP32 master parameters (host arrays): W1 [n_in][H],
 * b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1].  Setting resets Adam. */
int fstat_mlp_set_params(fstat_mlp *m, const float *W1, const float *b1, const float *W2, const float *b2,
                         const float *w3, const float *b3);
int fstat_mlp_get_params(fstat_mlp *m, float *W1, float *b1, float *W2, float *b2, float *w3, float *b3);

/* Logits s[B] of inputs X [B][n_in] (BF16 bits), B <= max_batch.  X and s
 * are host or device per `mem`; runs on cuda_stream, synchronises when mem is
 * host.  Errors: EINVAL. */
int fstat_mlp_forward(fstat_mlp *m, const uint16_t *X, int32_t B, float *logits, int32_t mem, void *cuda_stream);

/* One training step on a batch: forward, loss, backward, Adam update with
 * learning rate lr.  y[B] (FP32 0/1) host or device per `mem`; *loss (host,
 * may be NULL) receives the batch loss (this synchronises).  The gradients
 * of the step stay readable with fstat_mlp_get_grads. */
int fstat_mlp_train_step(fstat_mlp *m, const uint16_t *X, const float *y, int32_t B, float pos_weight, float lr,
                         float *loss, int32_t mem, void *cuda_stream);

/* Gradients of the last training step (FP32, host), same shapes as the
 * parameters.  Synchronises. */
int fstat_mlp_get_grads(fstat_mlp *m, float *dW1, float *db1, float *dW2, float *db2, float *dw3, float *db3);

/* Patches of the last 2F map computed by `ctx` (a bank with n_fdot = 1 whose
 * sky list is an n_a x n_d grid, index ia * n_d + id) as network inputs:
 * patch p = (sky patch (pa, pd) of size s_a x s_d, frequency start f_start[q]
 * of length n_fp) for pa in [0, n_a / s_a), pd in [0, n_d / s_d), q in
 * [0, n_q), ordered ((pa * (n_d / s_d)) + pd) * n_q + q; each row holds
 * x = max(2F - shift, 0) * scale rounded to BF16 (the subtraction, the
 * clamp and the product in FP32), ordered (ia_local, id_local, f_local); a
 * shift well above the noise mean leaves only excess power in the input.  out: device array [n_patches][s_a * s_d * n_fp] of BF16 bits.
 * f_start [n_q] host.  Runs on the context's last compute stream.
 * Errors: ESTATE (nothing computed), EINVAL (shapes). */
int fstat_extract_patches(fstat_ctx *ctx, int32_t n_a, int32_t n_d, int32_t s_a, int32_t s_d, int32_t n_fp,
                          const int32_t *f_start, int32_t n_q, float shift, float scale, uint16_t *out);

/* Windows of the same 2F map at arbitrary origins, for training data: window
 * w covers ia = (a0 + i) mod n_a for i < s_a (alpha wraps around the sky),
 * id = d0 .. d0 + s_d - 1 and f = f0 .. f0 + n_fp - 1, with
 * origin [n_w][3] = (a0, d0, f0) on the host; rows are laid out as in
 * fstat_extract_patches.  out: device array [n_w][s_a * s_d * n_fp].
 * Errors: ESTATE (nothing computed), EINVAL (an origin outside the grid). */
int fstat_extract_windows(fstat_ctx *ctx, int32_t n_a, int32_t n_d, int32_t s_a, int32_t s_d, int32_t n_fp,
                          const int32_t *origin, int32_t n_w, float shift, float scale, uint16_t *out);

#ifdef __cplusplus
}
#endif
#endif /* FSTAT_MLP_H */
