/*
 * vate_learned.h -- a small learned estimator beside the closed form of Eq. 11.
 *
 * The paper has no counterpart: Eq. 11 is its only estimator.  This adds an
 * MLP that maps what the pool knows about a host at the end of slice t to
 * log(1 + |OP(aip, t-k+1, k)|), trained on streams the method itself produces
 * with exact labels.  The counters stay exact integers; the closed form stays
 * available as the fallback and as the yardstick of the MLP's error.
 *
 * Features of a host (n_in = 2k + 2 floats, k <= 15):
 *   x[d]        = c_d / g for 0 <= d < k, c_d = the host's VATs at distance d
 *                 (last set d slices ago; vate_age_counts)
 *   x[k + d]    = h[d] / P for 0 <= d < k, the pool's ATs at distance d
 *                 (the census of the closed slice)
 *   x[2k]       = log2(g) / 16
 *   x[2k + 1]   = log1p(max(Eq. 11 estimate for k' = k, 0)) / 16
 * Model: y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3, hidden width 64, FP32
 * weights and accumulation.  y corrects the closed form in log space: the
 * estimate is expm1(8 y + log1p(max(Eq. 11 estimate, 0))), so a model that
 * outputs 0 reproduces the closed form (clamped at 0).  A gate tau completes
 * the model: where the corrected value and the closed form are both >= tau (a
 * host both call large, for which Eq. 11 is already accurate) the closed form
 * itself is returned.
 * Output rule for a host, in order: no active VAT in the window -> the closed
 * form, VATE_FLAG_FALLBACK; the corrected value not finite -> the closed form,
 * VATE_FLAG_FALLBACK; the corrected value and the closed form both >= tau ->
 * the closed form, VATE_FLAG_GATED; otherwise the corrected value.
 * Parameter layout (floats): W1[n_in][64], b1[64], W2[64][64], b2[64], w3[64], b3,
 * tau (vate_mlp_param_count(n_in) = 64 n_in + 4288 + 2).  Training leaves tau
 * alone (its gradient is 0); it is chosen after training (vate_mlp_apply lets
 * a caller score candidates on its training rows) -- +infinity never gates.
 *
 * Conventions are those of vate.h.
 */
#ifndef VATE_LEARNED_H
#define VATE_LEARNED_H

#include <stdint.h>
#include "vate.h"

#ifdef __cplusplus
extern "C" {
#endif

#define VATE_MLP_HIDDEN 64
#define VATE_FLAG_FALLBACK 4u   /* the closed form was returned: no active VAT, or no finite correction */
#define VATE_FLAG_GATED    8u   /* the closed form was returned: it and the corrected value are at or above the gate tau */

/* Number of parameters of the model for n_in inputs. */
uint64_t vate_mlp_param_count(uint32_t n_in);

/* Features (layout above) of n hosts at the end of the closed slice:
 * d_x device float[n * (2k+2)], row-major.  Errors: VATE_EINVAL if k > 15,
 * VATE_ESLICE if the slice is not closed. */
int vate_features(vate_handle *h, const uint32_t *d_aips, uint64_t n, float *d_x, void *stream);

/* Deterministic initialisation: weights uniform in +-sqrt(6 / (fan_in +
 * fan_out)) (Glorot) from a counter-based hash of (seed, index); biases 0;
 * the gate tau = +infinity. */
int vate_mlp_init(float *d_params, uint32_t n_in, uint64_t seed, void *stream);

/* y[i] = model(x[i]) for n rows of x (device float[n * n_in]) into d_y (device float[n]). */
int vate_mlp_forward(const float *d_params, uint32_t n_in, const float *d_x, uint64_t n, float *d_y, void *stream);

/* The output rule (above) on n feature rows d_x (device float[n * n_in],
 * n_in = 2k + 2) with their closed-form estimates d_plain (device float[n]):
 * d_out (device float[n]) and, if not NULL, d_flags (device uint8[n]: the
 * FALLBACK / GATED bits) -- what vate_estimate_learned returns for hosts with
 * these features.  A row has no active VAT when its first k features are 0. */
int vate_mlp_apply(const float *d_params, uint32_t n_in, const float *d_x, const float *d_plain, uint64_t n,
                   float *d_out, uint8_t *d_flags, void *stream);

/* Scratch floats that vate_mlp_train_step needs for a batch of n rows. */
uint64_t vate_mlp_train_scratch(uint32_t n_in, uint64_t n);

/* Loss of vate_mlp_train_step over the n rows, with row weights w (1 if NULL):
 *   VATE_MLP_LOSS_SQUARED   mean of w (y - target)^2
 *   VATE_MLP_LOSS_ABSOLUTE  mean of w |y - target|  (subgradient 0 at y = target) */
#define VATE_MLP_LOSS_SQUARED  0u
#define VATE_MLP_LOSS_ABSOLUTE 1u

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; t = step number >= 1) on
 * the loss above, in place on d_params with moments d_m, d_v (each
 * param_count floats, zero at t = 1).  d_weight: device float[n] or NULL.
 * The gradient is formed from per-tile partial sums added in a fixed order,
 * so training is bit-reproducible.  d_grad (param_count floats) and d_loss
 * (1 float) receive the batch gradient and loss; either may be NULL.
 * d_scratch: vate_mlp_train_scratch(n_in, n) floats. */
int vate_mlp_train_step(float *d_params, float *d_m, float *d_v, uint32_t n_in, const float *d_x,
                        const float *d_target, const float *d_weight, uint32_t loss, uint64_t n, float lr,
                        uint32_t t, float *d_scratch, uint64_t scratch_floats, float *d_grad, float *d_loss,
                        void *stream);

/* Learned estimate of |OP(aip, t-k+1, k)| for n hosts at the end of the
 * closed slice, in one gather per host, by the output rule above.  d_flags
 * also carries VATE_FLAG_SAT / VATE_FLAG_POOLFULL of the closed form.  For
 * seg_len >= 16 features, MLP, gate and the Eq. 11 fallback run fused in one
 * kernel; for seg_len <= 8 (where the host's g / seg_len segment reads bound
 * the close) the features and Eq. 11 of up to 2^17 hosts at a time go to a
 * device scratch of the handle, then the model runs over those rows -- the
 * results are the same bit for bit.  That scratch (2^17 (2k + 3) floats, at
 * most 17.3 MB) is allocated on the first such call and kept until
 * vate_destroy.  Errors: VATE_ENOMEM if it cannot be allocated. */
int vate_estimate_learned(vate_handle *h, const uint32_t *d_aips, uint64_t n, const float *d_params, float *d_out,
                          uint8_t *d_flags, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VATE_LEARNED_H */
