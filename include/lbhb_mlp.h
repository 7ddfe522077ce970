/*
 * Flow-curve surrogate of the lbhb library: a 4-layer perceptron
 * 5 -> 128 -> 128 -> 128 -> 2 (tanh hidden units) mapping
 * (log S, G_AA1, G_AA2, G_AB, tau) to (stress, yielded logit), trained and
 * served by hand-written BF16 tensor-core kernels with FP32 accumulation and
 * FP32 master weights.  The paper has no learned component: the network stands
 * in for repeated lattice Boltzmann runs of the Herschel-Bulkley flow curve
 * (sigma = sigma_Y + A S^beta, section "Numerical Results"), and the lattice
 * Boltzmann update stays the fallback and the reference for its error.
 *
 * Conventions: status codes are lb_status (lbhb.h).  x, targets and outputs
 * are DEVICE float32 buffers of the current device, caller-owned, rows of one
 * query each; calls are asynchronous on the handle's stream except where a host
 * output is returned.  One handle per host thread.
 *
 * Parameter vector (float32, mlp_param_count() entries): W1, b1, W2, b2, W3,
 * b3, W4, b4 with W_l row-major [out][in]; sizes 128x5, 128, 128x128, 128,
 * 128x128, 128, 2x128, 2.
 *
 * Model: z = (x - center) / half_range, h1 = tanh(W1 z + b1), h2 = tanh(W2 h1 + b2),
 * h3 = tanh(W3 h2 + b3), y = W4 h3 + b4; stress = y0 * sigma_scale, logit = y1.
 * Loss (per batch): mean (y0 - t)^2 + lam * mean BCE(y1, label), t = stress /
 * sigma_scale.  Adam with bias correction on the FP32 masters.
 */
#ifndef LBHB_MLP_H
#define LBHB_MLP_H

#include "lbhb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlp_handle mlp_handle;

typedef struct {
    int max_batch;               /* largest B of any call (>= 1) */
    double lam;                  /* weight of the classification term */
    double lr, beta1, beta2, eps;/* Adam */
    double center[5];            /* input normalisation: center of the training box */
    double half_range[5];        /* half width of the training box (> 0) */
    double sigma_scale;          /* stress = y0 * sigma_scale (> 0) */
    double logit_margin;         /* mlp_serve: |logit| below it sends the query to the LB */
} mlp_config;

/* Number of float32 parameters (34050). */
long long mlp_param_count(void);

/* Creates a handle and its device buffers for batches up to cfg->max_batch.
 * cuda_stream: a cudaStream_t of the current device or NULL (library stream).
 * Parameters start at zero: call mlp_set_params.  Errors: LB_ERR_INVALID,
 * LB_ERR_NOMEM, LB_ERR_CUDA. */
lb_status mlp_create(const mlp_config* cfg, void* cuda_stream, mlp_handle** out);

/* Copies the FP32 parameters from/to HOST memory (n = mlp_param_count()) and
 * resets the Adam state (set only).  Synchronous. */
lb_status mlp_set_params(mlp_handle* h, const float* params, long long n);
lb_status mlp_get_params(mlp_handle* h, float* params, long long n);

/* Forward pass: x [B][5] raw inputs -> out [B][2] = (stress, logit).  Async. */
lb_status mlp_forward(mlp_handle* h, const float* x, int batch, float* out);

/* Loss and its gradient with respect to every parameter, without updating:
 * grad (HOST, n floats) and *loss (HOST).  targets [B] stress, labels [B] in {0,1}.
 * Synchronous. */
lb_status mlp_gradients(mlp_handle* h, const float* x, const float* target_stress, const float* label,
                        int batch, float* grad, double* loss);

/* One Adam step on the batch: forward, loss, backward, update.  *loss_dev
 * (device, nullable) receives the batch loss.  Async. */
lb_status mlp_train_step(mlp_handle* h, const float* x, const float* target_stress, const float* label,
                         int batch, float* loss_dev);

/* Error budget of serving: bin_error (HOST, n_bins floats) is the stress error
 * the network showed on held-out LB points in n_bins equal bins of log S over
 * [log_s_lo, log_s_hi]; queries falling in a bin whose error exceeds `budget`
 * are sent to the LB by mlp_serve.  n_bins = 0 removes the table.  At most 256
 * bins.  Synchronous. */
lb_status mlp_set_error_budget(mlp_handle* h, const float* bin_error, int n_bins, double log_s_lo,
                               double log_s_hi, double budget);

/* Serving: forward pass plus the fallback decision per query, in one kernel
 * launch (the served stress and logit equal mlp_forward's bit for bit):
 * fallback[b] = 1
 * if any input lies outside the training box center +- half_range, if
 * |logit| < logit_margin (yielded/arrested undecided), or if the query's log S
 * bin is above the error budget (mlp_set_error_budget); 0 otherwise.  stress,
 * logit: device [B]; fallback: device int [B].  Async. */
lb_status mlp_serve(mlp_handle* h, const float* x, int batch, float* stress, float* logit, int* fallback);

/* Kernel launches enqueued by the handle since creation. */
long long mlp_kernel_launches(const mlp_handle* h);

/* Frees the handle (NULL is a no-op). */
void mlp_destroy(mlp_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* LBHB_MLP_H */
