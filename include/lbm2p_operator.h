/*
 * lbm2p_operator — a small convolutional operator that predicts the pressure of the next
 * physical step, used to warm-start the lattice Boltzmann pressure solve of lbm2p.h
 * (lbm2p_warm_start).  C ABI.
 *
 * The pressure solve of each step (Sec. 3: Eq. 3-1 iterated in pseudo time until steady)
 * starts from the previous step's populations; its length is set by how far that start is
 * from the new fixed point.  A predictor of the new pressure moves the start closer (the
 * equilibrium part of f, Eq. 3-3, moves to the prediction) while the solve still runs to the
 * same residual, so the prediction changes the number of sweeps, never the converged field.
 * The paper has no such predictor; this one is trained on (ln K, S, P history) -> P snapshots
 * that the solver itself produces.
 *
 * Network: five 3x3 convolutions with zero padding, ReLU between them, channels
 * C0 -> 32 -> 32 -> 32 -> 32 -> 1 (C0 = 16 input channels, the unused ones zero); weights
 * and activations BF16, products accumulated in FP32.  The convolutions run on the fifth-
 * generation tensor cores (tcgen05.mma, accumulators in tensor memory) as implicit GEMMs:
 * M = 128 pixels per tile, N = output channels, K = 9 taps x input channels (forward and
 * input gradient), or M = 128 (tap, input channel) rows, N = output channels, K = pixels
 * (weight gradient).
 *
 * Layouts.  Activations: BF16 [n_img][H][W][C] (channels fastest).  Weights: BF16
 * [9][C_out][C_in], tap t = 3 (dy + 1) + (dx + 1) for the input pixel (y + dy, x + dx).
 * Biases and master weights FP32.  All pointers are device pointers owned by the caller;
 * every call is asynchronous on `stream` (a cudaStream_t) and allocates nothing.  C_in and
 * C_out must be 16 or 32.  Errors: LBM2P_EINVAL for bad shapes or pointers (nothing is
 * launched); LBM2P_ECUDA when a launch fails (lbm2p_last_error(NULL) describes it).  A
 * kernel whose bounded wait on its tensor-core work gives up sets *err (device int) to 1
 * and leaves its output incomplete; callers read err after synchronising.
 */
#ifndef LBM2P_OPERATOR_H
#define LBM2P_OPERATOR_H

#include <stddef.h>

#include "lbm2p.h"

#ifdef __cplusplus
extern "C" {
#endif

/* y[p][co] = act(bias[co] + sum_{t, ci} x[p + d_t][ci] w[t][co][ci]), zero outside the image.
 * act: 0 = none, 1 = ReLU.  y (BF16 [npix][c_out]) and/or y0 (FP32 [npix], channel 0 only)
 * may be NULL.  mask (BF16 [npix][c_out] or NULL): when given, each output is multiplied by
 * (mask > 0) after the activation (the ReLU derivative in the input-gradient pass). */
lbm2p_status lbm2p_op_conv3x3(const void *x, const void *w, const float *bias, const void *mask,
                              void *y, float *y0, int n_img, int H, int W, int c_in, int c_out,
                              int act, int *err, void *stream);

/* Weight gradient of the convolution above: dw[t][co][ci] (+)= sum_p x[p + d_t][ci] g[p][co],
 * FP32 [9][c_out][c_in]; accumulate = 0 overwrites dw, 1 adds to it.  dbias (FP32 [c_out] or
 * NULL) (+)= sum_p g[p][co]. */
lbm2p_status lbm2p_op_conv3x3_wgrad(const void *x, const void *g, float *dw, float *dbias,
                                    int n_img, int H, int W, int c_in, int c_out, int accumulate,
                                    int *err, void *stream);

/* Weights of the input-gradient pass: wt[t][ci][co] = w[8 - t][co][ci] (BF16), so that
 * lbm2p_op_conv3x3(g, wt, ...) is the gradient of the convolution with respect to its input. */
lbm2p_status lbm2p_op_flip_weights(const void *w, void *wt, int c_in, int c_out, void *stream);

/* Adam step on FP32 master parameters p (n values) with gradient g, moments m and v, step
 * number t >= 1; writes the BF16 copy pb (may be NULL) used by the convolutions. */
lbm2p_status lbm2p_op_adam(float *p, const float *g, float *m, float *v, void *pb, long long n,
                           float lr, float beta1, float beta2, float eps, int t, void *stream);

/* Sums of a difference of two FP32 planes of n values: stats[0] += sum (a - b),
 * stats[1] += sum (a - b)^2 (FP64, device; the caller clears them).  The features, the
 * training target and the prediction below scale the increments of one lattice by their own
 * standard deviation sqrt(stats[1]/n - (stats[0]/n)^2), so an operator trained on one lattice
 * size applies to another. */
lbm2p_status lbm2p_op_diff_stats(const float *a, const float *b, long long n, double *stats,
                                 void *stream);

/* Features of one lattice for the operator, BF16 [H][W][16] (channels 4..15 zero):
 * 0: ln K;  1: (S - s_mean) / s_scale;  2: (S - S_prev) / sd(S - S_prev);
 * 3: (P - P_prev) / sd(P - P_prev);  sd from ds_stats and dp_stats (lbm2p_op_diff_stats).
 * lnK, S, S_prev, P, P_prev: FP32 [H][W] device planes. */
lbm2p_status lbm2p_op_features(const float *lnK, const float *S, const float *S_prev,
                               const float *P, const float *P_prev, const double *ds_stats,
                               const double *dp_stats, void *feat, int H, int W, float s_mean,
                               float s_scale, void *stream);

/* Training target of one lattice: tgt = (P_next - (2 P - P_prev)) / sd(P - P_prev), the
 * correction to the linear extrapolation in time in units of the last increment. */
lbm2p_status lbm2p_op_target(const float *P_next, const float *P, const float *P_prev,
                             const double *dp_stats, float *tgt, int H, int W, void *stream);

/* Pressure prediction from the operator's output d (FP32 [H][W]):
 * P_pred = 2 P - P_prev + sd(P - P_prev) d. */
lbm2p_status lbm2p_op_predict(const float *P, const float *P_prev, const float *d,
                              const double *dp_stats, float *P_pred, int H, int W, void *stream);

/* Mean-squared-error loss gradient for the operator's FP32 output y0 against target tgt
 * (both [npix]): g[p][0] = 2 (y0 - tgt) / npix as BF16 [npix][c_out] (other channels 0);
 * loss (device double, accumulated) += sum (y0 - tgt)^2 / npix. */
lbm2p_status lbm2p_op_mse_grad(const float *y0, const float *tgt, void *g, double *loss,
                               long long npix, int c_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM2P_OPERATOR_H */
