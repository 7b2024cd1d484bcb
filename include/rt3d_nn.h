/*
 * rt3d_nn.h -- layer kernels of the learned warm start (a small 3D U-Net that
 * predicts the converged ln J from (log10 chi, log10 eps, B, ln J_start)).
 * Not in the paper (arXiv:2102.01734); the solve started from the network's
 * prediction is certified by the same FP64 residual as any other start.
 *
 * Layouts. Activations are BF16, channel-last [S][V][C]: S samples, V =
 * nx*ny*nz voxels (x fastest), C a multiple of 16 (pad with zeros).
 * Convolutions are 3x3x3, periodic in x and y and zero-padded in z. Weights
 * are Wt[d][Ci][Co] (BF16) with d = (dz+1)*9 + (dy+1)*3 + (dx+1); the data
 * gradient uses the transposed copy WT[d][Co][Ci]. Gradient accumulators are
 * FP32 and must be zeroed by the caller. All pointers are device memory; all
 * work is issued on `stream` (NULL: legacy stream) without synchronising.
 * Every call returns RT3D_OK, RT3D_EINVAL for unsupported sizes, or
 * RT3D_ECUDA (message in rt3d_last_error()).
 */
#ifndef RT3D_NN_H
#define RT3D_NN_H

#include "rt3d.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Y[s][v][co] = act(bias[co] + sum_{d,ci} W[d][ci][co] X[s][v + sign d][ci]),
 * sign = +1, or -1 with transpose = 1 (then pass WT and swap Ci/Co: the data
 * gradient dX of a forward convolution). BF16 tensor-core products, FP32
 * accumulation. Ci: multiple of 16 up to 96; Co in {16, 32, 48, 64, 96}.
 * bias nullable (FP32 [Co]); Y (BF16) and Yf (FP32) nullable outputs; relu:
 * apply max(0, .). */
rt3d_status rt3d_nn_conv3d(const void *X, const void *W, const float *bias, void *Y, float *Yf,
                           int S, int nx, int ny, int nz, int Ci, int Co, int relu, int transpose,
                           void *stream);

/* dW[d][ci][co] += sum_{s,v} X[s][v+d][ci] dY[s][v][co] (FP32 accumulator
 * [27][Ci][Co]) and, if db is given, db[co] += sum dY[s][v][co].
 * (Ci/16)(Co/16) <= 16, Ci <= 96. */
rt3d_status rt3d_nn_conv3d_wgrad(const void *X, const void *dY, float *dW, float *db, int S,
                                 int nx, int ny, int nz, int Ci, int Co, void *stream);

/* out = dY where Y > 0, else 0 (n BF16 elements). */
rt3d_status rt3d_nn_relu_bwd(const void *dY, const void *Y, void *out, long long n, void *stream);

/* 2x2x2 average pooling to ((nx+1)/2, (ny+1)/2, (nz+1)/2): periodic in x and
 * y, a child above the top layer counts as zero (the sum is divided by 8). */
rt3d_status rt3d_nn_pool(const void *X, void *P, int S, int nx, int ny, int nz, int C,
                         void *stream);
/* dX32[child] += dP[parent] / 8 (FP32 accumulator of the fine grid). */
rt3d_status rt3d_nn_pool_bwd(const void *dP, float *dX32, int S, int nx, int ny, int nz, int C,
                             void *stream);

/* Nearest upsampling from the pooled grid of (nx, ny, nz) into channels
 * [coff, coff+C) of a Ctot-channel fine-grid tensor, and its gradient
 * (dX32[parent] += dU[child], FP32 accumulator of the coarse grid). */
rt3d_status rt3d_nn_upsample(const void *X, void *U, int S, int nx, int ny, int nz, int C,
                             int Ctot, int coff, void *stream);
rt3d_status rt3d_nn_upsample_bwd(const void *dU, float *dX32, int S, int nx, int ny, int nz,
                                 int C, int Ctot, int coff, void *stream);

/* dst[r][doff + c] = src[r][soff + c] for c < C over `rows` rows (BF16). */
rt3d_status rt3d_nn_channel_copy(const void *src, int Cs, int soff, void *dst, int Cd, int doff,
                                 int C, long long rows, void *stream);

rt3d_status rt3d_nn_f32_to_bf16(const float *a, void *b, long long n, void *stream);
/* out = a + b (BF16 = BF16 + FP32). */
rt3d_status rt3d_nn_add_bf16_f32(const void *a, const float *b, void *out, long long n,
                                 void *stream);

/* Network input from FP64 [rows] arrays: channels log10(chi)/3, log10(eps)/4,
 * B - 1, ln J0, then 12 zero channels (BF16 [rows][16]). */
rt3d_status rt3d_nn_features(const double *chi, const double *eps, const double *B,
                             const double *J0, void *X, long long rows, void *stream);

/* Output channel 0 of Yf ([rows][16] FP32) is the correction y = ln J - ln J0:
 * sse += sum (y - ln(target/J0))^2, dY[r][0] = 2 (y - ln(target/J0)) scale,
 * other channels 0 (BF16 [rows][16]). */
rt3d_status rt3d_nn_mse(const float *Yf, const double *target, const double *J0, void *dY,
                        float *sse, long long rows, float grad_scale, void *stream);

/* J = J0 exp(y) (FP64). */
rt3d_status rt3d_nn_apply(const float *Yf, const double *J0, double *J, long long rows,
                          void *stream);

/* Adam step (Kingma & Ba 2015) on an FP32 master copy w with gradient g and
 * moments m, v; `step` counts from 1. If Wt is given, also writes the BF16
 * copy Wt[d][ci][co] and its transpose WT[d][co][ci] (n = 27 Ci Co). */
rt3d_status rt3d_nn_adam(float *w, const float *g, float *m, float *v, int n, float lr, float b1,
                         float b2, float eps, int step, void *Wt, void *WT, int Ci, int Co,
                         void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RT3D_NN_H */
