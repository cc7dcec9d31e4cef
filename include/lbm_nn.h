/*
 * lbm_nn.h - C ABI of the warm-start network kernels.
 *
 * The paper has no learned component.  These kernels serve a learned warm
 * start of the steady side-heated cell: a 3D U-Net maps the (Ra, Pr) of a
 * cell and a coarse converged solution, trilinearly upsampled, to the steady
 * fine-grid fields (u, v, w, T), which then initialise the lattice Boltzmann
 * iteration.  Every operation of the network's forward pass, backward pass
 * and optimiser runs in these kernels; the caller only sequences them.
 *
 * Conventions: activations are FP32, one sample, channel-major [C][D][H][W]
 * with W fastest; convolution weights are BF16 [Cout][Cin][27] (taps ordered
 * dz, dy, dx each in -1, 0, 1, dx fastest) with FP32 accumulation and an FP32
 * bias.  The convolutions run on the tensor cores (BF16 x BF16 -> FP32): an
 * FP32 activation or gradient operand enters as the sum of two BF16 terms
 * (relative error at most 2^-18 per operand), so results agree with an FP32
 * convolution of the same BF16 weights to about 1e-6 relative.  All pointers are device pointers; every call is asynchronous on
 * `stream` (NULL: legacy default stream) and returns an lbm_status
 * (lbm_last_error(NULL) describes a failure).  Sizes must be positive.
 */
#ifndef LBM_NN_H
#define LBM_NN_H

#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* y[co] = bias[co] + sum_ci sum_tap w[co][ci][tap] x[ci][voxel + tap] (zero
 * padding), then max(., 0) when relu != 0.  y may be a channel slice of a
 * larger buffer (it holds Cout channels of D H W values). */
lbm_status lbm_nn_conv3d_forward(const float *x, int Cin, int D, int H, int W, const uint16_t *w_bf16,
                                 const float *bias, int Cout, float *y, int relu, void *stream);

/* dx[ci] (+)= sum_co sum_tap w[co][ci][tap] dy[co][voxel - tap]: the data
 * gradient of the convolution (accumulate != 0 adds to dx).  w_t_bf16 is the
 * scratch for the flipped, transposed weights [Cin][Cout][27]. */
lbm_status lbm_nn_conv3d_backward_data(const float *dy, int Cout, int D, int H, int W, const uint16_t *w_bf16,
                                       uint16_t *w_t_bf16, int Cin, float *dx, int accumulate, void *stream);

/* dw[co][ci][tap] += sum_voxels dy[co][voxel] x[ci][voxel + tap];
 * db[co] += sum_voxels dy[co][voxel]  (FP32, accumulated by atomic adds, so
 * the low bits depend on the order blocks finish; db may be NULL).
 * Cin <= 128 (LBM_ERR_PARAM otherwise). */
lbm_status lbm_nn_conv3d_backward_weight(const float *x, int Cin, int D, int H, int W, const float *dy, int Cout,
                                         float *dw, float *db, void *stream);

/* dy *= (y > 0): the ReLU backward, in place on n values. */
lbm_status lbm_nn_relu_backward(float *dy, const float *y, int64_t n, void *stream);

/* Average pooling by 2 per axis with ceil sizes (a window at an odd edge
 * averages the voxels it has): x [C][D][H][W] -> y [C][(D+1)/2][(H+1)/2][(W+1)/2];
 * the backward spreads dy over the window (accumulate != 0 adds to dx). */
lbm_status lbm_nn_avgpool2_forward(const float *x, int C, int D, int H, int W, float *y, void *stream);
lbm_status lbm_nn_avgpool2_backward(const float *dy, int C, int D, int H, int W, float *dx, int accumulate,
                                    void *stream);

/* Nearest upsampling to D H W: y[c][z][y][x] = x[c][z/2][y/2][x/2] with x of
 * size (D+1)/2 (H+1)/2 (W+1)/2; the backward sums dy over each parent. */
lbm_status lbm_nn_upsample2_forward(const float *x, int C, int D, int H, int W, float *y, void *stream);
lbm_status lbm_nn_upsample2_backward(const float *dy, int C, int D, int H, int W, float *dx, void *stream);

/* Trilinear interpolation of node-centred fields from a d h w lattice to a
 * D H W lattice over the same box (node j at (j + 1/2)/n; clamped at the
 * walls): the coarse-solution input of the network. */
lbm_status lbm_nn_trilinear(const float *x, int C, int d, int h, int w, float *y, int D, int H, int W,
                            void *stream);

/* y += a x over n values. */
lbm_status lbm_nn_axpy(float a, const float *x, float *y, int64_t n, void *stream);

/* Mean squared error over n values: loss[0] (+)= sum (p - t)^2 / n (FP64 sum,
 * accumulated), grad = 2 (p - t)/n (overwritten; may be NULL). */
lbm_status lbm_nn_mse(const float *p, const float *t, int64_t n, double *loss, float *grad, void *stream);

/* Adam step (Kingma & Ba, 2015) on n FP32 master weights with gradients g,
 * moments m and v, step count t >= 1; writes the BF16 copy w_bf16 (may be
 * NULL) and zeroes g. */
lbm_status lbm_nn_adam(float *w, uint16_t *w_bf16, float *g, float *m, float *v, int64_t n, float lr, float beta1,
                       float beta2, float eps, int t, void *stream);

/* FP32 -> BF16 (round to nearest even) over n values. */
lbm_status lbm_nn_to_bf16(const float *x, uint16_t *y, int64_t n, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_NN_H */
