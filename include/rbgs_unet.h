/*
 * rbgs_unet.h -- C ABI of the learned initial guess in librbgs.so.
 *
 * The paper has no counterpart: a small convolutional U-Net maps a Poisson problem's
 * right-hand side and Dirichlet data to an initial guess u0 for red-black Gauss-Seidel,
 * which then runs to the same tolerance as from u0 = 0 (so RBGS remains the fallback,
 * and the residual it reaches, not the network, decides the final error).
 *
 * Tensors are NHWC (channels fastest), batch B, height H, width W.  Activations and
 * operands of the convolutions are bfloat16 (uint16_t bit patterns); accumulation is
 * FP32; master weights, gradients and Adam moments are FP32.  All pointers are device
 * memory of the current device unless stated otherwise.  Work is ordered on the given
 * stream (a cudaStream_t; NULL = legacy default stream).  Status codes are rbgs_status.
 *
 * Network (4 levels, base width 32): per level two 3x3 convolutions with ReLU, 2x2
 * average pooling down, nearest-neighbour upsampling up, skip connections by channel
 * concatenation, widths 32/64/128/256, a final 1x1 convolution to one channel.  Input
 * channels: f, boundary mask (1 on the Dirichlet ring), boundary values g (0 off the
 * ring), and a smooth interpolation of g into the interior; zero-padded to 16 channels
 * internally.  H and W must be multiples of 8.
 */
#ifndef RBGS_UNET_H
#define RBGS_UNET_H

#include <stdint.h>

#include "rbgs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- layer kernels --- */

/*
 * Not in the paper: the learned-initial-guess growth direction (as every entry point
 * of this header).
 * 3x3 convolution, stride 1, zero padding 1 (cross-correlation, as in deep learning):
 *   Y[b,y,x,o] = act( bias[o] + sum_{dy,dx,c} Wt[o,dy,dx,c] * X[b,y+dy-1,x+dx-1,c] )
 * X: B*H*W*Cin bf16; Wt: Cout*3*3*Cin bf16; bias: Cout fp32 (may be NULL);
 * Y: B*H*W*Cout bf16, or fp32 when y_fp32 != 0.  act = ReLU when relu != 0.
 * Cin and Cout must be multiples of 8.  ksize is 3 (or 1 for a 1x1 convolution).
 */
rbgs_status rbgs_conv_forward(const uint16_t *X, const uint16_t *Wt, const float *bias, void *Y,
                              int B, int H, int W, int Cin, int Cout, int ksize, int relu,
                              int y_fp32, void *cuda_stream);

/*
 * Not in the paper (learned initial guess).
 * Backward of rbgs_conv_forward without the activation, given G = dLoss/d(pre-activation)
 * (B*H*W*Cout bf16):
 *   dX[b,y,x,c]  (+)= sum_{dy,dx,o} Wt[o,dy,dx,c] * G[b,y-dy+1,x-dx+1,o]   (fp32; added to
 *                     the existing contents when accumulate != 0; dX may be NULL)
 *   dW[o,dy,dx,c] += sum_{b,y,x} G[b,y,x,o] * X[b,y+dy-1,x+dx-1,c]       (fp32, accumulated)
 *   db[o]        += sum_{b,y,x} G[b,y,x,o]                                (fp32; may be NULL)
 * Wt_t is scratch of 9*Cin*Cout bf16 (device) used for the transposed weights.
 */
rbgs_status rbgs_conv_backward(const uint16_t *X, const uint16_t *Wt, const uint16_t *G, float *dX,
                               float *dW, float *db, uint16_t *Wt_t, int B, int H, int W, int Cin,
                               int Cout, int ksize, int accumulate, void *cuda_stream);

/*
 * Not in the paper (learned initial guess): library mechanics.
 * Engine of the convolution kernels (process-wide; applies to the network too):
 *   RBGS_CONV_TCGEN05        (default) 5th-generation tensor cores: tcgen05.mma from shared-
 *                            memory descriptors, FP32 accumulators in tensor memory, 128-row
 *                            tiles; operand tiles of the data-gradient product loaded by TMA
 *                            when the output channels split into chunks of 64, 32 and 16,
 *                            all other operand tiles gathered by cp.async;
 *   RBGS_CONV_MMA_SYNC       warp-level mma.sync tiles with register accumulators;
 *   RBGS_CONV_TCGEN05_GATHER tcgen05 with every operand tile gathered by cp.async.
 * All compute the same sums in FP32 (the order of accumulation differs).  Returns
 * RBGS_EINVAL for another value.  rbgs_conv_get_engine returns the current engine.
 */
#define RBGS_CONV_TCGEN05 0
#define RBGS_CONV_MMA_SYNC 1
#define RBGS_CONV_TCGEN05_GATHER 2
rbgs_status rbgs_conv_set_engine(int engine);
int rbgs_conv_get_engine(void);

/*
 * Not in the paper (learned initial guess): library mechanics.
 * Kernel of the 3x3 weight-gradient product under RBGS_CONV_TCGEN05 (process-wide):
 *   RBGS_WGRAD_AUTO   (default) per layer shape, the kernel that measured fastest on GB300
 *                     over the network's layers: RBGS_WGRAD_RING for Cin <= 32;
 *                     RBGS_WGRAD_TAPROW for image rows of at least 64 pixels when its work
 *                     split gives every SM at least 40 stages; RBGS_WGRAD_GATHER otherwise;
 *   RBGS_WGRAD_RING   all nine taps per stage: each activation row is staged once as three
 *                     copies shifted by one pixel and kept in a ring while the output rows
 *                     walk down the image (M = 3 Cin rows of (tap column, channel));
 *   RBGS_WGRAD_TAPROW one tap row per pass: the activation row staged once with a pixel of
 *                     halo, the three tap columns read at 16-byte descriptor offsets;
 *   RBGS_WGRAD_GATHER the operand tiles gathered by cp.async per tap (the kernel that
 *                     RBGS_CONV_TCGEN05_GATHER uses for every product).
 * A kernel whose tiling does not fit a shape falls back to the next one in the order ring,
 * tap row, gather.  All compute the same FP32 sums of the same bf16 products (the order of
 * accumulation differs), and all add into dW.  Returns RBGS_EINVAL for another value.
 * rbgs_conv_get_wgrad_kernel returns the current choice.  1x1 layers always gather.
 */
#define RBGS_WGRAD_AUTO 0
#define RBGS_WGRAD_RING 1
#define RBGS_WGRAD_TAPROW 2
#define RBGS_WGRAD_GATHER 3
rbgs_status rbgs_conv_set_wgrad_kernel(int kind);
int rbgs_conv_get_wgrad_kernel(void);

/*
 * Not in the paper (learned initial guess): library mechanics.
 * Synchronises `cuda_stream` and reports whether a tcgen05 convolution launched since
 * the last check gave up one of its bounded waits on the tensor cores (RBGS_ETIMEOUT; its
 * output is then incomplete).  Clears the condition.  RBGS_OK otherwise.
 */
rbgs_status rbgs_conv_check(void *cuda_stream);

/* -------------------------------------------------------------------- network --- */

typedef struct rbgs_unet *rbgs_unet_t;

/* Not in the paper (learned initial guess).  Creates the network with weights initialised
 * from `seed` (He-uniform, SplitMix64). */
rbgs_status rbgs_unet_create(uint64_t seed, void *cuda_stream, rbgs_unet_t *out);

/* Not in the paper (learned initial guess).  Number of FP32 parameters (weights and
 * biases of all layers, in a fixed order). */
long rbgs_unet_num_params(rbgs_unet_t net);

/* Not in the paper (learned initial guess).  Copies the FP32 master parameters to / from
 * `params` (host or device memory). */
rbgs_status rbgs_unet_get_params(rbgs_unet_t net, float *params);
rbgs_status rbgs_unet_set_params(rbgs_unet_t net, const float *params);

/*
 * Not in the paper (learned initial guess).
 * Forward pass: x is B*H*W*4 fp32 (the four input channels), y receives B*H*W fp32
 * predictions.
 * Buffers for B x H x W are allocated on first use and reused.
 */
rbgs_status rbgs_unet_forward(rbgs_unet_t net, const float *x, float *y, int B, int H, int W);

/*
 * Not in the paper (learned initial guess).
 * One training step: forward, loss = sum(mask_loss * (y - target)^2) / sum(mask_loss),
 * backward (every layer by the library's kernels), one Adam update (lr, beta1 0.9, beta2
 * 0.999, eps 1e-8) of the FP32 master weights, which are then rounded to bf16 for the
 * next forward.  mask_loss is B*H*W fp32 (1 where the loss counts).  *loss receives the
 * loss before the update (synchronises the stream).  When grads != NULL the step stops
 * after the backward pass (no update) and copies the FP32 gradient, in parameter order,
 * to grads (num_params values, host or device).
 */
rbgs_status rbgs_unet_train_step(rbgs_unet_t net, const float *x, const float *target,
                                 const float *mask_loss, int B, int H, int W, float lr,
                                 float *loss, float *grads);

/* Not in the paper (learned initial guess): library mechanics.  Frees the network (NULL is
 * ignored). */
void rbgs_unet_destroy(rbgs_unet_t net);

/* ------------------------------------------------------- grids of the guess --- */

/*
 * Not in the paper (learned initial guess).  Grid operations around the network, all on
 * device memory of the current device, asynchronous on the stream; g = n + 2 and
 * (n+2)^2 grids are row-major with the Dirichlet ring.  The transfinite (Coons)
 * interpolation of a ring, at point (i, j) with x = i/(g-1), y = j/(g-1), is
 *   (1-x) N_j + x S_j + (1-y) W_i + y E_i - ((1-x)(1-y) c00 + (1-x) y c01 + x (1-y) c10 + x y c11)
 * (N, S, W, E: rows 0, g-1 and columns 0, g-1; c: the corners).  It reproduces ring data
 * linear in x and in y, and the ring itself.
 *   rbgs_guess_blend:    out (g^2 doubles) = that interpolation of u_ring's ring.
 *   rbgs_guess_input:    x (size^2 x 4 floats, channels fastest; size >= g, a multiple of 8)
 *                        = f on the interior, the ring mask, the ring values, the blend;
 *                        zero outside the g x g corner.
 *   rbgs_guess_target:   t (size^2 floats) = sol - blend on the g x g corner, zero elsewhere
 *                        (what the network learns: the correction to the blend).
 *   rbgs_guess_assemble: u0 (g^2 doubles) = the ring of u_ring, interior blend + pred
 *                        (pred: size^2 floats, the network's output).
 * EINVAL for n < 1, a bad size or a pointer that is not device memory.
 */
rbgs_status rbgs_guess_blend(const double *u_ring, int n, double *out, void *cuda_stream);
rbgs_status rbgs_guess_input(const double *f, const double *u_ring, int n, int size, float *x, void *cuda_stream);
rbgs_status rbgs_guess_target(const double *sol, const double *u_ring, int n, int size, float *t,
                              void *cuda_stream);
rbgs_status rbgs_guess_assemble(const double *u_ring, const float *pred, int n, int size, double *u0,
                                void *cuda_stream);

/*
 * Not in the paper (learned initial guess).  Transfer between a fine n^2 grid and a coarse
 * nc^2 training grid whose nodes are fine nodes: r = (n+1)/(nc+1) must be an integer
 * (EINVAL otherwise), coarse node (ci, cj) sits on fine node (ci r, cj r).
 *   rbgs_guess_coarsen: fc (nc^2) = the mean of f over the (2r-1)^2 fine interior nodes
 *                       around each coarse interior node; uc_ring ((nc+2)^2) = u_ring at
 *                       the coarse nodes.
 *   rbgs_guess_refine:  u0 ((n+2)^2) = the bilinear interpolation of uc ((nc+2)^2) at the
 *                       fine interior nodes, the ring of u_ring.
 */
rbgs_status rbgs_guess_coarsen(const double *f, const double *u_ring, int n, int nc, double *fc, double *uc_ring,
                               void *cuda_stream);
rbgs_status rbgs_guess_refine(const double *uc, int nc, const double *u_ring, int n, double *u0, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RBGS_UNET_H */
