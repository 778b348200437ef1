/*
 * cl_nn.h -- C ABI of the learned warm start of the reactive-diffusion
 * solver in cl_lbm.h: a 4-level 3D U-Net (16/32/64/128 channels) that maps a
 * catalyst-layer structure to a correction of the linear initial field, so
 * that the D3Q7 iteration of Eq. 21 starts nearer its steady state.  The
 * paper itself starts every solve from a uniform or linear field
 * (Sec. 3.5); the network only chooses where the iteration starts, the
 * lattice Boltzmann steps still compute the answer, and D_eff (Eq. 19) is
 * read from the converged state exactly as without it.
 *
 * Building blocks for training and inference, every one a kernel of this
 * library (no cuDNN, no cuBLAS):
 *   - 3x3x3 convolutions as implicit GEMMs on the tensor cores (BF16
 *     operands, FP32 accumulation; tcgen05 with the accumulator in tensor
 *     memory when both channel counts are multiples of 16), forward, data
 *     gradient (the same
 *     convolution with the kernel flipped and its channel axes swapped) and
 *     weight gradient (reduced over voxels in fixed-size slices, summed in a
 *     fixed order: deterministic);
 *   - ReLU backward, 2x2x2 average pooling, 2x nearest upsampling, channel
 *     copies into concatenation buffers, a 1x1x1 FP32 head, the masked
 *     mean-squared loss, and Adam on FP32 master weights with BF16 copies.
 *
 * Conventions:
 *   - Activations are NDHWC, BF16 (uint16 bit patterns), element
 *     (n, z, y, x, c) at ((n*D + z)*H + y)*W + x)*stride + off + c: a layer
 *     may read or write a channel window [off, off + C) of a wider buffer.
 *   - M = N*D*H*W voxels.
 *   - Convolution weights are [27][co][ci], tap t = 9*kz + 3*ky + kx at
 *     offset (kz-1, ky-1, kx-1); BF16.  Biases FP32 [co].
 *   - x (the transport direction) is zero padded; y and z wrap when
 *     periodic_yz is nonzero (the structures are periodic there), else they
 *     are zero padded.
 *   - Every pointer is a DEVICE pointer; `stream` is a cudaStream_t or NULL.
 *     Calls only enqueue work; none synchronises unless stated.
 *   - Errors: CL_ERR_ARG for NULL pointers or sizes the kernels do not
 *     support (stated per call), CL_ERR_CUDA for a launch failure.
 */
#ifndef CL_NN_H
#define CL_NN_H

#include <stdint.h>

#include "cl_lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* out = relu?(conv3d(in, w) + bias).  in: channels [in_off, in_off+ci) of a
   buffer with in_stride channels; out: channels [out_off, out_off+co) of a
   buffer with out_stride channels.  ci a multiple of 16, co of 8
   (CL_ERR_ARG otherwise); bias may be NULL (zero). */
cl_status cl_nn_conv3d(const void* in, const void* w, const float* bias, void* out, int N, int D, int H, int W, int ci,
                       int co, int in_stride, int in_off, int out_stride, int out_off, int relu, int periodic_yz,
                       void* stream);

/* Bytes of FP32 workspace cl_nn_conv3d_wgrad needs for this geometry. */
long long cl_nn_wgrad_workspace(int N, int D, int H, int W, int ci, int co);

/* dw[27][co][ci] (FP32, overwritten) = sum over voxels of
   dout (x) shifted input: the weight gradient of cl_nn_conv3d.  `in` and
   `dout` use the channel windows of the forward call; workspace holds
   cl_nn_wgrad_workspace(...) bytes.  ci and co multiples of 16. */
cl_status cl_nn_conv3d_wgrad(const void* in, const void* dout, float* workspace, float* dw, int N, int D, int H, int W,
                             int ci, int co, int in_stride, int in_off, int out_stride, int out_off, int periodic_yz,
                             void* stream);

/* wd[27][ci][co] = w[26 - t][co][ci]: the kernel whose forward convolution
   is the data gradient of w's. */
cl_status cl_nn_wt_dgrad(const void* w, void* wd, int co, int ci, void* stream);

/* db[c] (FP32, overwritten) = sum over the M voxels of dout[., off + c]. */
cl_status cl_nn_bias_grad(const void* dout, long long M, int C, int stride, int off, float* db, void* stream);

/* dy[., off + c] = 0 where y[., off + c] <= 0 (ReLU backward, in place). */
cl_status cl_nn_relu_bwd(const void* y, void* dy, long long M, int C, int stride, int off, void* stream);

/* y [N, D/2, H/2, W/2, C] (dense) = 2x2x2 mean of x (channel window xs/xo).
   D, H, W even. */
cl_status cl_nn_pool(const void* x, void* y, int N, int D, int H, int W, int C, int xs, int xo, void* stream);

/* dx (window xs/xo, full resolution D x H x W) = dy / 8 broadcast to each
   2x2x2 block; added to dx when accumulate is nonzero. */
cl_status cl_nn_pool_bwd(const void* dy, void* dx, int N, int D, int H, int W, int C, int xs, int xo, int accumulate,
                         void* stream);

/* y (window ys/yo, resolution 2D x 2H x 2W) = nearest upsampling of the
   dense x [N, D, H, W, C]. */
cl_status cl_nn_upsample(const void* x, void* y, int N, int D, int H, int W, int C, int ys, int yo, void* stream);

/* dx [N, D, H, W, C] (dense, overwritten) = sum over each 2x2x2 block of dy
   (window ys/yo at resolution 2D x 2H x 2W). */
cl_status cl_nn_upsample_bwd(const void* dy, void* dx, int N, int D, int H, int W, int C, int ys, int yo, void* stream);

/* dst[., dof + c] (=|+=) src[., so + c], c < C, over M voxels. */
cl_status cl_nn_copy_channels(const void* src, int ss, int so, void* dst, int ds, int dof, long long M, int C,
                              int accumulate, void* stream);

/* y[v] (FP32) = b[0] + sum_c w[c] x[v, c]: the 1x1x1 output head, x dense
   with C channels. */
cl_status cl_nn_head(const void* x, const float* w, const float* b, float* y, long long M, int C, void* stream);

/* loss[0] (FP64, device) = sum_v mask[v] (y[v] - target[v])^2 / sum mask
   (0 when no voxel is masked in), loss[1] = sum mask: a deterministic
   two-stage reduction; workspace holds 512 doubles. */
cl_status cl_nn_mse(const float* y, const float* target, const uint8_t* mask, long long M, double* workspace,
                    double* loss, void* stream);

/* Backward of cl_nn_head under cl_nn_mse: gy[v] = dL/dy[v], dx = gy w
   (BF16, overwritten), dw[c] and db[0] (FP32, overwritten).  `loss` is the
   device pair cl_nn_mse wrote (its mask count normalises the gradient). */
cl_status cl_nn_head_bwd(const void* x, const float* w, const float* y, const float* target, const uint8_t* mask,
                         const double* loss, void* dx, float* gy, float* dw, float* db, long long M, int C,
                         void* stream);

/* One Adam update (bias-corrected with the 1-based `step`) of n FP32 master
   parameters p from gradient g with moments m, v; p_bf16 (may be NULL)
   receives the BF16 copy the convolutions read. */
cl_status cl_nn_adam(float* p, const float* g, float* m, float* v, void* p_bf16, long long n, float lr, float b1, float b2,
                     float eps, int step, void* stream);

/* Error state of the network kernels since the last call: synchronises
   the stream, returns CL_ERR_TIMEOUT (and clears it) if a bounded wait of a
   tensor-core convolution expired (its output is then incomplete), else
   CL_OK; CL_ERR_CUDA if the state cannot be read. */
cl_status cl_nn_check(void* stream);

/* b = BF16(a), round to nearest even, n elements. */
cl_status cl_nn_to_bf16(const float* a, void* b, long long n, void* stream);

/* --- glue between a solver handle (cl_lbm.h) and the network --- */

/* Network input from the handle's set-up: feat [nz][ny][nx][16] BF16,
   channels 0 active (inlet-connected transport cell), 1 solid, 2 ionomer,
   3 micropore, 4 max(0, 1 + ln(D/D_max)/6) on active cells with
   D/D_max = (1/omega - 1/2)/(tau_ref - 1/2) (Eq. 24), 5 the linear ramp
   c_in + (c_out - c_in)(x + 1/2)/nx, 6 the series-resistor profile s(x):
   the inlet half cell, the links between planes x and x+1 and the outlet
   half cell in series, each with the mean over its ny*nz cross-section of
   the steady D3Q7 face conductance (2 D/D_max for a half cell, the harmonic
   2 D_a D_b/(D_a + D_b) for a link between two active cells, 0 otherwise),
   s(x) = c_in - (c_in - c_out) (R_inlet + sum_{x'<x} R_link(x')) / R_total;
   7 (s(x) - ramp(x)) nx / (4 (c_in - c_out)), 8..15 zero.
   Uses the handle's readout scratch; synchronises the stream.
   Errors: CL_ERR_STATE without a structure, CL_ERR_ARG for NULL. */
cl_status cl_lbm_features(cl_handle h, void* feat);

/* Training target from the handle's current field: target[v] (FP32) =
   (C[v] - ramp(x)) nx / (c_in - c_out) on active cells, 0 elsewhere (a
   scale-free deviation from the ramp).  Synchronises the stream. */
cl_status cl_lbm_target(cl_handle h, float* target);

/* Initialise the handle's state (as cl_lbm_init) from
   C0 = ramp(x) + pred[v] (c_in - c_out) / nx on active cells, 0 elsewhere:
   pred is FP32 on the device, in the units of cl_lbm_target (the network's
   output).  Errors as cl_lbm_init. */
cl_status cl_lbm_init_warm(cl_handle h, const float* pred);

#ifdef __cplusplus
}
#endif

#endif /* CL_NN_H */
