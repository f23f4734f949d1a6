/* C ABI of the warm-start network kernels.
 *
 * The paper has no learned component.  These entry points train and run a
 * small convolutional network that predicts the steady density and velocity
 * of a lid-driven cavity from its geometry and Reynolds number; the
 * prediction only initialises the RMRT-LB solver (rmrtlb_batch_init_fields,
 * with the non-equilibrium part of Eq. fne), whose own residual decides
 * convergence.  Network: four 3 x 3 x 3 convolutions with zero padding,
 * 8 -> 32 -> 32 -> 32 -> 4 channels, SiLU between them; BF16 activations
 * and weights, FP32 accumulation, FP32 master weights.
 *
 * Layout: activations (n, d, h, w, c), channels last, w (x) fastest among
 * the spatial axes; weights (27, cin, cout) with tap t = 9 (dz + 1) +
 * 3 (dy + 1) + (dx + 1); output voxel v reads input voxel v + (dz, dy, dx)
 * (zero outside the volume).  BF16 values are passed as uint16_t bit
 * patterns.  Every pointer is device memory owned by the caller, 16-byte
 * aligned, unless stated otherwise.  Calls are asynchronous on `stream`
 * (a cudaStream_t, NULL for the legacy stream) and return RMRTLB_OK,
 * RMRTLB_EINVAL (bad size, unsupported channel pair, misaligned or NULL
 * pointer) or RMRTLB_ECUDA (launch failure); a give-up of a bounded wait
 * inside a kernel is reported by rmrtlb_cnn_check (RMRTLB_ETIMEOUT).  Sizes: n d h w < 2^31. */
#ifndef RMRTLB_CNN_H
#define RMRTLB_CNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Forward convolution, channel pairs (cin, cout) = (8, 32), (32, 32),
 * (32, 4):  z[v, co] = bias[co] + sum_t sum_ci x[v + tap_t, ci] w[t, ci, co]
 * in FP32 from BF16 x and w, as an implicit GEMM on the tensor cores
 * (tcgen05.mma kind::f16, FP32 accumulator in tensor memory; M = 128 voxels,
 * N = cout, K = 27 taps x cin).  Writes z (FP32, NULL to skip) and
 * a = silu(z) (apply_silu != 0) or z, rounded to BF16 (NULL to skip).
 * Every wait for tensor-core completion is bounded; a wait that gives up
 * leaves the output unwritten and is reported by rmrtlb_cnn_check. */
int rmrtlb_conv3d_forward(int n, int d, int h, int w, int cin, int cout,
                          const uint16_t* x, const uint16_t* weight, const float* bias,
                          int apply_silu, float* z, uint16_t* a, void* stream);

/* Bytes of device scratch rmrtlb_conv3d_backward_data can use (host only):
 * a BF16 copy of dy (cout = 32, or cout = 4 padded to 8 channels) when the
 * plane holds a 128-voxel box (the copy-fed kernel then runs), else 0. */
size_t rmrtlb_conv3d_backward_data_scratch(int n, int d, int h, int w, int cin, int cout);

/* Gradient with respect to the input, channel pairs (32, 32), (32, 4):
 * dx[v, ci] = sum_t sum_co dy[v - tap_t, co] w[t, ci, co], multiplied by
 * silu'(z_in[v, ci]) when z_in (the FP32 pre-activation that produced x)
 * is not NULL; the same tensor-core implicit GEMM with dy rounded to BF16
 * (nearest even).  dy, z_in, dx FP32.  With `scratch` (device, 16-byte
 * aligned, at least rmrtlb_conv3d_backward_data_scratch bytes) dy is first
 * rounded into it and the kernel is fed by the tensor-memory accelerator;
 * with NULL (or a short scratch) the threads gather and round dy
 * themselves.  Both give the same result. */
int rmrtlb_conv3d_backward_data(int n, int d, int h, int w, int cin, int cout,
                                const float* dy, const uint16_t* weight, const float* z_in,
                                float* dx, void* scratch, size_t scratch_bytes, void* stream);

/* Bytes of device scratch rmrtlb_conv3d_backward_weight needs (host only):
 * per-chunk partial sums of dweight and dbias, and on planes that hold a
 * 128-voxel box a BF16 copy of dy (cout = 4 padded to 8 channels). */
size_t rmrtlb_conv3d_backward_weight_scratch(int n, int d, int h, int w, int cin, int cout);

/* Gradient with respect to the weights and the bias, all three channel
 * pairs: dweight[t, ci, co] = sum_v x[v + tap_t, ci] dy[v, co] on the tensor
 * cores (a GEMM with K = voxels, M = taps x cin, both operands MN-major in
 * shared memory; dy rounded to BF16, nearest even), dbias[co] = sum_v dy[v,
 * co] on the FP32 pipes.  On planes that hold a 128-voxel box the
 * operands are brought by the tensor-memory accelerator box by box
 * (dy first rounded into the scratch) and dweight is summed per chunk of
 * 32 boxes; otherwise threads gather them and dweight is summed per chunk
 * of 4096 voxels; dbias is summed per chunk of 1024 voxels.  The partial
 * sums are then added over the chunks in a fixed order, so repeated calls
 * give bitwise the same result.  x, dy and scratch 16-byte aligned; scratch
 * at least rmrtlb_conv3d_backward_weight_scratch bytes (else
 * RMRTLB_ENOMEM). */
int rmrtlb_conv3d_backward_weight(int n, int d, int h, int w, int cin, int cout,
                                  const uint16_t* x, const float* dy, float* dweight, float* dbias,
                                  void* scratch, size_t scratch_bytes, void* stream);

/* Mean squared error of y against t (count FP32 values): dy = 2 (y - t) /
 * count, *loss = mean (y - t)^2 in FP64 (device pointer), summed in a fixed
 * order through `scratch` (device, at least 8192 bytes). */
int rmrtlb_mse(long long count, const float* y, const float* t, float* dy, double* loss,
               void* scratch, void* stream);

/* One Adam step (Kingma and Ba, Algorithm 1, bias-corrected) on count FP32
 * parameters with gradient grad and moments m, v (updated in place); step
 * counts from 1.  param_bf16 (may be NULL) receives the updated parameters
 * rounded to BF16. */
int rmrtlb_adam(long long count, float* param, uint16_t* param_bf16, const float* grad,
                float* m, float* v, int step, float lr, float beta1, float beta2, float eps,
                void* stream);

/* Network input of n cavities of d x h x w cells (BF16, 8 channels): the
 * cell-centred coordinates xh, yh, zh in (-1, 1), rh = (Re - 800) / 700,
 * and xh zh, yh zh, zh^2, rh zh.  re: n FP64 Reynolds numbers, device. */
int rmrtlb_cavity_features(int n, int d, int h, int w, const double* re, uint16_t* x,
                           void* stream);

/* Trilinear interpolation of src (d, h, w, c; FP32, c <= 8) between
 * cell-centred grids of one box onto D x H x W, written as c FP64 planes
 * dst[k] = offset[k] + scale[k] * value (scale, offset: host arrays of c
 * values).  Fine cell I of N along an axis reads source coordinate
 * (I + 1/2) n / N - 1/2, clamped to [0, n - 1]. */
int rmrtlb_upsample_fields(int d, int h, int w, int c, const float* src, int D, int H, int W,
                           const double* scale, const double* offset, double* dst, void* stream);

/* Synchronises `stream` and returns RMRTLB_ETIMEOUT if any tensor-core
 * convolution since the last call gave up waiting for its MMAs (a bounded
 * wait; the kernel then skips its outputs and returns), RMRTLB_ECUDA if the
 * stream reports an error, else RMRTLB_OK.  Clears the condition. */
int rmrtlb_cnn_check(void* stream);

/* Self-test of that bounded wait (no counterpart in the paper): one thread
 * initialises an mbarrier that nothing arrives on and waits for it with the
 * same polling routine the convolutions use, giving up after `polls` polls
 * (1 <= polls <= 2^20, else RMRTLB_EINVAL); the give-up is recorded exactly
 * as a convolution's, so the next rmrtlb_cnn_check returns
 * RMRTLB_ETIMEOUT, and the context stays usable. */
int rmrtlb_cnn_wait_selftest(unsigned polls, void* stream);

/* Training targets of one cavity from its fields: for each of n nodes,
 * out[4 i + 0] = (rho[i] - rho0) * rho_scale, out[4 i + 1 + a] =
 * u[a n + i] * u_scale (a < 3; zero for a missing third component when
 * d = 2).  rho, u FP64 planes (device), out FP32 (device). */
int rmrtlb_pack_fields(long long n, int d, const double* rho, const double* u, double rho0,
                       double rho_scale, double u_scale, float* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RMRTLB_CNN_H */
