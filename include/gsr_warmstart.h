/*
 * gsr_warmstart.h -- C ABI of the learned tracking warm-start network.
 *
 * The paper has no learned component: its tracker starts every frame from a
 * constant-velocity extrapolation of the two previous poses (Sec. 3.5) and
 * runs a fixed number of gradient iterations.  This network predicts, from the
 * residual between a low-resolution render at that initial pose and the input
 * frame, the left-multiplied twist that takes the initial pose to the true one,
 * so the tracker can start closer to its optimum.  The plain tracker remains
 * the fallback.
 *
 * Network (all sizes fixed):
 *   input   x [B, 120, 160, 8] FP32, NHWC; channel order
 *           (rendered R, G, B, rendered depth / 5 m,
 *            input - rendered R, G, B, (input - rendered depth) / 5 m or 0)
 *   6 x (3x3 convolution, stride 2, zero padding 1, bias, ReLU)
 *           channels 8 -> 32 -> 64 -> 128 -> 128 -> 256 -> 256,
 *           spatial 120x160 -> 60x80 -> 30x40 -> 15x20 -> 8x10 -> 4x5 -> 2x3
 *   dense 1536 -> 256 (ReLU) -> 6;  output [B, 6] = (rho, phi), translation
 *           first, a left perturbation T <- exp(xi^) T of the world-to-camera pose.
 * Arithmetic: BF16 weights and activations, FP32 accumulation on the tensor
 * cores; FP32 master weights, biases, gradients and Adam moments.
 *
 * Flat parameter vector (FP32, n = gsr_warmstart_num_params()): for each
 * layer in order, its weight then its bias; convolution weights are
 * [C_out][3][3][C_in], dense weights [out][in]; dense 1 reads its input
 * flattened in (y, x, c) order.
 *
 * Ownership and errors: every tensor argument is caller-owned DEVICE memory,
 * FP32, contiguous, unless marked host.  The network object owns its weights,
 * moments and activation scratch (sized for max_batch at creation).  Calls
 * are asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 * stream); argument errors return GSR_ERR_INVALID_ARG before any CUDA call,
 * CUDA failures GSR_ERR_CUDA / GSR_ERR_OOM, a batch above max_batch
 * GSR_ERR_CAPACITY; gsr_warmstart_last_error() describes the last failure.
 * One network object must not be used from two host threads at once.
 */
#ifndef GSR_WARMSTART_H
#define GSR_WARMSTART_H

#include "gsr.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsr_warmstart gsr_warmstart;

#define GSR_WS_IN_H 120
#define GSR_WS_IN_W 160
#define GSR_WS_IN_C 8
#define GSR_WS_OUT 6

/* Number of FP32 parameters of the network (no CUDA call). */
GSR_API int64_t gsr_warmstart_num_params(void);

/* Create a network for batches of up to max_batch (1..1024) samples, weights
 * He-normal from `seed` (the output layer scaled by 0.01), biases 0. */
GSR_API gsr_status gsr_warmstart_create(gsr_warmstart **out, int32_t max_batch, uint64_t seed);
GSR_API void gsr_warmstart_destroy(gsr_warmstart *net);
GSR_API const char *gsr_warmstart_last_error(const gsr_warmstart *net);

/* Copy the flat FP32 parameter vector in (re-deriving the BF16 copies) or out.
 * The Adam moments are reset by set_params. */
GSR_API gsr_status gsr_warmstart_set_params(gsr_warmstart *net, const float *params, void *stream);
GSR_API gsr_status gsr_warmstart_get_params(gsr_warmstart *net, float *params, void *stream);

/* out[B, 6] = f(x[B, 120, 160, 8]).  Keeps the activations for a following
 * gsr_warmstart_backward of the same batch.  out may be NULL.  x must be
 * 16-byte aligned (GSR_ERR_INVALID_ARG otherwise). */
GSR_API gsr_status gsr_warmstart_forward(gsr_warmstart *net, const float *x, int32_t batch, float *out,
                                         void *stream);

/* Gradient of sum(d_out * out) over the last forward's batch with respect to
 * the flat parameter vector, written to grad[n_params] (may be NULL: the
 * gradient then stays in the network's own buffer for a later Adam step). */
GSR_API gsr_status gsr_warmstart_backward(gsr_warmstart *net, const float *d_out, int32_t batch, float *grad,
                                          void *stream);

typedef struct {
    float lr;           /* Adam step size, default 1e-3 */
    float beta1, beta2; /* default 0.9, 0.999 */
    float eps;          /* default 1e-8 */
    float w[6];         /* per-output loss weights, default (1, 1, 1, 1, 1, 1) */
} gsr_warmstart_opts;

GSR_API void gsr_warmstart_default_opts(gsr_warmstart_opts *o);

/* Kernel choice for the forward products: those with a reduction length
 * K >= tcgen05_min_k run on the 5th-generation tensor cores (tcgen05.mma,
 * accumulators in tensor memory), the others -- and all of them when
 * tcgen05_min_k < 0 -- on the mma.sync kernel that also runs the backward
 * products.  Results agree to FP32 summation order.  The default is -1: on
 * GB300 the mma.sync kernel measured faster for every layer of this network
 * (its products are narrow and bound by operand movement). */
GSR_API gsr_status gsr_warmstart_set_kernels(gsr_warmstart *net, int32_t tcgen05_min_k);

/* Synchronises `stream` and returns GSR_ERR_TIMEOUT (clearing it) if a
 * tensor-core kernel's bounded wait expired since the last check; its
 * outputs are then invalid. */
GSR_API gsr_status gsr_warmstart_check(gsr_warmstart *net, void *stream);

/* One training step on a batch: forward, loss
 *   L = (1/B) sum_b sum_c w_c (out[b,c] - target[b,c])^2,
 * backward, Adam on the FP32 masters and re-derivation of the BF16 copies.
 * target [B, 6] device; loss (device, one float) may be NULL. */
GSR_API gsr_status gsr_warmstart_train_step(gsr_warmstart *net, const float *x, const float *target, int32_t batch,
                                            const gsr_warmstart_opts *opts, float *loss, void *stream);

/* Network input for one frame: the render at the initial pose made at
 * 160 x 120 (rgb_r [3,120,160], depth_r [120,160]) and the input frame at its
 * own resolution (rgb_i [3,h,w], depth_i [h,w]), box-averaged to 160 x 120
 * (output pixel (i, j) averages input rows [floor(i h/120), floor((i+1) h/120))
 * and the matching columns; depth averages only pixels with depth > 0, 0 if
 * none).  Depth channels are divided by depth_scale; the depth residual is 0
 * where either depth is 0.  out [120, 160, 8]; h >= 120, w >= 160. */
GSR_API gsr_status gsr_warmstart_make_input(const float *rgb_r, const float *depth_r, const float *rgb_i,
                                            const float *depth_i, int32_t h, int32_t w, float depth_scale,
                                            float *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif
