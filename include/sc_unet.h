/*
 * sc_unet.h -- C ABI of the BF16 U-Net denoiser trained and run on the GB300 tensor cores.
 *
 * The paper evaluates its images with a U-Net (Sec. IV-A, after Ronneberger et al. 2015); here a
 * U-Net of that family denoises low-sample renders.  Its input is 11 channels per pixel:
 * log1p of the noisy linear RGB (3), the first-hit albedo (3), the first-hit normal (3), the
 * normalised depth (1) and the object mask (1), i.e. the ground-truth buffers of Sec. III-D.
 * Its output is 3 channels: log1p of the denoised RGB.
 *
 * Architecture (fixed): 4 levels of widths 32, 48, 64, 128.  Encoder level l: [2x2 max pool if
 * l > 0] -> 3x3 conv + ReLU -> 3x3 conv + ReLU.  Decoder level l (deepest first): 2x2 stride-2
 * transposed conv -> concatenate [upsampled, encoder output of level l] -> 3x3 conv + ReLU ->
 * 3x3 conv + ReLU.  Output: 1x1 conv.  Zero padding; max-pool ties go to the first element of
 * the window in row-major order; 585,363 parameters.
 *
 * Loss (training): 0.16 * mean |p - t| + 0.84 * (1 - mean SSIM(p, t)), SSIM of Wang et al.
 * (2004) over valid 11x11 Gaussian windows (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2, averaged over
 * windows, channels and images.  Optimiser: Adam, beta1 0.9, beta2 0.999, eps 1e-8, bias
 * corrected.
 *
 * Precision: weights and activations are BF16, every contraction accumulates in FP32 on the
 * tensor cores (tcgen05.mma), biases, gradients of parameters, Adam state and master weights
 * are FP32.
 *
 * Parameters are exchanged as one flat FP32 vector: the tensors below in this order, each
 * row-major (C order):
 *   for l = 0..3:  enc{l}_c1_w (c_l, 3, 3, cin) , enc{l}_c1_b (c_l),
 *                  enc{l}_c2_w (c_l, 3, 3, c_l), enc{l}_c2_b (c_l)       (cin = 11, then c_{l-1})
 *   for l = 2..0:  up{l}_w (c_{l+1}, 2, 2, c_l), up{l}_b (c_l),
 *                  dec{l}_c1_w (c_l, 3, 3, 2 c_l), dec{l}_c1_b (c_l),
 *                  dec{l}_c2_w (c_l, 3, 3, c_l), dec{l}_c2_b (c_l)
 *   out_w (3, 32), out_b (3)
 * Conv weight w[o][dy][dx][c] multiplies input pixel (y + dy - 1, x + dx - 1); transposed-conv
 * weight w[c][a][e][o] maps input pixel (y, x) to output pixel (2y + a, 2x + e).
 *
 * Conventions: as in supercaustics.h (status codes, asynchronous work on the context stream,
 * caller-owned device buffers).  Images are NHWC FP32, H and W multiples of 8 and >= 16.
 */
#ifndef SC_UNET_H
#define SC_UNET_H

#include "supercaustics.h"

#ifdef __cplusplus
extern "C" {
#endif

#define SC_UNET_IN_CH 11
#define SC_UNET_OUT_CH 3
#define SC_UNET_LEVELS 4

typedef struct sc_unet sc_unet;

/* Number of FP32 values in the flat parameter vector (585,363). */
int sc_unet_param_count(int64_t *count);

/* Creates a network with workspace for up to max_batch images of height x width.
 * Parameters start at zero; Adam moments at zero, step 0. */
int sc_unet_create(sc_ctx *ctx, int32_t max_batch, int32_t height, int32_t width, sc_unet **out);
int sc_unet_destroy(sc_ctx *ctx, sc_unet *net);

/* Copies the flat FP32 parameters in (device pointer) and refreshes the BF16 copies the kernels
 * read.  Resets the Adam moments and the step count. */
int sc_unet_set_params(sc_ctx *ctx, sc_unet *net, const float *params);
/* Copies the flat FP32 master parameters out (device pointer, sc_unet_param_count floats). */
int sc_unet_get_params(sc_ctx *ctx, const sc_unet *net, float *params);
/* Gradient of the last sc_unet_loss_grad, same flat layout (device pointers). */
int sc_unet_get_grads(sc_ctx *ctx, const sc_unet *net, float *grads);
int sc_unet_set_grads(sc_ctx *ctx, sc_unet *net, const float *grads);

/* Inference: x [n, H, W, 11] FP32 (device) -> y [n, H, W, 3] FP32 (device); 1 <= n <= max_batch. */
int sc_unet_forward(sc_ctx *ctx, sc_unet *net, const float *x, int32_t n, float *y);

/* Forward, loss against target [n, H, W, 3] FP32 (device), and backward; the parameter gradient
 * is kept inside (sc_unet_get_grads).  y (optional, device) receives the prediction, loss
 * (optional, device) one FP32 value. */
int sc_unet_loss_grad(sc_ctx *ctx, sc_unet *net, const float *x, const float *target, int32_t n, float *y,
                      float *loss);

/* One Adam step with the stored gradient (step count += 1) and refresh of the BF16 copies. */
int sc_unet_adam(sc_ctx *ctx, sc_unet *net, float lr);

/* sc_unet_loss_grad followed by sc_unet_adam. */
int sc_unet_train_step(sc_ctx *ctx, sc_unet *net, const float *x, const float *target, int32_t n, float lr,
                       float *loss);

/* Training loss of sc_unet_loss_grad / sc_unet_train_step (default SC_UNET_LOSS_L1_SSIM, above).
 * SC_UNET_LOSS_BCE trains a segmentation network (the paper's Sec. IV trains its U-Net to segment
 * transparent objects and caustics): output channel 0 is a logit, target channel 0 a label in
 * [0, 1], loss = mean over pixels of softplus(y) - t y (binary cross-entropy with logits, FP64
 * partial sums in a fixed order); output channels 1 and 2 and target channels 1 and 2 take no part
 * (zero gradient).
 * SC_UNET_LOSS_L2_LINEAR: squared error in linear radiance, outputs and targets being log1p values:
 * mean over pixels and the three channels of (expm1(y) - expm1(t))^2 (FP64 partial sums in a fixed
 * order).  Trained on noisy targets it converges to their linear mean, which is what an MSE against
 * a converged reference rewards.  The loss stays set until changed. */
enum { SC_UNET_LOSS_L1_SSIM = 0, SC_UNET_LOSS_BCE = 1, SC_UNET_LOSS_L2_LINEAR = 2 };
int sc_unet_set_loss(sc_ctx *ctx, sc_unet *net, int32_t kind);

/* Training state (checkpoint / resume).  The state is the FP32 master parameters, the two Adam
 * moment vectors (sc_unet_param_count floats each, same flat layout) and the Adam step count, which
 * sets the bias corrections of the next step.  Restoring all of it and repeating the same calls
 * continues training bit for bit as if it had not been interrupted (every kernel of a training
 * step is deterministic).
 * sc_unet_get_state: copies the moments to adam_m / adam_v (device, either may be NULL) and the
 *   step count to *step (host, may be NULL).  Parameters: sc_unet_get_params.
 * sc_unet_set_state: parameters, moments (device) and step count in one call; refreshes the BF16
 *   copies the kernels read.  SC_ERR_INVALID_ARG on a null buffer or a step outside [0, 2^31).
 * sc_unet_save: writes the whole state to the file `path` (binary: an 8-byte tag "SCUNET1", the
 *   parameter count, the step count and the four level widths as int64, then the parameters,
 *   the first moment and the second moment as FP32, little-endian).  Synchronises the context
 *   stream.  SC_ERR_INVALID_ARG if the file cannot be written.
 * sc_unet_load: reads such a file into the network (any batch size or geometry: the state does
 *   not depend on them); SC_ERR_INVALID_ARG, with the network unchanged, if the file is missing,
 *   truncated or holds another architecture.  Synchronises the context stream. */
int sc_unet_get_state(sc_ctx *ctx, const sc_unet *net, float *adam_m, float *adam_v, int64_t *step);
int sc_unet_set_state(sc_ctx *ctx, sc_unet *net, const float *params, const float *adam_m, const float *adam_v,
                      int64_t step);
int sc_unet_save(sc_ctx *ctx, const sc_unet *net, const char *path);
int sc_unet_load(sc_ctx *ctx, sc_unet *net, const char *path);

/* The loss alone: pred, target [n, h, w, 3] FP32 (device); loss (device, 1 float, optional);
 * grad (device, [n, h, w, 3] FP32, optional) = d loss / d pred.  h, w >= 11. */
int sc_ssim_l1_loss(sc_ctx *ctx, const float *pred, const float *target, int32_t n, int32_t h, int32_t w,
                    float *loss, float *grad);

/* Which radiance estimate a network input / target is built from: the full image (camera paths
 * + light-traced caustics, sc_frame.rgb), the camera estimator alone (sc_frame.direct), in
 * which case the caustic buffer is added back after denoising (sc_unet_output_rgb's `add`), or
 * the light-traced caustic buffer alone (sc_frame.caustic), for a network that denoises the
 * caustics beside one that denoises the camera estimate. */
enum { SC_UNET_SRC_RGB = 0, SC_UNET_SRC_DIRECT = 1, SC_UNET_SRC_CAUSTIC = 2 };

/* Builds the 11-channel network input from a rendered frame's buffers (supercaustics.h
 * sc_frame: rgb or direct, albedo, normal_camera, depth_norm, mask) for image `index` of a
 * batch: x + index * H * W * 11 receives [log1p(max(L, 0)), albedo, normal, depth_norm,
 * mask != 0], L the estimate selected by `source`. */
int sc_unet_pack_frame(sc_ctx *ctx, const sc_frame *frame, int32_t source, float *x, int32_t index);

/* Training target of a rendered frame: t + index * H * W * 3 receives log1p(max(L, 0)). */
int sc_unet_pack_target(sc_ctx *ctx, const sc_frame *frame, int32_t source, float *t, int32_t index);
/* Denoised linear RGB from network outputs: rgb[p] = (expm1(y[p][0..2]) clamped at 0, plus
 * add[p].xyz when add is given, 1) for n_px pixels; y FP32 [n_px][3], add float4 [n_px] or NULL,
 * rgb float4 [n_px] (all device). */
int sc_unet_output_rgb(sc_ctx *ctx, const float *y, int64_t n_px, const float *add, float *rgb);

/* Self-test of the failure path shared by the tensor-core kernels (test use).  One CTA takes
 * the roles of a convolution CTA: a producer with a bulk copy in flight, an MMA issuer with one
 * MMA in flight (128 x 32 x 16, all-ones operands) and two epilogue warps; then each role waits on
 * an mbarrier that nothing arrives at.  After poll_limit polls (1 .. 2^24; the kernels use 2^24)
 * every wait gives up and raises the CTA's abort flag; the producer then waits (bounded) for its
 * copy, the issuer commits its MMA to a drain barrier and waits for it, the CTA frees its TMEM and
 * latches SC_STATUS_WATCHDOG in the context's status word, so the next sc_sync_status returns
 * SC_ERR_TIMEOUT (and clears it); the context stays usable.  out_host (host, 8 x int64):
 * [0] producer gave up, [1] its copy completed, [2] issuer gave up, [3] its MMA drained,
 * [4] the drained accumulator holds 16 everywhere, [5] epilogue warps that gave up (2),
 * [6] the copied bytes arrived intact, [7] nanoseconds the issuer spent in the abandoned wait.
 * Synchronises the context's stream. */
int sc_unet_wait_selftest(sc_ctx *ctx, uint32_t poll_limit, int64_t *out_host);

/* Internal tensors, for inspection by tests: id below, level 0..3. */
enum {
  SC_UNET_BUF_INPUT = 0,  /* BF16 network input, 16 channels (11 + zero padding), level 0 */
  SC_UNET_BUF_ENC1 = 1,   /* BF16 output of encoder conv 1 (after ReLU) */
  SC_UNET_BUF_ENC2 = 2,   /* BF16 output of encoder conv 2 (after ReLU): the skip tensor */
  SC_UNET_BUF_POOL = 3,   /* BF16 max-pooled input of encoder level l >= 1 */
  SC_UNET_BUF_UP = 4,     /* BF16 transposed-conv output at level l <= 2 */
  SC_UNET_BUF_DEC1 = 5,   /* BF16 decoder conv 1 output (after ReLU), l <= 2 */
  SC_UNET_BUF_DEC2 = 6,   /* BF16 decoder conv 2 output (after ReLU), l <= 2 */
  SC_UNET_BUF_OUT = 7,    /* FP32 network output, 3 channels, level 0 */
  SC_UNET_BUF_GOUT = 8,   /* BF16 d loss / d output, 8 channels (3 + zero padding), level 0 */
  SC_UNET_BUF_GDEC2 = 9,  /* BF16 d loss / d (pre-ReLU) decoder conv 2 output, l <= 2 */
  SC_UNET_BUF_GDEC1 = 10, /* BF16 d loss / d (pre-ReLU) decoder conv 1 output, l <= 2 */
  SC_UNET_BUF_GUP = 11,   /* BF16 d loss / d transposed-conv output, l <= 2 */
  SC_UNET_BUF_GSKIP = 12, /* FP32 d loss / d skip tensor through the concatenation, l <= 2 */
  SC_UNET_BUF_GENC2 = 13, /* BF16 d loss / d (pre-ReLU) encoder conv 2 output */
  SC_UNET_BUF_GENC1 = 14  /* BF16 d loss / d (pre-ReLU) encoder conv 1 output */
};
typedef struct {
  int32_t dtype;    /* 0 BF16, 1 FP32 */
  int32_t n, h, w;  /* images of the last call, geometry of the level */
  int32_t c;        /* logical channels */
} sc_unet_buffer_info;
int sc_unet_buffer(const sc_unet *net, int32_t id, int32_t level, sc_unet_buffer_info *info);
/* Copies the buffer densely ([n, h, w, c], its dtype) to dst (device). */
int sc_unet_copy_buffer(sc_ctx *ctx, const sc_unet *net, int32_t id, int32_t level, void *dst);

#ifdef __cplusplus
}
#endif
#endif
