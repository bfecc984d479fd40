/*
 * kknet.h -- C ABI of the learned refiner that sits on top of KK
 * beamforming: a convolutional encoder-decoder that maps the complex (IQ)
 * KK image of a compressed pair set (e.g. a 6 x 12 vernier subset) to an
 * estimate of the KK image of the full pair set, trained on the GPU with
 * the library's own forward and backward kernels.  The paper has no
 * network; it names compressed pair sets as the way to trade image quality
 * for speed (Sections II-D and IV), and this refiner recovers part of the
 * quality lost.  The plain KK sum stays the fallback and the judge of the
 * refined image (kk_net_judge below).
 *
 * Network (fixed topology; widths from base channels C = 32):
 *   level 0 (H x W):      conv 16->C, conv C->C                   skip s0
 *   level 1 (H/2 x W/2):  pool, conv C->2C, conv 2C->2C           skip s1
 *   level 2 (H/4):        pool, conv 2C->4C, conv 4C->4C          skip s2
 *   level 3 (H/8):        pool, conv 4C->8C                       skip s3
 *   level 4 (H/16):       pool, conv 8C->8C
 *   decoder: up + s3, conv 8C->4C; up + s2, conv 4C->2C; up + s1,
 *            conv 2C->C; up + s0, conv C->C; head conv C->16
 *   out = in + head[:, 0:2]
 * All convolutions are 3 x 3 with zero padding and a bias, ReLU after all
 * but the head; pooling is 2 x 2 averaging, upsampling nearest-neighbour
 * and skips are added.  Input channels 0, 1 carry (re, im) of the input
 * image times a per-image scale; channels 2..15 are zero.  About 1.58 M
 * parameters at C = 32.
 *
 * Numerics: BF16 weights and activations, FP32 accumulation, FP32 master
 * weights, Adam moments and weight gradients.  Every reduction runs in a
 * fixed order, so a training step is bitwise reproducible on one device.
 *
 * Layouts: complex images are [nb][H][W] cfloat (interleaved re, im float32;
 * H = rows = depth z, W = columns = lateral x, as kk_beamform writes a
 * group's image).  Parameters are one flat float32 vector: per layer in the
 * order above, weights [cout][3][3][cin] then bias [cout].
 *
 * Conventions as in kkbeam.h: device pointers unless named h_*, calls that
 * take a stream only enqueue, errors are returned as kk_status with
 * kk_last_error().
 */
#ifndef KKNET_H
#define KKNET_H

#include "kkbeam.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kk_net kk_net;

typedef struct kk_net_desc {
  int32_t max_batch;      /* images per call, >= 1 */
  int32_t height, width;  /* multiples of 16, >= 16 */
  int32_t base_channels;  /* C, a multiple of 16 (32 for the described net) */
  uint64_t seed;          /* weight initialisation (He-normal; head near 0) */
} kk_net_desc;

/* Creates a network with freshly initialised weights and zero Adam state;
 * allocates its parameters and activation buffers for max_batch images on
 * the current device (synchronous).  KK_ERR_INVALID_ARG for bad sizes,
 * KK_ERR_OOM when the buffers do not fit. */
kk_status kk_net_create(kk_net **out, const kk_net_desc *d);
void kk_net_destroy(kk_net *net);
/* number of parameters (floats of the flat vector) and Adam steps taken */
kk_status kk_net_info(const kk_net *net, int64_t *n_params, int64_t *step);
/* Device status word of the net's tensor-core kernels, read and reset
 * (synchronous): KK_OK, or KK_ERR_TIMEOUT when a CTA gave up on a bounded
 * wait (its outputs are then invalid). */
kk_status kk_net_status(kk_net *net, int32_t *status);
/* copy the FP32 master parameters out / in (device buffers of n_params
 * floats); set also refreshes the BF16 copies.  Enqueued on `stream`. */
kk_status kk_net_get_params(const kk_net *net, float *d_dst, void *stream);
kk_status kk_net_set_params(kk_net *net, const float *d_src, void *stream);

/*
 * Forward pass of nb <= max_batch images: d_out = net(d_in * in_scale).
 * d_in_scale [nb] per-image factor (NULL = 1).  d_out [nb][H][W] cfloat is
 * in the scaled units of the input.
 */
kk_status kk_net_forward(kk_net *net, int32_t nb, const void *d_in, const float *d_in_scale,
                         void *d_out, void *stream);

/*
 * Loss and gradients: forward, then
 *   loss = sum over images, pixels and (re, im) of
 *          (out - target * target_scale)^2 / (2 nb H W),
 * written to d_loss[0] (device float), and backward into the net's FP32
 * gradient vector (copied to d_grad [n_params] when non-NULL).
 * d_out (nullable) receives the forward output.
 */
kk_status kk_net_loss_grad(kk_net *net, int32_t nb, const void *d_in, const float *d_in_scale,
                           const void *d_target, const float *d_target_scale, float *d_loss,
                           float *d_grad, void *d_out, void *stream);

/*
 * One Adam step (Kingma & Ba) on the gradient of the last kk_net_loss_grad:
 *   g += wd w;  m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),  t = step + 1.
 */
kk_status kk_net_adam(kk_net *net, float lr, float beta1, float beta2, float eps, float weight_decay,
                      void *stream);

/*
 * Checkpoint: parameters, Adam moments and step count in one file
 * (synchronises `stream` first; host file I/O).  Loading checks that the
 * file's topology (H, W, C, n_params) matches the net.  KK_ERR_INVALID_ARG
 * on a bad or mismatched file.
 */
kk_status kk_net_save(const kk_net *net, const char *path, void *stream);
kk_status kk_net_load(kk_net *net, const char *path, void *stream);

/*
 * Fallback judge.  kk_net_judge_filter sets, from the KK images of one point
 * scatterer formed with the compressed pair set (d_psf_c) and with the full
 * pair set (d_psf_f), both [H][W] cfloat on the net's grid, the k-space
 * filter G = DFT(psf_c) / DFT(psf_f) on the mask where both spectra reach
 * rho times their maxima (0 elsewhere).  G maps a full-pair image to the
 * compressed pair set's view of it (Section II-E: each pair is one k-space
 * sample, so a pair subset is a k-space mask).
 *
 * kk_net_judge writes two statistics per image n:
 *   d_stat[2n]   = 1 - |<G A, M C>|^2 / (|G A|^2 |M C|^2), the residual of
 *                  the best complex-scaled fit of the refined image, seen
 *                  through the compressed pair set, to the compressed KK
 *                  image (0 = consistent, 1 = unrelated);
 *   d_stat[2n+1] = energy of C outside M / energy of C: how far the input
 *                  is from being a KK image of the compressed pair set,
 *                  whose spectrum lies on M (0 = in band);
 * with A = DFT(d_out[n]), C = DFT(d_xc[n]) and M the mask (G != 0).  The
 * caller accepts d_out[n] when both are at most its tolerances (fixed on
 * training data) and otherwise falls back to the plain full-pair KK image.
 * Needs kk_net_judge_filter first (KK_ERR_INVALID_ARG otherwise).
 */
kk_status kk_net_judge_filter(kk_net *net, const void *d_psf_c, const void *d_psf_f, float rho,
                              void *stream);
kk_status kk_net_judge(kk_net *net, int32_t nb, const void *d_out, const void *d_xc, float *d_stat,
                       void *stream);

/* d_scale[n] = 1 / sqrt(mean over pixels of |d_img[n]|^2) (0 for an
 * all-zero image), for nb images of h x w cfloat: the per-image scale the
 * refiner's inputs and targets are normalised with. */
kk_status kk_net_image_scale(const void *d_img, int32_t nb, int32_t h, int32_t w, float *d_scale,
                             void *stream);

/*
 * Layer-level calls (the network's own kernels, for tests and tools).
 * x: [n][h][w][cin] bf16 NHWC, w: [cout][3][3][cin] bf16, bias [cout] fp32
 * (nullable); cin, cout multiples of 16.
 *   kk_nn_conv3x3:       y = act(conv(x, w) + bias) into d_y (bf16, nullable)
 *                        and / or d_yf (fp32, nullable), [n][h][w][cout];
 *                        tensor cores (tcgen05), FP32 accumulation
 *   kk_nn_conv3x3_dgrad: dx = conv(dy, flip(w)^T) (adjoint in x), bf16
 *                        [n][h][w][cin]; needs a workspace of
 *                        cout*9*cin*2 bytes
 *   kk_nn_status:        status word of the layer calls' tensor-core
 *                        kernels, read and reset (synchronous)
 *   kk_nn_conv3x3_wgrad: dw [cout][3][3][cin] and db [cout] (fp32,
 *                        overwritten) from x and dy [n][h][w][cout] bf16;
 *                        workspace size from kk_nn_conv3x3_wgrad_workspace
 */
kk_status kk_nn_conv3x3(const void *d_x, int32_t n, int32_t h, int32_t w, int32_t cin, const void *d_w,
                        int32_t cout, const float *d_bias, int32_t relu, void *d_y, float *d_yf,
                        void *stream);
kk_status kk_nn_conv3x3_dgrad(const void *d_dy, int32_t n, int32_t h, int32_t w, int32_t cout,
                              const void *d_w, int32_t cin, void *d_dx, void *d_workspace, void *stream);
kk_status kk_nn_status(int32_t *status);
kk_status kk_nn_conv3x3_wgrad_workspace(int32_t n, int32_t h, int32_t w, int32_t cin, int32_t cout,
                                        size_t *bytes);
kk_status kk_nn_conv3x3_wgrad(const void *d_x, int32_t n, int32_t h, int32_t w, int32_t cin,
                              const void *d_dy, int32_t cout, float *d_dw, float *d_db,
                              void *d_workspace, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* KKNET_H */
