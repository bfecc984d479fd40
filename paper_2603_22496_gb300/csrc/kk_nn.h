// kk_nn.h -- kernels of the learned refiner (convolutional encoder-decoder).
// Internal to the library; the public calls are in include/kknet.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

namespace kk {
namespace nn {

// NHWC bfloat16 activation tensor; c is a multiple of 16 for every tensor a
// convolution reads.
struct Tensor4 {
  __nv_bfloat16 *p;
  int n, h, w, c;
  size_t count() const { return (size_t)n * h * w * c; }
};

// y = act(conv3x3(x, w) + bias), zero padding 1, stride 1, on the tensor
// cores (tcgen05, TMEM accumulator).  w is [cout][3][3][cin] bf16; bias
// (nullable) fp32; y bf16 and / or yf fp32 (either nullable), both
// [pixels][cout]; cin, cout multiples of 16.  A CTA that gives up on a
// bounded wait writes KK_ERR_TIMEOUT to *status (nullable: the library's
// layer status word).
cudaError_t conv3x3_tc(const Tensor4 &x, const __nv_bfloat16 *w, int cout, const float *bias, bool relu,
                       __nv_bfloat16 *y, float *yf, int *status, cudaStream_t s);
// read and reset the layer status word
cudaError_t conv_status(int *out);

// TMA-fed forms (kk_conv_tma.cu) for shapes whose pixel tiles are whole row
// segments or rows of one image: return false (nothing launched) when the
// shape does not qualify, else launch and put the launch error in *err.
bool conv3x3_tma(const Tensor4 &x, const __nv_bfloat16 *w, int cout, const float *bias, bool relu,
                 __nv_bfloat16 *y, float *yf, int *status, cudaStream_t s, cudaError_t *err);
bool wgrad_tma(const Tensor4 &x, const __nv_bfloat16 *dy, int cout, float *part, int splits, int pix_per_split,
               int *status, cudaStream_t s, cudaError_t *err);
cudaError_t tma_status(int *out);

// Weight (and bias) gradient of a 3x3 convolution on the tensor cores.  The
// weight partial sums of pixel split i go to part[i][cout * 9 * cin]
// (n_split splits), then the bias partials of pixel block b to
// part[n_split * cout * 9 * cin + b * cout + co] (n_bias blocks);
// reduce_splits sums each in a fixed order (deterministic).
int wgrad_splits(const Tensor4 &x, int cout);
int bias_blocks(int pixels, int cout);
size_t wgrad_part_floats(const Tensor4 &x, int cout);
cudaError_t conv3x3_wgrad(const Tensor4 &x, const __nv_bfloat16 *dy, int cout, float *part, int *n_split,
                          int *n_bias, int *status, cudaStream_t s);
// out[j] = sum_{i < n_part} part[i * stride + j] for j < n_out, in a fixed order
cudaError_t reduce_splits(const float *part, int n_part, size_t stride, size_t n_out, float *out,
                          cudaStream_t s);

// backward-data weights: wt[ci][2-kh][2-kw][co] = w[co][kh][kw][ci]
cudaError_t flip_transpose(const __nv_bfloat16 *w, int cout, int cin, __nv_bfloat16 *wt, cudaStream_t s);

cudaError_t relu_bwd(__nv_bfloat16 *dy, const __nv_bfloat16 *y, size_t n, cudaStream_t s);
cudaError_t pool2(const Tensor4 &x, __nv_bfloat16 *y, cudaStream_t s);
// dx (= or +=) adjoint of pool2 applied to dy (dx has the full resolution)
cudaError_t pool2_bwd(const __nv_bfloat16 *dy, const Tensor4 &dx, bool accumulate, cudaStream_t s);
cudaError_t up2(const Tensor4 &x, __nv_bfloat16 *y, cudaStream_t s);
// dx = adjoint of up2 applied to dy (dx has the half resolution)
cudaError_t up2_bwd(const __nv_bfloat16 *dy, const Tensor4 &dx, cudaStream_t s);
// y = up2(x) + skip  (skip has y's shape)
cudaError_t up2_add(const Tensor4 &x, const __nv_bfloat16 *skip, __nv_bfloat16 *y, cudaStream_t s);

// complex images [nb][hw] -> NHWC bf16 with c channels (re, im, zeros),
// multiplied by scale[n] (nullable: 1)
cudaError_t pack_iq(const float2 *img, const float *scale, int nb, int hw, int c, __nv_bfloat16 *x,
                    cudaStream_t s);
// out = x[:, 0:2] + head[:, 0:2]; with a target t: per-block squared-error
// partials in block_loss[] and dhead = d loss / d head, loss =
// sum (out - t * tscale)^2 / (2 nb hw).  Returns the number of blocks.
int residual_blocks(int nb, int hw);
cudaError_t residual_mse(const __nv_bfloat16 *xin, int cx, const float *head, int ch, const float2 *target,
                         const float *tscale, int nb, int hw, float2 *out, __nv_bfloat16 *dhead,
                         float *block_loss, cudaStream_t s);
// loss = sum(part[0..n)) * k, fixed-order tree in one block
cudaError_t sum_scalar(const float *part, int n, float k, float *loss, cudaStream_t s);

cudaError_t adam(float *w, const float *g, float *m, float *v, __nv_bfloat16 *wb, size_t n, float lr, float b1,
                 float b2, float eps, float bc1, float bc2, float wd, cudaStream_t s);
cudaError_t to_bf16(const float *a, __nv_bfloat16 *b, size_t n, cudaStream_t s);

// 2-D DFT of nb complex h x w images, exp(sign 2 pi i (jk/L)) per axis
cudaError_t dft2(const float2 *in, int nb, int h, int w, int sign, float2 *tmp, float2 *out, cudaStream_t s);
// judge filter from the two point-spread spectra: mask where both
// magnitudes reach rho times their maxima, G = Sc / Sf there, 0 elsewhere
cudaError_t judge_filter(const float2 *Sc, const float2 *Sf, int hw, float rho, float2 *G, cudaStream_t s);
// per image n: stat[2n] = 1 - |<G A, M C>|^2 / (|G A|^2 |M C|^2),
// stat[2n+1] = energy of C outside M / energy of C; A = DFT(out),
// C = DFT(xc), M = (G != 0)
cudaError_t judge_stat(const float2 *A, const float2 *C, const float2 *G, int nb, int hw, float *stat,
                       cudaStream_t s);
// scale[n] = 1 / sqrt(mean |img_n|^2), 0 for an all-zero image
cudaError_t image_scale(const float2 *img, int nb, int hw, float *scale, cudaStream_t s);

}  // namespace nn
}  // namespace kk
