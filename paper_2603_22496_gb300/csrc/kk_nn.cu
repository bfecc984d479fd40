// kk_nn.cu -- the learned refiner's kernels around its convolutions (which
// are in kk_conv_tc.cu): split-partial reduction, backward-data weight
// flip, ReLU backward, pooling and upsampling with their adjoints, input
// packing, residual output and loss, Adam, and the fallback judge (2-D DFT,
// k-space filter, consistency statistic).
//
// Activations are NHWC bfloat16.  Every reduction here runs in a fixed
// order (per-split partial buffers and fixed trees, no floating-point
// atomics), so a training step is bitwise reproducible.
#include <cuda_bf16.h>

#include "kk_internal.h"
#include "kk_nn.h"

#include <algorithm>

namespace kk {
namespace nn {
namespace {

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// out[j] = sum_i part[i * stride + j]: 32 outputs per block, 8 groups of
// partials (group g sums i = g, g + 8, ... in order), then the 8 group sums
// in order -- a fixed summation tree
__global__ void __launch_bounds__(256)
    k_reduce_splits(const float *__restrict__ part, int n_part, size_t stride, size_t n_out,
                    float *__restrict__ out) {
  __shared__ float red[8][33];
  const int jl = threadIdx.x & 31, g = threadIdx.x >> 5;
  const size_t j = blockIdx.x * (size_t)32 + jl;
  float s = 0.f;
  if (j < n_out)
    for (int i = g; i < n_part; i += 8) s += part[(size_t)i * stride + j];
  red[g][jl] = s;
  __syncthreads();
  if (g == 0 && j < n_out) {
    float t = red[0][jl];
#pragma unroll
    for (int q = 1; q < 8; ++q) t += red[q][jl];
    out[j] = t;
  }
}

// W[co][kh][kw][ci] -> Wt[ci][2-kh][2-kw][co] (backward-data weights)
__global__ void k_flip_transpose(const __nv_bfloat16 *__restrict__ Wsrc, int Cout, int Cin,
                                 __nv_bfloat16 *__restrict__ Wdst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Cout * 9 * Cin) return;
  const int ci = i % Cin, tap = (i / Cin) % 9, co = i / (9 * Cin);
  const int kh = tap / 3, kw = tap % 3;
  Wdst[((size_t)ci * 9 + (2 - kh) * 3 + (2 - kw)) * Cout + co] = Wsrc[i];
}

// Eight bf16 channels as four bf16x2 <-> eight floats.
struct V8 {
  float f[8];
};
__device__ __forceinline__ V8 ld8(const __nv_bfloat16 *p) {
  const uint4 u = *reinterpret_cast<const uint4 *>(p);
  const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
  V8 r;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 t = __bfloat1622float2(h[q]);
    r.f[2 * q] = t.x;
    r.f[2 * q + 1] = t.y;
  }
  return r;
}
__device__ __forceinline__ void st8(__nv_bfloat16 *p, const V8 &v) {
  uint4 u;
  __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
  for (int q = 0; q < 4; ++q) h[q] = __floats2bfloat162_rn(v.f[2 * q], v.f[2 * q + 1]);
  *reinterpret_cast<uint4 *>(p) = u;
}

// dY *= (Y > 0) in place (ReLU backward, Y is the post-ReLU activation);
// 8 channels per thread
__global__ void k_relu_bwd(__nv_bfloat16 *__restrict__ dY, const __nv_bfloat16 *__restrict__ Y, size_t n8) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n8) return;
  V8 d = ld8(dY + 8 * i);
  const V8 y = ld8(Y + 8 * i);
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (!(y.f[q] > 0.f)) d.f[q] = 0.f;
  st8(dY + 8 * i, d);
}

// 2x2 average pooling (H, W even) and its adjoint; one thread per 8 channels
// of a coarse pixel
__global__ void k_pool2(const __nv_bfloat16 *__restrict__ X, int Nb, int H, int W, int C,
                        __nv_bfloat16 *__restrict__ Y) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const int Ho = H / 2, Wo = W / 2, C8 = C / 8;
  if (i >= (size_t)Nb * Ho * Wo * C8) return;
  const int c = (int)(i % C8) * 8;
  const size_t q = i / C8;
  const int wo = q % Wo, ho = (q / Wo) % Ho, n = q / ((size_t)Wo * Ho);
  const size_t b = (((size_t)n * H + 2 * ho) * W + 2 * wo) * C + c;
  const size_t row = (size_t)W * C;
  const V8 a0 = ld8(X + b), a1 = ld8(X + b + C), a2 = ld8(X + b + row), a3 = ld8(X + b + row + C);
  V8 o;
#pragma unroll
  for (int k = 0; k < 8; ++k) o.f[k] = 0.25f * ((a0.f[k] + a1.f[k]) + (a2.f[k] + a3.f[k]));
  st8(Y + q * C + c, o);
}
__global__ void k_pool2_bwd(const __nv_bfloat16 *__restrict__ dY, int Nb, int H, int W, int C,
                            __nv_bfloat16 *__restrict__ dX, int accumulate) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const int Ho = H / 2, Wo = W / 2, C8 = C / 8;
  if (i >= (size_t)Nb * Ho * Wo * C8) return;
  const int c = (int)(i % C8) * 8;
  const size_t q = i / C8;
  const int wo = q % Wo, ho = (q / Wo) % Ho, n = q / ((size_t)Wo * Ho);
  V8 g = ld8(dY + q * C + c);
#pragma unroll
  for (int k = 0; k < 8; ++k) g.f[k] *= 0.25f;
  const size_t b = (((size_t)n * H + 2 * ho) * W + 2 * wo) * C + c;
  const size_t off[4] = {0, (size_t)C, (size_t)W * C, (size_t)W * C + C};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    V8 o = g;
    if (accumulate) {
      const V8 d = ld8(dX + b + off[t]);
#pragma unroll
      for (int k = 0; k < 8; ++k) o.f[k] = d.f[k] + g.f[k];
    }
    st8(dX + b + off[t], o);
  }
}
// nearest 2x upsampling plus a skip tensor (nullable), and the adjoint of
// the upsampling; one thread per 8 channels of a coarse pixel
__global__ void k_up2_add(const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ skip, int Nb,
                          int H, int W, int C, __nv_bfloat16 *__restrict__ Y) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const int C8 = C / 8;
  if (i >= (size_t)Nb * H * W * C8) return;
  const int c = (int)(i % C8) * 8;
  const size_t q = i / C8;
  const int w = q % W, h = (q / W) % H, n = q / ((size_t)W * H);
  const V8 v = ld8(X + q * C + c);
  const size_t b = (((size_t)n * 2 * H + 2 * h) * 2 * W + 2 * w) * C + c;
  const size_t off[4] = {0, (size_t)C, (size_t)2 * W * C, (size_t)2 * W * C + C};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    V8 o = v;
    if (skip) {
      const V8 k8 = ld8(skip + b + off[t]);
#pragma unroll
      for (int k = 0; k < 8; ++k) o.f[k] = v.f[k] + k8.f[k];
    }
    st8(Y + b + off[t], o);
  }
}
__global__ void k_up2_bwd(const __nv_bfloat16 *__restrict__ dY, int Nb, int H, int W, int C,
                          __nv_bfloat16 *__restrict__ dX) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const int C8 = C / 8;
  if (i >= (size_t)Nb * H * W * C8) return;
  const int c = (int)(i % C8) * 8;
  const size_t q = i / C8;
  const int w = q % W, h = (q / W) % H, n = q / ((size_t)W * H);
  const size_t b = (((size_t)n * 2 * H + 2 * h) * 2 * W + 2 * w) * C + c;
  const size_t row = (size_t)2 * W * C;
  const V8 a0 = ld8(dY + b), a1 = ld8(dY + b + C), a2 = ld8(dY + b + row), a3 = ld8(dY + b + row + C);
  V8 o;
#pragma unroll
  for (int k = 0; k < 8; ++k) o.f[k] = (a0.f[k] + a1.f[k]) + (a2.f[k] + a3.f[k]);
  st8(dX + q * C + c, o);
}

// Complex images [Nb][HW] (float2) -> NHWC bf16 with C channels: (re, im)
// times scale[n], zeros in channels 2..C-1
__global__ void k_pack_iq(const float2 *__restrict__ img, const float *__restrict__ scale, int Nb, int HW,
                          int C, __nv_bfloat16 *__restrict__ X) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)Nb * HW) return;
  const int n = i / HW;
  const float2 v = img[i];
  const float s = scale ? scale[n] : 1.f;
  uint32_t *o = reinterpret_cast<uint32_t *>(X + i * C);
  o[0] = pack2(__float2bfloat16_rn(v.x * s), __float2bfloat16_rn(v.y * s));
  for (int c = 1; c < C / 2; ++c) o[c] = 0u;
}

constexpr int kRedThreads = 256;

// Residual output, squared-error partials per block and d loss / d head.
__global__ void __launch_bounds__(kRedThreads)
    k_residual_mse(const __nv_bfloat16 *__restrict__ Xin, int Cx, const float *__restrict__ head, int Ch,
                   const float2 *__restrict__ target, const float *__restrict__ tscale, int Nb, int HW,
                   float2 *__restrict__ out, __nv_bfloat16 *__restrict__ dhead, float *__restrict__ block_loss) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < (size_t)Nb * HW) {
    const int n = i / HW;
    const float2 o = make_float2(__bfloat162float(Xin[i * Cx]) + head[i * Ch],
                                 __bfloat162float(Xin[i * Cx + 1]) + head[i * Ch + 1]);
    if (out) out[i] = o;
    if (target) {
      const float s = tscale ? tscale[n] : 1.f;
      const float2 t = target[i];
      const float ex = o.x - t.x * s, ey = o.y - t.y * s;
      l = ex * ex + ey * ey;
      if (dhead) {
        const float k = 1.f / ((float)Nb * (float)HW);  // d/dhead of sum e^2 / (2 nb hw)
        uint32_t *d = reinterpret_cast<uint32_t *>(dhead + i * Ch);
        d[0] = pack2(__float2bfloat16_rn(k * ex), __float2bfloat16_rn(k * ey));
        for (int c = 1; c < Ch / 2; ++c) d[c] = 0u;
      }
    }
  }
  __shared__ float red[kRedThreads];
  red[threadIdx.x] = l;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && block_loss) block_loss[blockIdx.x] = red[0];
}

// one block: fixed strided partial sums, then a fixed tree
__global__ void __launch_bounds__(kRedThreads)
    k_sum_scalar(const float *__restrict__ part, int n, float k, float *__restrict__ out) {
  __shared__ float red[kRedThreads];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += kRedThreads) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * k;
}

// Adam (with decoupled-free L2 term wd * w added to the gradient) on FP32
// master weights; writes the BF16 working copy
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, size_t n, float lr,
                       float b1, float b2, float eps, float bc1, float bc2, float wd) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i] + wd * w[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  w[i] = wi;
  if (wb) wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// Direct DFT of complex [Nb][H][W] images along one axis:
// out[..k..] = sum_j in[..j..] exp(sign 2 pi i j k / L); axis 0 = rows (H),
// 1 = columns (W).  The twiddle comes from the exact integer phase j k mod L.
__global__ void k_dft_axis(const float2 *__restrict__ in, int Nb, int H, int W, int axis, int sign,
                           float2 *__restrict__ out) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)Nb * H * W) return;
  const int w = i % W, h = (i / W) % H, n = i / ((size_t)W * H);
  const int L = axis == 0 ? H : W;
  const int k = axis == 0 ? h : w;
  float2 acc = make_float2(0.f, 0.f);
  int m = 0;  // j k mod L
  for (int j = 0; j < L; ++j) {
    const float2 x = axis == 0 ? in[((size_t)n * H + j) * W + w] : in[((size_t)n * H + h) * W + j];
    float sn, cs;
    sincospif(2.f * (float)sign * (float)m / (float)L, &sn, &cs);
    acc.x = fmaf(x.x, cs, fmaf(-x.y, sn, acc.x));
    acc.y = fmaf(x.x, sn, fmaf(x.y, cs, acc.y));
    m += k;
    if (m >= L) m -= L;
  }
  out[i] = acc;
}

// Radix-2 Stockham FFT along one axis of complex [Nb][H][W] images, for a
// power-of-two length L (the row length W or the column length H).  A block
// takes 16 lines (16 consecutive columns for the column pass, so that each
// row of the tile is one 128-byte segment) and ping-pongs them through shared
// memory: at span Ns, element j and j + L/2 combine with the twiddle
// exp(sign 2 pi i (j mod Ns) / (2 Ns)) into positions (j / Ns) 2 Ns + j mod Ns
// and that + Ns, which leaves the result in natural order.
constexpr int kFftLines = 16;
__global__ void __launch_bounds__(256)
    k_fft_axis(const float2 *__restrict__ in, int Nb, int H, int W, int axis, int sign, int logL,
               float2 *__restrict__ out) {
  extern __shared__ float2 fbuf[];  // 2 x kFftLines x L
  const int L = 1 << logL;
  float2 *x = fbuf, *y = fbuf + kFftLines * L;
  const int lines_per_img = axis == 0 ? W : H;  // columns (axis 0) or rows (axis 1)
  const int line0 = blockIdx.x * kFftLines;     // over Nb * lines_per_img
  const int img = line0 / lines_per_img, l0 = line0 - img * lines_per_img;
  const size_t base = (size_t)img * H * W;
  // load: element e of line q at x[q * L + e]
  for (int t = threadIdx.x; t < kFftLines * L; t += blockDim.x) {
    int q, e;
    size_t g;
    if (axis == 0) {  // columns l0 + q, rows e: tile rows are contiguous
      q = t % kFftLines;
      e = t / kFftLines;
      g = base + (size_t)e * W + l0 + q;
    } else {          // rows l0 + q
      q = t / L;
      e = t % L;
      g = base + (size_t)(l0 + q) * W + e;
    }
    x[q * L + e] = in[g];
  }
  __syncthreads();
  for (int ls = 0; ls < logL; ++ls) {
    const int Ns = 1 << ls;
    for (int t = threadIdx.x; t < kFftLines * (L / 2); t += blockDim.x) {
      const int q = t / (L / 2), j = t % (L / 2);
      const int k = j & (Ns - 1);
      float sn, cs;
      sincospif((float)sign * (float)k / (float)Ns, &sn, &cs);  // angle = sign 2 pi k / (2 Ns)
      const float2 v0 = x[q * L + j], a = x[q * L + j + L / 2];
      const float2 v1 = make_float2(a.x * cs - a.y * sn, a.x * sn + a.y * cs);
      const int d = ((j >> ls) << (ls + 1)) + k;
      y[q * L + d] = make_float2(v0.x + v1.x, v0.y + v1.y);
      y[q * L + d + Ns] = make_float2(v0.x - v1.x, v0.y - v1.y);
    }
    __syncthreads();
    float2 *tmp = x;
    x = y;
    y = tmp;
  }
  for (int t = threadIdx.x; t < kFftLines * L; t += blockDim.x) {
    int q, e;
    size_t g;
    if (axis == 0) {
      q = t % kFftLines;
      e = t / kFftLines;
      g = base + (size_t)e * W + l0 + q;
    } else {
      q = t / L;
      e = t % L;
      g = base + (size_t)(l0 + q) * W + e;
    }
    out[g] = x[q * L + e];
  }
}

// one block: maxima of |Sc|, |Sf|, then G = Sc / Sf on the joint mask
__global__ void __launch_bounds__(kRedThreads)
    k_judge_filter(const float2 *__restrict__ Sc, const float2 *__restrict__ Sf, int hw, float rho,
                   float2 *__restrict__ G) {
  __shared__ float rc[kRedThreads], rf[kRedThreads];
  float mc = 0.f, mf = 0.f;
  for (int i = threadIdx.x; i < hw; i += kRedThreads) {
    mc = fmaxf(mc, hypotf(Sc[i].x, Sc[i].y));
    mf = fmaxf(mf, hypotf(Sf[i].x, Sf[i].y));
  }
  rc[threadIdx.x] = mc;
  rf[threadIdx.x] = mf;
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      rc[threadIdx.x] = fmaxf(rc[threadIdx.x], rc[threadIdx.x + h]);
      rf[threadIdx.x] = fmaxf(rf[threadIdx.x], rf[threadIdx.x + h]);
    }
    __syncthreads();
  }
  mc = rc[0];
  mf = rf[0];
  for (int i = threadIdx.x; i < hw; i += kRedThreads) {
    const float2 c = Sc[i], f = Sf[i];
    const float ac = hypotf(c.x, c.y), af = hypotf(f.x, f.y);
    float2 g = make_float2(0.f, 0.f);
    if (ac >= rho * mc && af >= rho * mf && af > 0.f) {
      const float d = f.x * f.x + f.y * f.y;  // c / f = c conj(f) / |f|^2
      g = make_float2((c.x * f.x + c.y * f.y) / d, (c.y * f.x - c.x * f.y) / d);
    }
    G[i] = g;
  }
}

// one block per image: stat[2n] = consistency residual, stat[2n+1] =
// out-of-band energy fraction of C
__global__ void __launch_bounds__(kRedThreads)
    k_judge_stat(const float2 *__restrict__ A, const float2 *__restrict__ C, const float2 *__restrict__ G,
                 int hw, float *__restrict__ stat) {
  __shared__ float r[5][kRedThreads];
  const size_t base = (size_t)blockIdx.x * hw;
  float aa = 0.f, cc = 0.f, re = 0.f, im = 0.f, ct = 0.f;
  for (int i = threadIdx.x; i < hw; i += kRedThreads) {
    const float2 g = G[i], c = C[base + i];
    const float c2 = c.x * c.x + c.y * c.y;
    ct += c2;
    if (g.x == 0.f && g.y == 0.f) continue;
    const float2 a0 = A[base + i];
    const float2 a = make_float2(g.x * a0.x - g.y * a0.y, g.x * a0.y + g.y * a0.x);
    aa += a.x * a.x + a.y * a.y;
    cc += c2;
    re += a.x * c.x + a.y * c.y;  // conj(a) c
    im += a.x * c.y - a.y * c.x;
  }
  r[0][threadIdx.x] = aa;
  r[1][threadIdx.x] = cc;
  r[2][threadIdx.x] = re;
  r[3][threadIdx.x] = im;
  r[4][threadIdx.x] = ct;
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int q = 0; q < 5; ++q) r[q][threadIdx.x] += r[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float den = r[0][0] * r[1][0];
    stat[2 * blockIdx.x] =
        den > 0.f ? fmaxf(0.f, 1.f - (r[2][0] * r[2][0] + r[3][0] * r[3][0]) / den) : 1.f;
    stat[2 * blockIdx.x + 1] = r[4][0] > 0.f ? fmaxf(0.f, (r[4][0] - r[1][0]) / r[4][0]) : 1.f;
  }
}

// one block per image: scale[n] = 1 / sqrt(mean |img|^2) (0 for a zero image)
__global__ void __launch_bounds__(kRedThreads)
    k_image_scale(const float2 *__restrict__ img, int hw, float *__restrict__ scale) {
  __shared__ float r[kRedThreads];
  const size_t base = (size_t)blockIdx.x * hw;
  float s = 0.f;
  for (int i = threadIdx.x; i < hw; i += kRedThreads) {
    const float2 v = img[base + i];
    s += v.x * v.x + v.y * v.y;
  }
  r[threadIdx.x] = s;
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) r[threadIdx.x] += r[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) scale[blockIdx.x] = r[0] > 0.f ? rsqrtf(r[0] / (float)hw) : 0.f;
}

inline unsigned blocks(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t reduce_splits(const float *part, int n_part, size_t stride, size_t n_out, float *out,
                          cudaStream_t s) {
  k_reduce_splits<<<(unsigned)((n_out + 31) / 32), 256, 0, s>>>(part, n_part, stride, n_out, out);
  return cudaGetLastError();
}

cudaError_t flip_transpose(const __nv_bfloat16 *w, int cout, int cin, __nv_bfloat16 *wt, cudaStream_t s) {
  k_flip_transpose<<<blocks((size_t)cout * 9 * cin), 256, 0, s>>>(w, cout, cin, wt);
  return cudaGetLastError();
}

cudaError_t relu_bwd(__nv_bfloat16 *dy, const __nv_bfloat16 *y, size_t n, cudaStream_t s) {
  k_relu_bwd<<<blocks(n / 8), 256, 0, s>>>(dy, y, n / 8);
  return cudaGetLastError();
}

cudaError_t pool2(const Tensor4 &x, __nv_bfloat16 *y, cudaStream_t s) {
  k_pool2<<<blocks(x.count() / 32), 256, 0, s>>>(x.p, x.n, x.h, x.w, x.c, y);
  return cudaGetLastError();
}

cudaError_t pool2_bwd(const __nv_bfloat16 *dy, const Tensor4 &dx, bool accumulate, cudaStream_t s) {
  k_pool2_bwd<<<blocks(dx.count() / 32), 256, 0, s>>>(dy, dx.n, dx.h, dx.w, dx.c, dx.p, accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t up2(const Tensor4 &x, __nv_bfloat16 *y, cudaStream_t s) { return up2_add(x, nullptr, y, s); }

cudaError_t up2_add(const Tensor4 &x, const __nv_bfloat16 *skip, __nv_bfloat16 *y, cudaStream_t s) {
  k_up2_add<<<blocks(x.count() / 8), 256, 0, s>>>(x.p, skip, x.n, x.h, x.w, x.c, y);
  return cudaGetLastError();
}

cudaError_t up2_bwd(const __nv_bfloat16 *dy, const Tensor4 &dx, cudaStream_t s) {
  k_up2_bwd<<<blocks(dx.count() / 8), 256, 0, s>>>(dy, dx.n, dx.h, dx.w, dx.c, dx.p);
  return cudaGetLastError();
}

cudaError_t pack_iq(const float2 *img, const float *scale, int nb, int hw, int c, __nv_bfloat16 *x,
                    cudaStream_t s) {
  k_pack_iq<<<blocks((size_t)nb * hw), 256, 0, s>>>(img, scale, nb, hw, c, x);
  return cudaGetLastError();
}

int residual_blocks(int nb, int hw) { return (int)blocks((size_t)nb * hw, kRedThreads); }

cudaError_t residual_mse(const __nv_bfloat16 *xin, int cx, const float *head, int ch, const float2 *target,
                         const float *tscale, int nb, int hw, float2 *out, __nv_bfloat16 *dhead,
                         float *block_loss, cudaStream_t s) {
  k_residual_mse<<<residual_blocks(nb, hw), kRedThreads, 0, s>>>(xin, cx, head, ch, target, tscale, nb, hw, out,
                                                                 dhead, block_loss);
  return cudaGetLastError();
}

cudaError_t sum_scalar(const float *part, int n, float k, float *loss, cudaStream_t s) {
  k_sum_scalar<<<1, kRedThreads, 0, s>>>(part, n, k, loss);
  return cudaGetLastError();
}

cudaError_t adam(float *w, const float *g, float *m, float *v, __nv_bfloat16 *wb, size_t n, float lr, float b1,
                 float b2, float eps, float bc1, float bc2, float wd, cudaStream_t s) {
  k_adam<<<blocks(n), 256, 0, s>>>(w, g, m, v, wb, n, lr, b1, b2, eps, bc1, bc2, wd);
  return cudaGetLastError();
}

cudaError_t to_bf16(const float *a, __nv_bfloat16 *b, size_t n, cudaStream_t s) {
  k_to_bf16<<<blocks(n), 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

namespace {
int log2_exact(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return (1 << l) == n ? l : -1;
}
}  // namespace

// Stockham FFT along an axis when its length is a power of two (and the
// lines split into blocks of 16), else the direct DFT
cudaError_t dft_axis(const float2 *in, int nb, int h, int w, int axis, int sign, float2 *out, cudaStream_t s) {
  const int L = axis == 0 ? h : w, lines = axis == 0 ? w : h;
  const int lg = log2_exact(L);
  if (lg >= 1 && L <= 512 && lines % kFftLines == 0) {
    const size_t smem = 2 * (size_t)kFftLines * L * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(k_fft_axis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fft_axis<<<(unsigned)((size_t)nb * lines / kFftLines), 256, smem, s>>>(in, nb, h, w, axis, sign, lg, out);
  } else {
    k_dft_axis<<<blocks((size_t)nb * h * w), 256, 0, s>>>(in, nb, h, w, axis, sign, out);
  }
  return cudaGetLastError();
}

cudaError_t dft2(const float2 *in, int nb, int h, int w, int sign, float2 *tmp, float2 *out, cudaStream_t s) {
  cudaError_t e = dft_axis(in, nb, h, w, 1, sign, tmp, s);
  if (e == cudaSuccess) e = dft_axis(tmp, nb, h, w, 0, sign, out, s);
  return e;
}

cudaError_t judge_filter(const float2 *Sc, const float2 *Sf, int hw, float rho, float2 *G, cudaStream_t s) {
  k_judge_filter<<<1, kRedThreads, 0, s>>>(Sc, Sf, hw, rho, G);
  return cudaGetLastError();
}

cudaError_t judge_stat(const float2 *A, const float2 *C, const float2 *G, int nb, int hw, float *stat,
                       cudaStream_t s) {
  k_judge_stat<<<nb, kRedThreads, 0, s>>>(A, C, G, hw, stat);
  return cudaGetLastError();
}

cudaError_t image_scale(const float2 *img, int nb, int hw, float *scale, cudaStream_t s) {
  k_image_scale<<<nb, kRedThreads, 0, s>>>(img, hw, scale);
  return cudaGetLastError();
}

}  // namespace nn
}  // namespace kk
