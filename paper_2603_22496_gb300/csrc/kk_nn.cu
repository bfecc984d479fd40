// kk_nn.cu -- kernels of the learned refiner: BF16 3x3 convolutions (forward,
// backward-data, backward-weight) as implicit GEMMs on the tensor cores with
// FP32 accumulation, and the small elementwise / pooling / loss / optimiser
// kernels around them.
//
// Activations are NHWC bfloat16 with the channel count a multiple of 16;
// weights are [Cout][3][3][Cin] bfloat16 (FP32 master copies live in the
// optimiser).  The convolution GEMM for a layer is
//     Y[p][co] = sum_{kh,kw,ci} X[p + (kh-1, kw-1)][ci] W[co][kh][kw][ci]
// with M = pixels, N = Cout, K = 9 Cin, zero padding at the image border.
// This file holds the warp-level form (mma.sync.m16n8k16, bf16 in, fp32
// accumulate), which every layer shape supports; it also serves the weight
// gradient, whose K dimension (pixels) is split over CTAs.
//
// Every reduction here runs in a fixed order (per-split partial buffers and
// fixed trees, no floating-point atomics), so a training step is bitwise
// reproducible.
#include <cuda_bf16.h>

#include "kk_internal.h"
#include "kk_nn.h"

#include <algorithm>

namespace kk {
namespace nn {
namespace {

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ---------------------------------------------------------------------------
// Forward convolution (also backward-data with flipped, transposed weights).
// CTA tile: 64 pixels x 64 output channels, 4 warps as 2 x 2, each warp
// 32 x 32 = 2 (m16) x 4 (n8) mma tiles; K chunks of 16 (one mma K).
// ---------------------------------------------------------------------------
constexpr int kTM = 64, kTN = 64, kTK = 16;

__global__ void __launch_bounds__(128)
    k_conv3x3(const __nv_bfloat16 *__restrict__ X, int Nb, int H, int W, int Cin,
              const __nv_bfloat16 *__restrict__ Wt, int Cout, const float *__restrict__ bias,
              int relu, __nv_bfloat16 *__restrict__ Y, float *__restrict__ Yf) {
  __shared__ __align__(16) __nv_bfloat16 As[kTM][kTK + 8];  // pixels x k (padded rows)
  __shared__ __align__(16) __nv_bfloat16 Bs[kTN][kTK + 8];  // cout x k
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 1, wn = warp & 1;
  const int P = Nb * H * W;
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * kTN;
  const int K = 9 * Cin;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

  // loader mapping: 128 threads; A: 64 rows x 16 k = 64 x 2 chunks of 8 bf16
  const int lr = tid >> 1, lc = (tid & 1) * 8;
  const int pm = m0 + lr;
  int pn = 0, ph = 0, pw = 0;
  if (pm < P) {
    pn = pm / (H * W);
    const int r = pm - pn * H * W;
    ph = r / W;
    pw = r - ph * W;
  }
  for (int k0 = 0; k0 < K; k0 += kTK) {
    const int tap = k0 / Cin, ci0 = k0 - tap * Cin;
    const int kh = tap / 3, kw = tap - kh * 3;
    // A: pixel lr, channels ci0 + lc .. +7 at tap (kh, kw)
    {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      const int hh = ph + kh - 1, ww = pw + kw - 1;
      if (pm < P && hh >= 0 && hh < H && ww >= 0 && ww < W)
        v = *reinterpret_cast<const uint4 *>(X + (((size_t)pn * H + hh) * W + ww) * Cin + ci0 + lc);
      *reinterpret_cast<uint4 *>(&As[lr][lc]) = v;
    }
    // B: output channel lr, k0 + lc .. +7
    {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      const int co = n0 + lr;
      if (co < Cout) v = *reinterpret_cast<const uint4 *>(Wt + (size_t)co * K + k0 + lc);
      *reinterpret_cast<uint4 *>(&Bs[lr][lc]) = v;
    }
    __syncthreads();
    const int g = lane >> 2, t2 = (lane & 3) * 2;
    uint32_t af[2][4], bf[4][2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int r = wm * 32 + a * 16 + g;
      af[a][0] = *reinterpret_cast<const uint32_t *>(&As[r][t2]);
      af[a][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][t2]);
      af[a][2] = *reinterpret_cast<const uint32_t *>(&As[r][t2 + 8]);
      af[a][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][t2 + 8]);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = wn * 32 + b * 8 + g;
      bf[b][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][t2]);
      bf[b][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][t2 + 8]);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) mma_bf16_16816(acc[a][b], af[a], bf[b]);
    __syncthreads();
  }
  // epilogue: rows (pixels) g, g+8; cols t2, t2+1
  const int g = lane >> 2, t2 = (lane & 3) * 2;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int hrow = 0; hrow < 2; ++hrow) {
      const int p = m0 + wm * 32 + a * 16 + g + hrow * 8;
      if (p >= P) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int co = n0 + wn * 32 + b * 8 + t2;
        if (co >= Cout) continue;
        float v0 = acc[a][b][hrow * 2], v1 = acc[a][b][hrow * 2 + 1];
        if (bias) {
          v0 += bias[co];
          if (co + 1 < Cout) v1 += bias[co + 1];
        }
        if (relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (Y) {
          Y[(size_t)p * Cout + co] = __float2bfloat16_rn(v0);
          if (co + 1 < Cout) Y[(size_t)p * Cout + co + 1] = __float2bfloat16_rn(v1);
        }
        if (Yf) {
          Yf[(size_t)p * Cout + co] = v0;
          if (co + 1 < Cout) Yf[(size_t)p * Cout + co + 1] = v1;
        }
      }
    }
}

// Weight and bias gradients: part[split][co][tap][ci] = sum_p dY[p][co] X[p + tap][ci]
// over the split's pixel range, and part[split][Cout*9*Cin + co] = sum_p dY[p][co].
// GEMM M = Cout, N = 9 Cin, K = pixels; CTA tile 64 x 64, pixel chunks of 16.
__global__ void __launch_bounds__(128)
    k_conv3x3_wgrad(const __nv_bfloat16 *__restrict__ X, int Nb, int H, int W, int Cin,
                    const __nv_bfloat16 *__restrict__ dY, int Cout, int pix_per_split,
                    float *__restrict__ part) {
  __shared__ __align__(16) __nv_bfloat16 As[kTM][kTK + 8];  // cout x pixels (dY^T)
  __shared__ __align__(16) __nv_bfloat16 Bs[kTN][kTK + 8];  // (tap, ci) x pixels (patches^T)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 1, wn = warp & 1;
  const int P = Nb * H * W;
  const int Ncol = 9 * Cin;
  const size_t stride = (size_t)Cout * Ncol + Cout;
  const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * kTN;
  const int pb = blockIdx.z * pix_per_split, pe = min(P, pb + pix_per_split);
  const bool do_bias = blockIdx.y == 0;
  float bsum = 0.f;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const int px = tid >> 3, c8 = (tid & 7) * 8;  // loaders: 16 pixels x 8 chunks of 8
  for (int k0 = pb; k0 < pe; k0 += kTK) {
    const int p = k0 + px;
    {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (p < pe && m0 + c8 < Cout) v = *reinterpret_cast<const uint4 *>(dY + (size_t)p * Cout + m0 + c8);
      const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
      for (int q = 0; q < 8; ++q) As[c8 + q][px] = e[q];
    }
    {
      const int col = n0 + c8;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (p < pe && col < Ncol) {
        const int tap = col / Cin, ci = col - tap * Cin;
        const int kh = tap / 3, kw = tap - kh * 3;
        const int n = p / (H * W), r = p - n * H * W;
        const int hh = r / W + kh - 1, ww = r % W + kw - 1;
        if (hh >= 0 && hh < H && ww >= 0 && ww < W)
          v = *reinterpret_cast<const uint4 *>(X + (((size_t)n * H + hh) * W + ww) * Cin + ci);
      }
      const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
      for (int q = 0; q < 8; ++q) Bs[c8 + q][px] = e[q];
    }
    __syncthreads();
    if (do_bias && tid < kTM) {
#pragma unroll
      for (int q = 0; q < kTK; ++q) bsum += __bfloat162float(As[tid][q]);
    }
    const int g = lane >> 2, t2 = (lane & 3) * 2;
    uint32_t af[2][4], bf[4][2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int r = wm * 32 + a * 16 + g;
      af[a][0] = *reinterpret_cast<const uint32_t *>(&As[r][t2]);
      af[a][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][t2]);
      af[a][2] = *reinterpret_cast<const uint32_t *>(&As[r][t2 + 8]);
      af[a][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][t2 + 8]);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = wn * 32 + b * 8 + g;
      bf[b][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][t2]);
      bf[b][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][t2 + 8]);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) mma_bf16_16816(acc[a][b], af[a], bf[b]);
    __syncthreads();
  }
  float *dst = part + (size_t)blockIdx.z * stride;
  const int g = lane >> 2, t2 = (lane & 3) * 2;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int hrow = 0; hrow < 2; ++hrow) {
      const int co = m0 + wm * 32 + a * 16 + g + hrow * 8;
      if (co >= Cout) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int col = n0 + wn * 32 + b * 8 + t2;  // Ncol is a multiple of 16: col + 1 < Ncol too
        if (col < Ncol)
          *reinterpret_cast<float2 *>(dst + (size_t)co * Ncol + col) =
              make_float2(acc[a][b][hrow * 2], acc[a][b][hrow * 2 + 1]);
      }
    }
  if (do_bias && tid < kTM && m0 + tid < Cout) dst[(size_t)Cout * Ncol + m0 + tid] = bsum;
}

__global__ void k_reduce_splits(const float *__restrict__ part, int n_part, size_t stride, size_t n_out,
                                float *__restrict__ out) {
  const size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (j >= n_out) return;
  float s = 0.f;
  for (int i = 0; i < n_part; ++i) s += part[(size_t)i * stride + j];
  out[j] = s;
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

// dY *= (Y > 0)  in place (ReLU backward, Y is the post-ReLU activation)
__global__ void k_relu_bwd(__nv_bfloat16 *__restrict__ dY, const __nv_bfloat16 *__restrict__ Y, size_t n) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n && !(__bfloat162float(Y[i]) > 0.f)) dY[i] = __float2bfloat16_rn(0.f);
}

// 2x2 average pooling (H, W even) and its adjoint
__global__ void k_pool2(const __nv_bfloat16 *__restrict__ X, int Nb, int H, int W, int C,
                        __nv_bfloat16 *__restrict__ Y) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const int Ho = H / 2, Wo = W / 2;
  if (i >= (size_t)Nb * Ho * Wo * C) return;
  const int c = i % C;
  const size_t q = i / C;
  const int wo = q % Wo, ho = (q / Wo) % Ho, n = q / ((size_t)Wo * Ho);
  const size_t b = (((size_t)n * H + 2 * ho) * W + 2 * wo) * C + c;
  const size_t row = (size_t)W * C;
  const float s = (__bfloat162float(X[b]) + __bfloat162float(X[b + C])) +
                  (__bfloat162float(X[b + row]) + __bfloat162float(X[b + row + C]));
  Y[i] = __float2bfloat16_rn(0.25f * s);
}
__global__ void k_pool2_bwd(const __nv_bfloat16 *__restrict__ dY, int Nb, int H, int W, int C,
                            __nv_bfloat16 *__restrict__ dX, int accumulate) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)Nb * H * W * C) return;
  const int c = i % C;
  const size_t q = i / C;
  const int w = q % W, h = (q / W) % H, n = q / ((size_t)W * H);
  const float g = 0.25f * __bfloat162float(dY[(((size_t)n * (H / 2) + h / 2) * (W / 2) + w / 2) * C + c]);
  dX[i] = __float2bfloat16_rn(accumulate ? __bfloat162float(dX[i]) + g : g);
}
// nearest 2x upsampling plus a skip tensor, and the adjoint of the upsampling
__global__ void k_up2_add(const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ skip, int Nb,
                          int H, int W, int C, __nv_bfloat16 *__restrict__ Y) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const int Ho = 2 * H, Wo = 2 * W;
  if (i >= (size_t)Nb * Ho * Wo * C) return;
  const int c = i % C;
  const size_t q = i / C;
  const int wo = q % Wo, ho = (q / Wo) % Ho, n = q / ((size_t)Wo * Ho);
  const __nv_bfloat16 v = X[(((size_t)n * H + ho / 2) * W + wo / 2) * C + c];
  Y[i] = skip ? __float2bfloat16_rn(__bfloat162float(v) + __bfloat162float(skip[i])) : v;
}
__global__ void k_up2_bwd(const __nv_bfloat16 *__restrict__ dY, int Nb, int H, int W, int C,
                          __nv_bfloat16 *__restrict__ dX) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)Nb * H * W * C) return;
  const int c = i % C;
  const size_t q = i / C;
  const int w = q % W, h = (q / W) % H, n = q / ((size_t)W * H);
  const size_t b = (((size_t)n * 2 * H + 2 * h) * 2 * W + 2 * w) * C + c;
  const size_t row = (size_t)2 * W * C;
  dX[i] = __float2bfloat16_rn((__bfloat162float(dY[b]) + __bfloat162float(dY[b + C])) +
                              (__bfloat162float(dY[b + row]) + __bfloat162float(dY[b + row + C])));
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

cudaError_t conv3x3(const Tensor4 &x, const __nv_bfloat16 *w, int cout, const float *bias, bool relu,
                    __nv_bfloat16 *y, float *yf, cudaStream_t s) {
  const int P = x.n * x.h * x.w;
  dim3 grid((P + kTM - 1) / kTM, (cout + kTN - 1) / kTN);
  k_conv3x3<<<grid, 128, 0, s>>>(x.p, x.n, x.h, x.w, x.c, w, cout, bias, relu ? 1 : 0, y, yf);
  return cudaGetLastError();
}

// Pixel splits of the weight gradient: about 4 x 152 CTAs in total (a fixed
// count, so that results do not depend on the device), at least 256 pixels
// per split.
int wgrad_splits(const Tensor4 &x, int cout) {
  const int P = x.n * x.h * x.w;
  const int tiles = ((cout + kTM - 1) / kTM) * ((9 * x.c + kTN - 1) / kTN);
  int want = std::max(1, (608 + tiles - 1) / tiles);
  want = std::min(want, std::max(1, P / 256));
  const int per = ((P + want - 1) / want + kTK - 1) / kTK * kTK;
  return (P + per - 1) / per;
}

size_t wgrad_part_floats(const Tensor4 &x, int cout) {
  return (size_t)wgrad_splits(x, cout) * ((size_t)cout * 9 * x.c + cout);
}

cudaError_t conv3x3_wgrad(const Tensor4 &x, const __nv_bfloat16 *dy, int cout, float *part, int *n_split,
                          cudaStream_t s) {
  const int P = x.n * x.h * x.w;
  const int splits = wgrad_splits(x, cout);
  const int per = ((P + splits - 1) / splits + kTK - 1) / kTK * kTK;
  dim3 grid((cout + kTM - 1) / kTM, (9 * x.c + kTN - 1) / kTN, splits);
  k_conv3x3_wgrad<<<grid, 128, 0, s>>>(x.p, x.n, x.h, x.w, x.c, dy, cout, per, part);
  *n_split = splits;
  return cudaGetLastError();
}

cudaError_t reduce_splits(const float *part, int n_part, size_t stride, size_t n_out, float *out,
                          cudaStream_t s) {
  k_reduce_splits<<<blocks(n_out), 256, 0, s>>>(part, n_part, stride, n_out, out);
  return cudaGetLastError();
}

cudaError_t flip_transpose(const __nv_bfloat16 *w, int cout, int cin, __nv_bfloat16 *wt, cudaStream_t s) {
  k_flip_transpose<<<blocks((size_t)cout * 9 * cin), 256, 0, s>>>(w, cout, cin, wt);
  return cudaGetLastError();
}

cudaError_t relu_bwd(__nv_bfloat16 *dy, const __nv_bfloat16 *y, size_t n, cudaStream_t s) {
  k_relu_bwd<<<blocks(n), 256, 0, s>>>(dy, y, n);
  return cudaGetLastError();
}

cudaError_t pool2(const Tensor4 &x, __nv_bfloat16 *y, cudaStream_t s) {
  k_pool2<<<blocks(x.count() / 4), 256, 0, s>>>(x.p, x.n, x.h, x.w, x.c, y);
  return cudaGetLastError();
}

cudaError_t pool2_bwd(const __nv_bfloat16 *dy, const Tensor4 &dx, bool accumulate, cudaStream_t s) {
  k_pool2_bwd<<<blocks(dx.count()), 256, 0, s>>>(dy, dx.n, dx.h, dx.w, dx.c, dx.p, accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t up2(const Tensor4 &x, __nv_bfloat16 *y, cudaStream_t s) { return up2_add(x, nullptr, y, s); }

cudaError_t up2_add(const Tensor4 &x, const __nv_bfloat16 *skip, __nv_bfloat16 *y, cudaStream_t s) {
  k_up2_add<<<blocks(x.count() * 4), 256, 0, s>>>(x.p, skip, x.n, x.h, x.w, x.c, y);
  return cudaGetLastError();
}

cudaError_t up2_bwd(const __nv_bfloat16 *dy, const Tensor4 &dx, cudaStream_t s) {
  k_up2_bwd<<<blocks(dx.count()), 256, 0, s>>>(dy, dx.n, dx.h, dx.w, dx.c, dx.p);
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

cudaError_t dft2(const float2 *in, int nb, int h, int w, int sign, float2 *tmp, float2 *out, cudaStream_t s) {
  const size_t n = (size_t)nb * h * w;
  k_dft_axis<<<blocks(n), 256, 0, s>>>(in, nb, h, w, 1, sign, tmp);
  k_dft_axis<<<blocks(n), 256, 0, s>>>(tmp, nb, h, w, 0, sign, out);
  return cudaGetLastError();
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
