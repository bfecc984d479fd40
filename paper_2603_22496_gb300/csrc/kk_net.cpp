// kk_net.cpp -- the learned refiner: network object, forward, backward,
// Adam, checkpoints, the fallback judge and the layer-level calls of
// include/kknet.h.  All arithmetic runs in the kernels of kk_nn.cu; this
// file only sequences launches and owns the buffers.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/kknet.h"
#include "kk_internal.h"
#include "kk_nn.h"

using kk::nn::Tensor4;

namespace {

constexpr int kInChannels = 16;   // (re, im) + 14 zero channels
constexpr int kHeadChannels = 16; // head outputs (re, im) + 14 unused
constexpr int kLevels = 5;
constexpr int kLayers = 13;

struct Layer {
  int cin, cout, level;
  bool relu;
  size_t w_off, b_off;  // in the flat parameter vector
};

// Bump allocator over one device allocation (256-byte aligned pieces).
struct Arena {
  size_t size = 0;
  char *base = nullptr;
  template <class T>
  T *take(size_t count) {
    const size_t off = size;
    size = (size + count * sizeof(T) + 255) & ~(size_t)255;
    return reinterpret_cast<T *>(base + off);
  }
};

uint64_t splitmix64(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// standard normal by Box-Muller on two 53-bit uniforms
double normal(uint64_t &s) {
  const double u1 = ((double)(splitmix64(s) >> 11) + 1.0) * 0x1p-53;
  const double u2 = (double)(splitmix64(s) >> 11) * 0x1p-53;
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

struct kk_net {
  int device = 0;
  int B = 0, H = 0, W = 0, C = 0;
  uint64_t seed = 0;
  int64_t step = 0;
  Layer layer[kLayers];
  size_t n_params = 0;
  void *block = nullptr;
  // parameters and optimiser state (flat, layer order)
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *wb = nullptr;  // BF16 working copy of w
  __nv_bfloat16 *wt = nullptr;  // flipped / transposed BF16 weights (backward-data)
  float *part = nullptr;        // weight-gradient split partials
  float *loss_part = nullptr;
  int *status = nullptr;        // device status word of the tensor-core kernels
  // activations (for max_batch images)
  __nv_bfloat16 *x = nullptr;
  __nv_bfloat16 *a[12] = {};
  __nv_bfloat16 *p[4] = {};
  __nv_bfloat16 *u[4] = {};
  float *head = nullptr;
  __nv_bfloat16 *dhead = nullptr;
  __nv_bfloat16 *ga[kLevels] = {}, *gb[kLevels] = {};
  // judge
  float2 *G = nullptr, *dft_tmp = nullptr, *dft_A = nullptr, *dft_C = nullptr;
  bool have_filter = false;

  int hl(int l) const { return H >> l; }
  int wl(int l) const { return W >> l; }
  Tensor4 t(__nv_bfloat16 *ptr, int nb, int level, int c) const { return Tensor4{ptr, nb, hl(level), wl(level), c}; }
};

namespace {

using kk::cuda_fail;
using kk::set_error;

#define KK_TRY(expr, what)                        \
  do {                                            \
    const cudaError_t e_ = (expr);                \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)
#define KK_STEP(call) \
  if ((st = (call)) != KK_OK) return st

void define_layers(kk_net &n) {
  const int C = n.C;
  const int spec[kLayers][4] = {
      {kInChannels, C, 0, 1}, {C, C, 0, 1},           // level 0
      {C, 2 * C, 1, 1},       {2 * C, 2 * C, 1, 1},   // level 1
      {2 * C, 4 * C, 2, 1},   {4 * C, 4 * C, 2, 1},   // level 2
      {4 * C, 8 * C, 3, 1},                           // level 3
      {8 * C, 8 * C, 4, 1},                           // level 4
      {8 * C, 4 * C, 3, 1},   {4 * C, 2 * C, 2, 1},   // decoder
      {2 * C, C, 1, 1},       {C, C, 0, 1},
      {C, kHeadChannels, 0, 0}};                      // head
  size_t off = 0;
  for (int i = 0; i < kLayers; ++i) {
    Layer &L = n.layer[i];
    L.cin = spec[i][0];
    L.cout = spec[i][1];
    L.level = spec[i][2];
    L.relu = spec[i][3] != 0;
    L.w_off = off;
    off += (size_t)L.cout * 9 * L.cin;
    L.b_off = off;
    off += (size_t)L.cout;
  }
  n.n_params = off;
}

// He-normal weights (fan-in 9 x the channels that carry data), zero biases;
// the head starts near zero (out ~ in) with its unused outputs at zero.
std::vector<float> init_params(const kk_net &n) {
  std::vector<float> h(n.n_params, 0.f);
  uint64_t s = n.seed;
  for (int i = 0; i < kLayers; ++i) {
    const Layer &L = n.layer[i];
    const int fan_cin = (i == 0) ? 2 : L.cin;
    double sd = std::sqrt(2.0 / (9.0 * fan_cin));
    if (i == kLayers - 1) sd = 0.1 * std::sqrt(1.0 / (9.0 * L.cin));
    for (int co = 0; co < L.cout; ++co)
      for (int k = 0; k < 9 * L.cin; ++k) {
        const double r = normal(s);
        const bool used = (i != kLayers - 1 || co < 2) && (i != 0 || (k % L.cin) < 2);
        h[L.w_off + (size_t)co * 9 * L.cin + k] = used ? (float)(sd * r) : 0.f;
      }
  }
  return h;
}

size_t max_part_floats(const kk_net &n) {
  size_t mx = 0;
  for (int i = 0; i < kLayers; ++i) {
    const Layer &L = n.layer[i];
    Tensor4 x{nullptr, n.B, n.hl(L.level), n.wl(L.level), L.cin};
    mx = std::max(mx, kk::nn::wgrad_part_floats(x, L.cout));
  }
  return mx;
}

// two passes: size, then carve
void carve(kk_net &n, Arena &A) {
  const size_t np = n.n_params;
  const int C = n.C, B = n.B;
  auto px = [&](int l) { return (size_t)B * n.hl(l) * n.wl(l); };
  n.w = A.take<float>(np);
  n.g = A.take<float>(np);
  n.m = A.take<float>(np);
  n.v = A.take<float>(np);
  n.wb = A.take<__nv_bfloat16>(np);
  n.wt = A.take<__nv_bfloat16>(np);
  n.part = A.take<float>(max_part_floats(n));
  n.loss_part = A.take<float>((size_t)kk::nn::residual_blocks(B, n.H * n.W));
  n.status = A.take<int>(1);
  n.x = A.take<__nv_bfloat16>(px(0) * kInChannels);
  for (int i = 0; i < 12; ++i) n.a[i] = A.take<__nv_bfloat16>(px(n.layer[i].level) * n.layer[i].cout);
  const int pc[4] = {C, 2 * C, 4 * C, 8 * C};  // pooled p_l lives at level l + 1
  for (int l = 0; l < 4; ++l) n.p[l] = A.take<__nv_bfloat16>(px(l + 1) * pc[l]);
  const int uc[4] = {C, 2 * C, 4 * C, 8 * C};  // u_l = up + skip at level l
  for (int l = 0; l < 4; ++l) n.u[l] = A.take<__nv_bfloat16>(px(l) * uc[l]);
  n.head = A.take<float>(px(0) * kHeadChannels);
  n.dhead = A.take<__nv_bfloat16>(px(0) * kHeadChannels);
  const int gc[kLevels] = {C, 2 * C, 4 * C, 8 * C, 8 * C};
  for (int l = 0; l < kLevels; ++l) {
    n.ga[l] = A.take<__nv_bfloat16>(px(l) * gc[l]);
    n.gb[l] = A.take<__nv_bfloat16>(px(l) * gc[l]);
  }
}

kk_status check_net(const kk_net *n, int nb) {
  if (!n) { set_error("null net"); return KK_ERR_INVALID_ARG; }
  if (nb < 1 || nb > n->B) { set_error("nb out of range (1..max_batch)"); return KK_ERR_INVALID_ARG; }
  return KK_OK;
}

kk_status conv(const kk_net &n, int i, const Tensor4 &x, __nv_bfloat16 *y, float *yf, cudaStream_t s) {
  const Layer &L = n.layer[i];
  KK_TRY(kk::nn::conv3x3_tc(x, n.wb + L.w_off, L.cout, n.w + L.b_off, L.relu, y, yf, n.status, s), "conv launch");
  return KK_OK;
}

// weight and bias gradient of layer i into n.g (W then b, contiguous)
kk_status wgrad(const kk_net &n, int i, const Tensor4 &x, const __nv_bfloat16 *dy, cudaStream_t s) {
  const Layer &L = n.layer[i];
  int splits = 0, nb = 0;
  KK_TRY(kk::nn::conv3x3_wgrad(x, dy, L.cout, n.part, &splits, &nb, n.status, s), "wgrad launch");
  const size_t nw = (size_t)L.cout * 9 * L.cin;
  KK_TRY(kk::nn::reduce_splits(n.part, splits, nw, nw, n.g + L.w_off, s), "wgrad reduce");
  KK_TRY(kk::nn::reduce_splits(n.part + (size_t)splits * nw, nb, L.cout, L.cout, n.g + L.b_off, s), "bias reduce");
  return KK_OK;
}

// gradient w.r.t. layer i's input: conv of dy with the flipped weights
kk_status dgrad(const kk_net &n, int i, const Tensor4 &dy, __nv_bfloat16 *dx, cudaStream_t s) {
  const Layer &L = n.layer[i];
  KK_TRY(kk::nn::conv3x3_tc(dy, n.wt + L.w_off, L.cin, nullptr, false, dx, nullptr, n.status, s), "dgrad launch");
  return KK_OK;
}

kk_status forward(kk_net &n, int nb, const void *in, const float *in_scale, cudaStream_t s) {
  namespace K = kk::nn;
  const int C = n.C;
  const int hw = n.H * n.W;
  KK_TRY(K::pack_iq((const float2 *)in, in_scale, nb, hw, kInChannels, n.x, s), "pack");
  kk_status st;
  KK_STEP(conv(n, 0, n.t(n.x, nb, 0, kInChannels), n.a[0], nullptr, s));
  KK_STEP(conv(n, 1, n.t(n.a[0], nb, 0, C), n.a[1], nullptr, s));
  KK_TRY(K::pool2(n.t(n.a[1], nb, 0, C), n.p[0], s), "pool");
  KK_STEP(conv(n, 2, n.t(n.p[0], nb, 1, C), n.a[2], nullptr, s));
  KK_STEP(conv(n, 3, n.t(n.a[2], nb, 1, 2 * C), n.a[3], nullptr, s));
  KK_TRY(K::pool2(n.t(n.a[3], nb, 1, 2 * C), n.p[1], s), "pool");
  KK_STEP(conv(n, 4, n.t(n.p[1], nb, 2, 2 * C), n.a[4], nullptr, s));
  KK_STEP(conv(n, 5, n.t(n.a[4], nb, 2, 4 * C), n.a[5], nullptr, s));
  KK_TRY(K::pool2(n.t(n.a[5], nb, 2, 4 * C), n.p[2], s), "pool");
  KK_STEP(conv(n, 6, n.t(n.p[2], nb, 3, 4 * C), n.a[6], nullptr, s));
  KK_TRY(K::pool2(n.t(n.a[6], nb, 3, 8 * C), n.p[3], s), "pool");
  KK_STEP(conv(n, 7, n.t(n.p[3], nb, 4, 8 * C), n.a[7], nullptr, s));
  KK_TRY(K::up2_add(n.t(n.a[7], nb, 4, 8 * C), n.a[6], n.u[3], s), "up");
  KK_STEP(conv(n, 8, n.t(n.u[3], nb, 3, 8 * C), n.a[8], nullptr, s));
  KK_TRY(K::up2_add(n.t(n.a[8], nb, 3, 4 * C), n.a[5], n.u[2], s), "up");
  KK_STEP(conv(n, 9, n.t(n.u[2], nb, 2, 4 * C), n.a[9], nullptr, s));
  KK_TRY(K::up2_add(n.t(n.a[9], nb, 2, 2 * C), n.a[3], n.u[1], s), "up");
  KK_STEP(conv(n, 10, n.t(n.u[1], nb, 1, 2 * C), n.a[10], nullptr, s));
  KK_TRY(K::up2_add(n.t(n.a[10], nb, 1, C), n.a[1], n.u[0], s), "up");
  KK_STEP(conv(n, 11, n.t(n.u[0], nb, 0, C), n.a[11], nullptr, s));
  KK_STEP(conv(n, 12, n.t(n.a[11], nb, 0, C), nullptr, n.head, s));
  return KK_OK;
}

kk_status backward(kk_net &n, int nb, cudaStream_t s) {
  namespace K = kk::nn;
  const int C = n.C;
  kk_status st;
  for (int i = 0; i < kLayers; ++i) {
    const Layer &L = n.layer[i];
    KK_TRY(K::flip_transpose(n.wb + L.w_off, L.cout, L.cin, n.wt + L.w_off, s), "flip");
  }
  auto relu_b = [&](__nv_bfloat16 *d, const __nv_bfloat16 *y, int level, int c) {
    return K::relu_bwd(d, y, (size_t)nb * n.hl(level) * n.wl(level) * c, s);
  };
  // head and d0 (level 0)
  KK_STEP(wgrad(n, 12, n.t(n.a[11], nb, 0, C), n.dhead, s));
  KK_STEP(dgrad(n, 12, n.t(n.dhead, nb, 0, kHeadChannels), n.ga[0], s));
  KK_TRY(relu_b(n.ga[0], n.a[11], 0, C), "relu");
  KK_STEP(wgrad(n, 11, n.t(n.u[0], nb, 0, C), n.ga[0], s));
  KK_STEP(dgrad(n, 11, n.t(n.ga[0], nb, 0, C), n.gb[0], s));           // d u0 = d a1 (skip part)
  KK_TRY(K::up2_bwd(n.gb[0], n.t(n.ga[1], nb, 1, C), s), "up bwd");  // d a10
  KK_TRY(relu_b(n.ga[1], n.a[10], 1, C), "relu");
  KK_STEP(wgrad(n, 10, n.t(n.u[1], nb, 1, 2 * C), n.ga[1], s));
  KK_STEP(dgrad(n, 10, n.t(n.ga[1], nb, 1, C), n.gb[1], s));           // d u1 = d a3 (skip part)
  KK_TRY(K::up2_bwd(n.gb[1], n.t(n.ga[2], nb, 2, 2 * C), s), "up bwd");  // d a9
  KK_TRY(relu_b(n.ga[2], n.a[9], 2, 2 * C), "relu");
  KK_STEP(wgrad(n, 9, n.t(n.u[2], nb, 2, 4 * C), n.ga[2], s));
  KK_STEP(dgrad(n, 9, n.t(n.ga[2], nb, 2, 2 * C), n.gb[2], s));        // d u2 = d a5 (skip part)
  KK_TRY(K::up2_bwd(n.gb[2], n.t(n.ga[3], nb, 3, 4 * C), s), "up bwd");  // d a8
  KK_TRY(relu_b(n.ga[3], n.a[8], 3, 4 * C), "relu");
  KK_STEP(wgrad(n, 8, n.t(n.u[3], nb, 3, 8 * C), n.ga[3], s));
  KK_STEP(dgrad(n, 8, n.t(n.ga[3], nb, 3, 4 * C), n.gb[3], s));        // d u3 = d a6 (skip part)
  KK_TRY(K::up2_bwd(n.gb[3], n.t(n.ga[4], nb, 4, 8 * C), s), "up bwd");  // d a7
  KK_TRY(relu_b(n.ga[4], n.a[7], 4, 8 * C), "relu");
  // encoder, deepest first
  KK_STEP(wgrad(n, 7, n.t(n.p[3], nb, 4, 8 * C), n.ga[4], s));
  KK_STEP(dgrad(n, 7, n.t(n.ga[4], nb, 4, 8 * C), n.gb[4], s));        // d p3
  KK_TRY(K::pool2_bwd(n.gb[4], n.t(n.gb[3], nb, 3, 8 * C), true, s), "pool bwd");  // d a6 total
  KK_TRY(relu_b(n.gb[3], n.a[6], 3, 8 * C), "relu");
  KK_STEP(wgrad(n, 6, n.t(n.p[2], nb, 3, 4 * C), n.gb[3], s));
  KK_STEP(dgrad(n, 6, n.t(n.gb[3], nb, 3, 8 * C), n.ga[3], s));        // d p2
  KK_TRY(K::pool2_bwd(n.ga[3], n.t(n.gb[2], nb, 2, 4 * C), true, s), "pool bwd");  // d a5 total
  KK_TRY(relu_b(n.gb[2], n.a[5], 2, 4 * C), "relu");
  KK_STEP(wgrad(n, 5, n.t(n.a[4], nb, 2, 4 * C), n.gb[2], s));
  KK_STEP(dgrad(n, 5, n.t(n.gb[2], nb, 2, 4 * C), n.ga[2], s));        // d a4
  KK_TRY(relu_b(n.ga[2], n.a[4], 2, 4 * C), "relu");
  KK_STEP(wgrad(n, 4, n.t(n.p[1], nb, 2, 2 * C), n.ga[2], s));
  KK_STEP(dgrad(n, 4, n.t(n.ga[2], nb, 2, 4 * C), n.gb[2], s));        // d p1
  KK_TRY(K::pool2_bwd(n.gb[2], n.t(n.gb[1], nb, 1, 2 * C), true, s), "pool bwd");  // d a3 total
  KK_TRY(relu_b(n.gb[1], n.a[3], 1, 2 * C), "relu");
  KK_STEP(wgrad(n, 3, n.t(n.a[2], nb, 1, 2 * C), n.gb[1], s));
  KK_STEP(dgrad(n, 3, n.t(n.gb[1], nb, 1, 2 * C), n.ga[1], s));        // d a2
  KK_TRY(relu_b(n.ga[1], n.a[2], 1, 2 * C), "relu");
  KK_STEP(wgrad(n, 2, n.t(n.p[0], nb, 1, C), n.ga[1], s));
  KK_STEP(dgrad(n, 2, n.t(n.ga[1], nb, 1, 2 * C), n.gb[1], s));        // d p0
  KK_TRY(K::pool2_bwd(n.gb[1], n.t(n.gb[0], nb, 0, C), true, s), "pool bwd");  // d a1 total
  KK_TRY(relu_b(n.gb[0], n.a[1], 0, C), "relu");
  KK_STEP(wgrad(n, 1, n.t(n.a[0], nb, 0, C), n.gb[0], s));
  KK_STEP(dgrad(n, 1, n.t(n.gb[0], nb, 0, C), n.ga[0], s));            // d a0
  KK_TRY(relu_b(n.ga[0], n.a[0], 0, C), "relu");
  KK_STEP(wgrad(n, 0, n.t(n.x, nb, 0, kInChannels), n.ga[0], s));
  return KK_OK;
}

}  // namespace

extern "C" {

kk_status kk_net_create(kk_net **out, const kk_net_desc *d) {
  if (!out || !d) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  *out = nullptr;
  if (d->max_batch < 1 || d->height < 16 || d->width < 16 || d->height % 16 || d->width % 16 ||
      d->base_channels < 16 || d->base_channels % 16 || d->base_channels > 64) {
    set_error("bad net description (H, W multiples of 16; C in {16, 32, 48, 64})");
    return KK_ERR_INVALID_ARG;
  }
  if ((double)d->max_batch * d->height * d->width > 2.0e9 / 64) {
    set_error("max_batch x H x W too large");
    return KK_ERR_INVALID_ARG;
  }
  kk_net *n = new kk_net();
  cudaGetDevice(&n->device);
  n->B = d->max_batch;
  n->H = d->height;
  n->W = d->width;
  n->C = d->base_channels;
  n->seed = d->seed;
  define_layers(*n);
  Arena sizing;
  carve(*n, sizing);
  cudaError_t e = cudaMalloc(&n->block, sizing.size);
  if (e != cudaSuccess) {
    delete n;
    cudaGetLastError();
    set_error("device allocation of the net failed");
    return e == cudaErrorMemoryAllocation ? KK_ERR_OOM : KK_ERR_CUDA;
  }
  Arena A;
  A.base = (char *)n->block;
  carve(*n, A);
  const std::vector<float> h = init_params(*n);
  e = cudaMemcpy(n->w, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, n->n_params * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, n->n_params * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->status, 0, sizeof(int));
  if (e == cudaSuccess) e = kk::nn::to_bf16(n->w, n->wb, n->n_params, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    kk_status st = cuda_fail(e, "net initialisation");
    cudaFree(n->block);
    delete n;
    return st;
  }
  *out = n;
  return KK_OK;
}

void kk_net_destroy(kk_net *n) {
  if (!n) return;
  kk::DeviceGuard g(n->device);
  cudaFree(n->block);
  cudaFree(n->G);
  delete n;
}

kk_status kk_net_info(const kk_net *n, int64_t *n_params, int64_t *step) {
  if (!n) { set_error("null net"); return KK_ERR_INVALID_ARG; }
  if (n_params) *n_params = (int64_t)n->n_params;
  if (step) *step = n->step;
  return KK_OK;
}

kk_status kk_net_status(kk_net *n, int32_t *status) {
  if (!n || !status) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  kk::DeviceGuard g(n->device);
  int v = 0, zero = 0;
  KK_TRY(cudaMemcpy(&v, n->status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
  KK_TRY(cudaMemcpy(n->status, &zero, sizeof(int), cudaMemcpyHostToDevice), "reset status");
  *status = v;
  return KK_OK;
}

kk_status kk_net_get_params(const kk_net *n, float *d_dst, void *stream) {
  if (!n || !d_dst) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  kk::DeviceGuard g(n->device);
  KK_TRY(cudaMemcpyAsync(d_dst, n->w, n->n_params * sizeof(float), cudaMemcpyDeviceToDevice,
                         (cudaStream_t)stream), "copy params");
  return KK_OK;
}

kk_status kk_net_set_params(kk_net *n, const float *d_src, void *stream) {
  if (!n || !d_src) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  kk::DeviceGuard g(n->device);
  const cudaStream_t s = (cudaStream_t)stream;
  KK_TRY(cudaMemcpyAsync(n->w, d_src, n->n_params * sizeof(float), cudaMemcpyDeviceToDevice, s), "copy params");
  KK_TRY(kk::nn::to_bf16(n->w, n->wb, n->n_params, s), "bf16 copy");
  return KK_OK;
}

kk_status kk_net_forward(kk_net *n, int32_t nb, const void *d_in, const float *d_in_scale, void *d_out,
                         void *stream) {
  kk_status st = check_net(n, nb);
  if (st != KK_OK) return st;
  if (!d_in || !d_out || !aligned(d_in, 8) || !aligned(d_out, 8)) {
    set_error("null or misaligned image pointer");
    return KK_ERR_INVALID_ARG;
  }
  kk::DeviceGuard g(n->device);
  kk::NvtxRange range("kk_net_forward");
  const cudaStream_t s = (cudaStream_t)stream;
  if ((st = forward(*n, nb, d_in, d_in_scale, s)) != KK_OK) return st;
  KK_TRY(kk::nn::residual_mse(n->x, kInChannels, n->head, kHeadChannels, nullptr, nullptr, nb, n->H * n->W,
                              (float2 *)d_out, nullptr, nullptr, s), "residual");
  return KK_OK;
}

kk_status kk_net_loss_grad(kk_net *n, int32_t nb, const void *d_in, const float *d_in_scale,
                           const void *d_target, const float *d_target_scale, float *d_loss, float *d_grad,
                           void *d_out, void *stream) {
  kk_status st = check_net(n, nb);
  if (st != KK_OK) return st;
  if (!d_in || !d_target || !d_loss || !aligned(d_in, 8) || !aligned(d_target, 8) ||
      (d_out && !aligned(d_out, 8))) {
    set_error("null or misaligned pointer");
    return KK_ERR_INVALID_ARG;
  }
  kk::DeviceGuard g(n->device);
  kk::NvtxRange range("kk_net_loss_grad");
  const cudaStream_t s = (cudaStream_t)stream;
  if ((st = forward(*n, nb, d_in, d_in_scale, s)) != KK_OK) return st;
  const int hw = n->H * n->W;
  KK_TRY(kk::nn::residual_mse(n->x, kInChannels, n->head, kHeadChannels, (const float2 *)d_target,
                              d_target_scale, nb, hw, (float2 *)d_out, n->dhead, n->loss_part, s), "loss");
  KK_TRY(kk::nn::sum_scalar(n->loss_part, kk::nn::residual_blocks(nb, hw), 1.f / (2.f * (float)nb * (float)hw),
                            d_loss, s), "loss sum");
  kk::NvtxRange rb("kk_net_loss_grad/backward");
  if ((st = backward(*n, nb, s)) != KK_OK) return st;
  if (d_grad)
    KK_TRY(cudaMemcpyAsync(d_grad, n->g, n->n_params * sizeof(float), cudaMemcpyDeviceToDevice, s), "grad copy");
  return KK_OK;
}

kk_status kk_net_adam(kk_net *n, float lr, float b1, float b2, float eps, float wd, void *stream) {
  if (!n) { set_error("null net"); return KK_ERR_INVALID_ARG; }
  if (!(lr >= 0.f) || !(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f) || !(eps > 0.f) || !(wd >= 0.f)) {
    set_error("bad Adam hyper-parameters");
    return KK_ERR_INVALID_ARG;
  }
  kk::DeviceGuard g(n->device);
  const double t = (double)(n->step + 1);
  const float bc1 = (float)(1.0 - std::pow((double)b1, t));
  const float bc2 = (float)(1.0 - std::pow((double)b2, t));
  KK_TRY(kk::nn::adam(n->w, n->g, n->m, n->v, n->wb, n->n_params, lr, b1, b2, eps, bc1, bc2, wd,
                      (cudaStream_t)stream), "adam");
  n->step += 1;
  return KK_OK;
}

// ---- checkpoints ---------------------------------------------------------
namespace {
struct CkptHeader {
  char magic[8];
  int32_t H, W, C, version;
  int64_t n_params, step;
  uint64_t seed;
};
constexpr char kMagic[8] = {'K', 'K', 'N', 'E', 'T', 'C', 'K', '1'};
}  // namespace

kk_status kk_net_save(const kk_net *n, const char *path, void *stream) {
  if (!n || !path) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  kk::DeviceGuard g(n->device);
  KK_TRY(cudaStreamSynchronize((cudaStream_t)stream), "sync before save");
  std::vector<float> h(3 * n->n_params);
  KK_TRY(cudaMemcpy(h.data(), n->w, n->n_params * 4, cudaMemcpyDeviceToHost), "read w");
  KK_TRY(cudaMemcpy(h.data() + n->n_params, n->m, n->n_params * 4, cudaMemcpyDeviceToHost), "read m");
  KK_TRY(cudaMemcpy(h.data() + 2 * n->n_params, n->v, n->n_params * 4, cudaMemcpyDeviceToHost), "read v");
  CkptHeader hd{};
  std::memcpy(hd.magic, kMagic, 8);
  hd.H = n->H;
  hd.W = n->W;
  hd.C = n->C;
  hd.version = 1;
  hd.n_params = (int64_t)n->n_params;
  hd.step = n->step;
  hd.seed = n->seed;
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "wb");
  if (!f) { set_error("cannot open checkpoint for writing"); return KK_ERR_INVALID_ARG; }
  const bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1 && std::fwrite(h.data(), 4, h.size(), f) == h.size();
  if (std::fclose(f) != 0 || !ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    set_error("checkpoint write failed");
    return KK_ERR_INVALID_ARG;
  }
  return KK_OK;
}

kk_status kk_net_load(kk_net *n, const char *path, void *stream) {
  if (!n || !path) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  kk::DeviceGuard g(n->device);
  FILE *f = std::fopen(path, "rb");
  if (!f) { set_error("cannot open checkpoint"); return KK_ERR_INVALID_ARG; }
  CkptHeader hd{};
  std::vector<float> h(3 * n->n_params);
  bool ok = std::fread(&hd, sizeof hd, 1, f) == 1 && std::memcmp(hd.magic, kMagic, 8) == 0 && hd.version == 1 &&
            hd.H == n->H && hd.W == n->W && hd.C == n->C && hd.n_params == (int64_t)n->n_params;
  ok = ok && std::fread(h.data(), 4, h.size(), f) == h.size();
  std::fclose(f);
  if (!ok) { set_error("checkpoint does not match this net or is truncated"); return KK_ERR_INVALID_ARG; }
  const cudaStream_t s = (cudaStream_t)stream;
  KK_TRY(cudaStreamSynchronize(s), "sync before load");
  KK_TRY(cudaMemcpy(n->w, h.data(), n->n_params * 4, cudaMemcpyHostToDevice), "write w");
  KK_TRY(cudaMemcpy(n->m, h.data() + n->n_params, n->n_params * 4, cudaMemcpyHostToDevice), "write m");
  KK_TRY(cudaMemcpy(n->v, h.data() + 2 * n->n_params, n->n_params * 4, cudaMemcpyHostToDevice), "write v");
  KK_TRY(kk::nn::to_bf16(n->w, n->wb, n->n_params, s), "bf16 copy");
  KK_TRY(cudaStreamSynchronize(s), "sync after load");
  n->step = hd.step;
  n->seed = hd.seed;
  return KK_OK;
}

// ---- judge -------------------------------------------------------------------
static kk_status ensure_judge_buffers(kk_net *n) {
  if (n->G) return KK_OK;
  const size_t hw = (size_t)n->H * n->W;
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, (hw + 3 * (size_t)n->B * hw) * sizeof(float2));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("judge buffers: device allocation failed");
    return KK_ERR_OOM;
  }
  n->G = (float2 *)p;
  n->dft_tmp = n->G + hw;
  n->dft_A = n->dft_tmp + n->B * hw;
  n->dft_C = n->dft_A + n->B * hw;
  return KK_OK;
}

kk_status kk_net_judge_filter(kk_net *n, const void *d_psf_c, const void *d_psf_f, float rho, void *stream) {
  if (!n || !d_psf_c || !d_psf_f || !(rho > 0.f && rho < 1.f)) {
    set_error("null argument or rho outside (0, 1)");
    return KK_ERR_INVALID_ARG;
  }
  kk::DeviceGuard g(n->device);
  kk_status st = ensure_judge_buffers(n);
  if (st != KK_OK) return st;
  const cudaStream_t s = (cudaStream_t)stream;
  const size_t hw = (size_t)n->H * n->W;
  // spectra of the two PSFs in dft_A[0], dft_C[0]
  KK_TRY(kk::nn::dft2((const float2 *)d_psf_c, 1, n->H, n->W, -1, n->dft_tmp, n->dft_A, s), "dft");
  KK_TRY(kk::nn::dft2((const float2 *)d_psf_f, 1, n->H, n->W, -1, n->dft_tmp, n->dft_C, s), "dft");
  KK_TRY(kk::nn::judge_filter(n->dft_A, n->dft_C, (int)hw, rho, n->G, s), "filter");
  n->have_filter = true;
  return KK_OK;
}

kk_status kk_net_judge(kk_net *n, int32_t nb, const void *d_out, const void *d_xc, float *d_stat, void *stream) {
  kk_status st = check_net(n, nb);
  if (st != KK_OK) return st;
  if (!d_out || !d_xc || !d_stat) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  if (!n->have_filter) { set_error("kk_net_judge_filter has not been called"); return KK_ERR_INVALID_ARG; }
  kk::DeviceGuard g(n->device);
  const cudaStream_t s = (cudaStream_t)stream;
  KK_TRY(kk::nn::dft2((const float2 *)d_out, nb, n->H, n->W, -1, n->dft_tmp, n->dft_A, s), "dft");
  KK_TRY(kk::nn::dft2((const float2 *)d_xc, nb, n->H, n->W, -1, n->dft_tmp, n->dft_C, s), "dft");
  KK_TRY(kk::nn::judge_stat(n->dft_A, n->dft_C, n->G, nb, n->H * n->W, d_stat, s), "judge");
  return KK_OK;
}

kk_status kk_net_image_scale(const void *d_img, int32_t nb, int32_t h, int32_t w, float *d_scale, void *stream) {
  if (!d_img || !d_scale || nb < 1 || h < 1 || w < 1 || (double)h * w > 2.0e9 || !aligned(d_img, 8)) {
    set_error("bad image-scale arguments");
    return KK_ERR_INVALID_ARG;
  }
  KK_TRY(kk::nn::image_scale((const float2 *)d_img, nb, h * w, d_scale, (cudaStream_t)stream), "image scale");
  return KK_OK;
}

// ---- layer-level calls --------------------------------------------------------
static kk_status check_layer(const void *x, int n, int h, int w, int cin, const void *wt, int cout) {
  if (!x || !wt) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  if (n < 1 || h < 1 || w < 1 || cin < 16 || cout < 16 || cin % 16 || cout % 16 || cin > 1024 || cout > 1024 ||
      (double)n * h * w * std::max(cin, cout) > 2.0e9) {
    set_error("bad layer shape (cin, cout multiples of 16)");
    return KK_ERR_INVALID_ARG;
  }
  if (!aligned(x, 16) || !aligned(wt, 16)) { set_error("operands must be 16-byte aligned"); return KK_ERR_INVALID_ARG; }
  return KK_OK;
}

kk_status kk_nn_conv3x3(const void *d_x, int32_t n, int32_t h, int32_t w, int32_t cin, const void *d_w, int32_t cout,
                        const float *d_bias, int32_t relu, void *d_y, float *d_yf, void *stream) {
  kk_status st = check_layer(d_x, n, h, w, cin, d_w, cout);
  if (st != KK_OK) return st;
  if (!d_y && !d_yf) { set_error("no output"); return KK_ERR_INVALID_ARG; }
  Tensor4 x{(__nv_bfloat16 *)d_x, n, h, w, cin};
  KK_TRY(kk::nn::conv3x3_tc(x, (const __nv_bfloat16 *)d_w, cout, d_bias, relu != 0, (__nv_bfloat16 *)d_y, d_yf,
                            nullptr, (cudaStream_t)stream), "conv");
  return KK_OK;
}

kk_status kk_nn_conv3x3_dgrad(const void *d_dy, int32_t n, int32_t h, int32_t w, int32_t cout, const void *d_w,
                              int32_t cin, void *d_dx, void *d_ws, void *stream) {
  kk_status st = check_layer(d_dy, n, h, w, cout, d_w, cin);
  if (st != KK_OK) return st;
  if (!d_dx || !d_ws || !aligned(d_ws, 16)) { set_error("null or misaligned output / workspace"); return KK_ERR_INVALID_ARG; }
  const cudaStream_t s = (cudaStream_t)stream;
  KK_TRY(kk::nn::flip_transpose((const __nv_bfloat16 *)d_w, cout, cin, (__nv_bfloat16 *)d_ws, s), "flip");
  Tensor4 dy{(__nv_bfloat16 *)d_dy, n, h, w, cout};
  KK_TRY(kk::nn::conv3x3_tc(dy, (const __nv_bfloat16 *)d_ws, cin, nullptr, false, (__nv_bfloat16 *)d_dx, nullptr,
                            nullptr, s), "dgrad");
  return KK_OK;
}

kk_status kk_nn_status(int32_t *status) {
  if (!status) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  int v = 0;
  KK_TRY(kk::nn::conv_status(&v), "layer status");
  *status = v;
  return KK_OK;
}

kk_status kk_nn_conv3x3_wgrad_workspace(int32_t n, int32_t h, int32_t w, int32_t cin, int32_t cout, size_t *bytes) {
  static const char dummy[16] = {};
  kk_status st = check_layer(dummy, n, h, w, cin, dummy, cout);
  if (st != KK_OK) return st;
  if (!bytes) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  Tensor4 x{nullptr, n, h, w, cin};
  *bytes = kk::nn::wgrad_part_floats(x, cout) * sizeof(float);
  return KK_OK;
}

kk_status kk_nn_conv3x3_wgrad(const void *d_x, int32_t n, int32_t h, int32_t w, int32_t cin, const void *d_dy,
                              int32_t cout, float *d_dw, float *d_db, void *d_ws, void *stream) {
  kk_status st = check_layer(d_x, n, h, w, cin, d_dy, cout);
  if (st != KK_OK) return st;
  if (!d_dw || !d_ws) { set_error("null output or workspace"); return KK_ERR_INVALID_ARG; }
  const cudaStream_t s = (cudaStream_t)stream;
  Tensor4 x{(__nv_bfloat16 *)d_x, n, h, w, cin};
  int splits = 0, nb = 0;
  KK_TRY(kk::nn::conv3x3_wgrad(x, (const __nv_bfloat16 *)d_dy, cout, (float *)d_ws, &splits, &nb, nullptr, s),
         "wgrad");
  const size_t nw = (size_t)cout * 9 * cin;
  KK_TRY(kk::nn::reduce_splits((const float *)d_ws, splits, nw, nw, d_dw, s), "wgrad reduce");
  if (d_db)
    KK_TRY(kk::nn::reduce_splits((const float *)d_ws + (size_t)splits * nw, nb, cout, cout, d_db, s), "bias reduce");
  return KK_OK;
}

}  // extern "C"
