// Image-quality measures of beamformed images: gCNR of an inclusion against
// a background region and half-amplitude widths of point targets (the
// contrast and resolution judgements of Section III, Figs. 4 and 5).
//
// Layout on the device:
//  - per region pair m, a label box covering the union of both regions'
//    pixel bounding boxes: labels[off + r*bw + c] (bit 0 inside, bit 1
//    outside) for pixel (bx0 + c, bz0 + r), built once at creation;
//  - the images themselves, read twice per region pair (range, then
//    histogram) by one CTA per (pair, image); the second read hits L1/L2.
// Every integer (label, bin, argmax, crossing index) is decided with
// explicitly rounded IEEE operations (no contraction), as the header states.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "kk_internal.h"
#include "kkquality.h"

using kk::DeviceGuard;
using kk::cuda_fail;
using kk::set_error;

namespace {

struct LabelBox {
  int bx0, bz0, bw, bh;
  long long off;
};

constexpr int kGcnrThreads = 256;
constexpr int kFwhmWarps = 8;
constexpr int kMaxBins = 4096;
constexpr int kUnroll = 4;  // columns per lane per step of the gCNR passes

__device__ __forceinline__ bool in_region(const kk_region &R, double x, double z) {
  if (R.kind == KK_REGION_RECT) return x >= R.a && x <= R.b && z >= R.c && z <= R.d;
  const double ex = __dsub_rn(x, R.a), ez = __dsub_rn(z, R.b);
  const double d2 = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ez, ez));
  if (R.kind == KK_REGION_DISK) return d2 <= __dmul_rn(R.c, R.c);
  return d2 > __dmul_rn(R.c, R.c) && d2 <= __dmul_rn(R.d, R.d);
}

__global__ void k_labels(const kk_region *inside, const kk_region *outside, const LabelBox *boxes,
                         uint8_t *labels, double x0, double dx, double z0, double dz) {
  const int m = blockIdx.y;
  const LabelBox b = boxes[m];
  const long long n = (long long)b.bw * b.bh;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / b.bw), c = (int)(e % b.bw);
    const double x = __dadd_rn(x0, __dmul_rn((double)(b.bx0 + c), dx));
    const double z = __dadd_rn(z0, __dmul_rn((double)(b.bz0 + r), dz));
    labels[b.off + e] = (uint8_t)((in_region(inside[m], x, z) ? 1 : 0) |
                                  (in_region(outside[m], x, z) ? 2 : 0));
  }
}

template <int KIND>
__device__ __forceinline__ float envelope(const void *img, long long i) {
  if (KIND == KK_IMAGE_COMPLEX) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(img) + i);
    return __fsqrt_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)));
  } else {
    return __fsqrt_rn(__ldg(reinterpret_cast<const float *>(img) + i));
  }
}

// One CTA per (region pair m = blockIdx.x, image n = blockIdx.y).
template <int KIND>
__global__ void __launch_bounds__(kGcnrThreads)
    k_gcnr(const void *img, long long img_elems, int nx, const LabelBox *boxes,
           const uint8_t *labels, int n_bins, int n_contrast, double *out) {
  extern __shared__ int hist[];  // [2][n_bins]
  __shared__ float s_lo[kGcnrThreads / 32], s_hi[kGcnrThreads / 32];
  __shared__ int s_nin[kGcnrThreads / 32], s_nout[kGcnrThreads / 32];
  __shared__ long long s_ovl[kGcnrThreads / 32];
  const int m = blockIdx.x, n = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const LabelBox b = boxes[m];
  const long long base = (long long)n * img_elems + (long long)b.bz0 * nx + b.bx0;

  // Both passes walk the label box row by row (one warp per row, lanes
  // along the row) and take kUnroll columns per lane per step, issuing all
  // of that step's loads before using them.
  float lo = INFINITY, hi = -INFINITY;
  int nin = 0, nout = 0;
  for (int r = warp; r < b.bh; r += nwarp) {
    const uint8_t *lrow = labels + b.off + (long long)r * b.bw;
    const long long prow = base + (long long)r * nx;
    for (int c0 = lane; c0 < b.bw; c0 += 32 * kUnroll) {
      int L[kUnroll];
      float e[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int c = c0 + 32 * u;
        L[u] = c < b.bw ? lrow[c] : 0;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) e[u] = L[u] ? envelope<KIND>(img, prow + c0 + 32 * u) : 0.f;
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (L[u]) {
          lo = fminf(lo, e[u]);
          hi = fmaxf(hi, e[u]);
          nin += L[u] & 1;
          nout += L[u] >> 1;
        }
    }
  }
  for (int o = 16; o; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    nin += __shfl_xor_sync(0xffffffffu, nin, o);
    nout += __shfl_xor_sync(0xffffffffu, nout, o);
  }
  if (lane == 0) {
    s_lo[warp] = lo;
    s_hi[warp] = hi;
    s_nin[warp] = nin;
    s_nout[warp] = nout;
  }
  for (int i = threadIdx.x; i < 2 * n_bins; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  lo = s_lo[0];
  hi = s_hi[0];
  nin = s_nin[0];
  nout = s_nout[0];
  for (int w = 1; w < nwarp; ++w) {
    lo = fminf(lo, s_lo[w]);
    hi = fmaxf(hi, s_hi[w]);
    nin += s_nin[w];
    nout += s_nout[w];
  }
  if (nin == 0 || nout == 0) {
    if (threadIdx.x == 0) out[(long long)n * n_contrast + m] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const bool flat = !(hi > lo);
  const float w = __fsub_rn(hi, lo);
  const float nb = (float)n_bins;
  for (int r = warp; r < b.bh; r += nwarp) {
    const uint8_t *lrow = labels + b.off + (long long)r * b.bw;
    const long long prow = base + (long long)r * nx;
    for (int c0 = lane; c0 < b.bw; c0 += 32 * kUnroll) {
      int L[kUnroll];
      float e[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int c = c0 + 32 * u;
        L[u] = c < b.bw ? lrow[c] : 0;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        e[u] = (L[u] && !flat) ? envelope<KIND>(img, prow + c0 + 32 * u) : 0.f;
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (!L[u]) continue;
        int bin = 0;
        if (!flat) {
          const float q = __fdiv_rn(__fmul_rn(__fsub_rn(e[u], lo), nb), w);
          bin = min((int)q, n_bins - 1);
        }
        if (L[u] & 1) atomicAdd(&hist[bin], 1);
        if (L[u] & 2) atomicAdd(&hist[n_bins + bin], 1);
      }
    }
  }
  __syncthreads();
  long long s = 0;
  for (int i = threadIdx.x; i < n_bins; i += blockDim.x) {
    const long long a = (long long)hist[i] * nout, c = (long long)hist[n_bins + i] * nin;
    s += a < c ? a : c;
  }
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) s_ovl[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int i = 0; i < nwarp; ++i) t += s_ovl[i];
    const double den = __dmul_rn((double)nin, (double)nout);
    out[(long long)n * n_contrast + m] = __dsub_rn(1.0, __ddiv_rn((double)t, den));
  }
}

// Half-maximum crossing walking from the peak k_pk in direction dir along a
// line of n samples (element stride `stride` from `line`); coordinate of
// sample k is o + k*d.  Warp-cooperative; every lane returns the result.
template <int KIND>
__device__ double half_crossing(const void *img, long long line, long long stride, int n, int k_pk,
                                float half, int dir, double o, double d) {
  const int lane = threadIdx.x & 31;
  for (int k0 = k_pk + dir;; k0 += 32 * dir) {
    const int k = k0 + lane * dir;
    const bool valid = k >= 0 && k < n;
    const bool below = valid && envelope<KIND>(img, line + (long long)k * stride) < half;
    const unsigned bal = __ballot_sync(0xffffffffu, below);
    const unsigned out = __ballot_sync(0xffffffffu, !valid);
    if (bal) {
      const int kn = k0 + (__ffs(bal) - 1) * dir, kin = kn - dir;
      const float ein = envelope<KIND>(img, line + (long long)kin * stride);
      const float eout = envelope<KIND>(img, line + (long long)kn * stride);
      const double t = __ddiv_rn(__dsub_rn((double)ein, (double)half),
                                 __dsub_rn((double)ein, (double)eout));
      const double cin = __dadd_rn(o, __dmul_rn((double)kin, d));
      const double cout = __dadd_rn(o, __dmul_rn((double)kn, d));
      return __dadd_rn(cin, __dmul_rn(t, __dsub_rn(cout, cin)));
    }
    if (out) return __longlong_as_double(0x7ff8000000000000ll);
  }
}

// One warp per (image, target) item.
template <int KIND>
__global__ void __launch_bounds__(kFwhmWarps * 32)
    k_fwhm(const void *img, long long img_elems, int nx, int nz, double x0, double dx, double z0,
           double dz, const kk_target *targets, int n_targets, long long n_items,
           kk_fwhm_result *out) {
  const int lane = threadIdx.x & 31;
  const long long item = (long long)blockIdx.x * kFwhmWarps + (threadIdx.x >> 5);
  if (item >= n_items) return;
  const long long n = item / n_targets;
  const kk_target t = targets[item % n_targets];
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const long long x_lo = max((long long)t.ix - t.wx, 0ll), x_hi = min((long long)t.ix + t.wx, (long long)nx - 1);
  const long long z_lo = max((long long)t.iz - t.wz, 0ll), z_hi = min((long long)t.iz + t.wz, (long long)nz - 1);
  kk_fwhm_result r;
  r.ix = r.iz = -1;
  r.peak = __int_as_float(0x7fc00000);
  r.reserved = 0;
  r.lateral = r.axial = nan;
  if (x_lo > x_hi || z_lo > z_hi) {
    if (lane == 0) out[item] = r;
    return;
  }
  const long long base = n * img_elems;
  float best = -INFINITY;
  long long bidx = std::numeric_limits<long long>::max();
  for (long long zz = z_lo; zz <= z_hi; ++zz)
    for (long long xx = x_lo + lane; xx <= x_hi; xx += 32) {
      const long long f = zz * nx + xx;
      const float e = envelope<KIND>(img, base + f);
      if (e > best || (e == best && f < bidx)) {
        best = e;
        bidx = f;
      }
    }
  for (int o = 16; o; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ob > best || (ob == best && oi < bidx)) {
      best = ob;
      bidx = oi;
    }
  }
  const int bz = (int)(bidx / nx), bx = (int)(bidx % nx);
  const float half = __fmul_rn(best, 0.5f);
  const long long row = base + (long long)bz * nx, col = base + bx;
  const double xr = half_crossing<KIND>(img, row, 1, nx, bx, half, +1, x0, dx);
  const double xl = half_crossing<KIND>(img, row, 1, nx, bx, half, -1, x0, dx);
  const double zr = half_crossing<KIND>(img, col, nx, nz, bz, half, +1, z0, dz);
  const double zl = half_crossing<KIND>(img, col, nx, nz, bz, half, -1, z0, dz);
  r.ix = bx;
  r.iz = bz;
  r.peak = best;
  r.lateral = __dsub_rn(xr, xl);
  r.axial = __dsub_rn(zr, zl);
  if (lane == 0) out[item] = r;
}

bool is_finite(double v) { return std::isfinite(v); }

// Conservative pixel-index bounding box of a region (one pixel of margin on
// each side; membership itself is decided per pixel on the device).
void region_box(const kk_region &R, const kk_grid &g, int box[4]) {
  double xa, xb, za, zb;
  if (R.kind == KK_REGION_RECT) {
    xa = R.a; xb = R.b; za = R.c; zb = R.d;
  } else {
    const double r = R.kind == KK_REGION_DISK ? R.c : R.d;
    xa = R.a - r; xb = R.a + r; za = R.b - r; zb = R.b + r;
  }
  auto idx = [](double v, double o, double d, int n, bool up) {
    double t = (v - o) / d;
    t = up ? std::ceil(t) + 1.0 : std::floor(t) - 1.0;
    t = std::fmin(std::fmax(t, -1.0), (double)n);
    return (int)t;
  };
  box[0] = std::max(idx(xa, g.x0, g.dx, g.nx, false), 0);
  box[1] = std::min(idx(xb, g.x0, g.dx, g.nx, true), g.nx - 1);
  box[2] = std::max(idx(za, g.z0, g.dz, g.nz, false), 0);
  box[3] = std::min(idx(zb, g.z0, g.dz, g.nz, true), g.nz - 1);
}

bool valid_region(const kk_region &R, std::string &why) {
  if (!(is_finite(R.a) && is_finite(R.b) && is_finite(R.c) && is_finite(R.d))) {
    why = "region parameters must be finite";
    return false;
  }
  switch (R.kind) {
    case KK_REGION_DISK:
      if (R.c < 0) { why = "disk radius must be >= 0"; return false; }
      return true;
    case KK_REGION_ANNULUS:
      if (R.c < 0 || R.d < R.c) { why = "annulus needs 0 <= r1 <= r2"; return false; }
      return true;
    case KK_REGION_RECT:
      return true;
    default:
      why = "unknown region kind";
      return false;
  }
}

}  // namespace

struct kk_quality {
  int device = 0;
  kk_grid g{};
  int kind = 0, n_contrast = 0, n_bins = 0, n_targets = 0;
  LabelBox *d_boxes = nullptr;
  uint8_t *d_labels = nullptr;
  kk_target *d_targets = nullptr;
  ~kk_quality() {
    if (d_boxes) cudaFree(d_boxes);
    if (d_labels) cudaFree(d_labels);
    if (d_targets) cudaFree(d_targets);
  }
};

extern "C" kk_status kk_quality_create(kk_quality **out, const kk_quality_desc *d) {
  if (!out || !d) {
    set_error("kk_quality_create: null argument");
    return KK_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const kk_grid &g = d->grid;
  if (g.nx < 1 || g.nz < 1 || !(g.dx > 0) || !(g.dz > 0) || !is_finite(g.dx) || !is_finite(g.dz) ||
      !is_finite(g.x0) || !is_finite(g.z0)) {
    set_error("kk_quality_create: grid needs nx, nz >= 1, finite x0, z0 and dx, dz > 0");
    return KK_ERR_INVALID_ARG;
  }
  if (d->image_kind != KK_IMAGE_COMPLEX && d->image_kind != KK_IMAGE_INTENSITY) {
    set_error("kk_quality_create: image_kind must be KK_IMAGE_COMPLEX or KK_IMAGE_INTENSITY");
    return KK_ERR_INVALID_ARG;
  }
  if (d->n_contrast < 0 || d->n_targets < 0 || d->n_bins < 1 || d->n_bins > kMaxBins) {
    set_error("kk_quality_create: need n_contrast >= 0, n_targets >= 0 and 1 <= n_bins <= 4096");
    return KK_ERR_INVALID_ARG;
  }
  if ((d->n_contrast > 0 && (!d->inside || !d->outside)) || (d->n_targets > 0 && !d->targets)) {
    set_error("kk_quality_create: null region or target array");
    return KK_ERR_INVALID_ARG;
  }
  std::string why;
  for (int m = 0; m < d->n_contrast; ++m)
    if (!valid_region(d->inside[m], why) || !valid_region(d->outside[m], why)) {
      set_error("kk_quality_create: region pair " + std::to_string(m) + ": " + why);
      return KK_ERR_INVALID_ARG;
    }
  for (int t = 0; t < d->n_targets; ++t)
    if (d->targets[t].wx < 0 || d->targets[t].wz < 0) {
      set_error("kk_quality_create: target " + std::to_string(t) + " has a negative half-width");
      return KK_ERR_INVALID_ARG;
    }
  DeviceGuard guard(d->device);
  if (!guard.ok) {
    set_error("kk_quality_create: cannot select device " + std::to_string(d->device));
    return KK_ERR_CUDA;
  }
  kk_quality *q = new (std::nothrow) kk_quality;
  if (!q) {
    set_error("kk_quality_create: host allocation failed");
    return KK_ERR_OOM;
  }
  q->device = d->device;
  q->g = g;
  q->kind = d->image_kind;
  q->n_contrast = d->n_contrast;
  q->n_bins = d->n_bins;
  q->n_targets = d->n_targets;

  std::vector<LabelBox> boxes(d->n_contrast);
  long long total = 0, max_px = 0;
  for (int m = 0; m < d->n_contrast; ++m) {
    int a[4], b[4];
    region_box(d->inside[m], g, a);
    region_box(d->outside[m], g, b);
    const bool ea = a[0] > a[1] || a[2] > a[3], eb = b[0] > b[1] || b[2] > b[3];
    int u[4];
    if (ea && eb) {
      u[0] = 0; u[1] = -1; u[2] = 0; u[3] = -1;
    } else if (ea) {
      std::memcpy(u, b, sizeof u);
    } else if (eb) {
      std::memcpy(u, a, sizeof u);
    } else {
      u[0] = std::min(a[0], b[0]); u[1] = std::max(a[1], b[1]);
      u[2] = std::min(a[2], b[2]); u[3] = std::max(a[3], b[3]);
    }
    LabelBox &L = boxes[m];
    L.bx0 = u[0];
    L.bz0 = u[2];
    L.bw = std::max(u[1] - u[0] + 1, 0);
    L.bh = std::max(u[3] - u[2] + 1, 0);
    if (L.bw == 0 || L.bh == 0) L.bw = L.bh = 0;
    L.off = total;
    total += (long long)L.bw * L.bh;
    max_px = std::max(max_px, (long long)L.bw * L.bh);
  }

  auto fail = [&](cudaError_t e, const char *what) {
    delete q;
    return e == cudaErrorMemoryAllocation ? (set_error(std::string(what) + ": out of device memory"), KK_ERR_OOM)
                                          : cuda_fail(e, what);
  };
  cudaError_t e = cudaSuccess;
  if (d->n_contrast > 0) {
    e = cudaMalloc(&q->d_boxes, sizeof(LabelBox) * d->n_contrast);
    if (e != cudaSuccess) return fail(e, "kk_quality_create: cudaMalloc");
    e = cudaMemcpy(q->d_boxes, boxes.data(), sizeof(LabelBox) * d->n_contrast, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(e, "kk_quality_create: cudaMemcpy");
    if (total > 0) {
      e = cudaMalloc(&q->d_labels, (size_t)total);
      if (e != cudaSuccess) return fail(e, "kk_quality_create: cudaMalloc");
      kk_region *d_reg = nullptr;
      e = cudaMalloc(&d_reg, sizeof(kk_region) * 2 * d->n_contrast);
      if (e != cudaSuccess) return fail(e, "kk_quality_create: cudaMalloc");
      e = cudaMemcpy(d_reg, d->inside, sizeof(kk_region) * d->n_contrast, cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(d_reg + d->n_contrast, d->outside, sizeof(kk_region) * d->n_contrast,
                       cudaMemcpyHostToDevice);
      if (e == cudaSuccess) {
        const int threads = 256;
        const long long blocks = std::min<long long>((max_px + threads - 1) / threads, 1024);
        k_labels<<<dim3((unsigned)blocks, (unsigned)d->n_contrast), threads>>>(
            d_reg, d_reg + d->n_contrast, q->d_boxes, q->d_labels, g.x0, g.dx, g.z0, g.dz);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
      }
      cudaFree(d_reg);
      if (e != cudaSuccess) return fail(e, "kk_quality_create: label kernel");
    }
  }
  if (d->n_targets > 0) {
    e = cudaMalloc(&q->d_targets, sizeof(kk_target) * d->n_targets);
    if (e != cudaSuccess) return fail(e, "kk_quality_create: cudaMalloc");
    e = cudaMemcpy(q->d_targets, d->targets, sizeof(kk_target) * d->n_targets, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(e, "kk_quality_create: cudaMemcpy");
  }
  *out = q;
  return KK_OK;
}

extern "C" void kk_quality_destroy(kk_quality *q) {
  if (!q) return;
  DeviceGuard guard(q->device);
  delete q;
}

extern "C" kk_status kk_quality_gcnr(const kk_quality *q, const void *d_images, int32_t n_images,
                                     double *d_gcnr, void *stream) {
  if (!q || n_images < 0) {
    set_error("kk_quality_gcnr: null plan or negative image count");
    return KK_ERR_INVALID_ARG;
  }
  if (n_images == 0 || q->n_contrast == 0) return KK_OK;
  if (!d_images || !d_gcnr) {
    set_error("kk_quality_gcnr: null image or output pointer");
    return KK_ERR_INVALID_ARG;
  }
  if (n_images > 65535) {
    set_error("kk_quality_gcnr: at most 65535 images per call");
    return KK_ERR_INVALID_ARG;
  }
  DeviceGuard guard(q->device);
  const long long elems = (long long)q->g.nx * q->g.nz;
  const size_t smem = sizeof(int) * 2 * (size_t)q->n_bins;
  const dim3 grid((unsigned)q->n_contrast, (unsigned)n_images);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (q->kind == KK_IMAGE_COMPLEX)
    k_gcnr<KK_IMAGE_COMPLEX><<<grid, kGcnrThreads, smem, s>>>(d_images, elems, q->g.nx, q->d_boxes,
                                                             q->d_labels, q->n_bins, q->n_contrast, d_gcnr);
  else
    k_gcnr<KK_IMAGE_INTENSITY><<<grid, kGcnrThreads, smem, s>>>(d_images, elems, q->g.nx, q->d_boxes,
                                                               q->d_labels, q->n_bins, q->n_contrast, d_gcnr);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KK_OK : cuda_fail(e, "kk_quality_gcnr: launch");
}

extern "C" kk_status kk_quality_fwhm(const kk_quality *q, const void *d_images, int32_t n_images,
                                     kk_fwhm_result *d_out, void *stream) {
  if (!q || n_images < 0) {
    set_error("kk_quality_fwhm: null plan or negative image count");
    return KK_ERR_INVALID_ARG;
  }
  if (n_images == 0 || q->n_targets == 0) return KK_OK;
  if (!d_images || !d_out) {
    set_error("kk_quality_fwhm: null image or output pointer");
    return KK_ERR_INVALID_ARG;
  }
  DeviceGuard guard(q->device);
  const long long elems = (long long)q->g.nx * q->g.nz;
  const long long items = (long long)n_images * q->n_targets;
  const long long blocks = (items + kFwhmWarps - 1) / kFwhmWarps;
  if (blocks > 0x7fffffffll) {
    set_error("kk_quality_fwhm: too many (image, target) items");
    return KK_ERR_INVALID_ARG;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const kk_grid &g = q->g;
  if (q->kind == KK_IMAGE_COMPLEX)
    k_fwhm<KK_IMAGE_COMPLEX><<<(unsigned)blocks, kFwhmWarps * 32, 0, s>>>(
        d_images, elems, g.nx, g.nz, g.x0, g.dx, g.z0, g.dz, q->d_targets, q->n_targets, items, d_out);
  else
    k_fwhm<KK_IMAGE_INTENSITY><<<(unsigned)blocks, kFwhmWarps * 32, 0, s>>>(
        d_images, elems, g.nx, g.nz, g.x0, g.dx, g.z0, g.dz, q->d_targets, q->n_targets, items, d_out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KK_OK : cuda_fail(e, "kk_quality_fwhm: launch");
}
