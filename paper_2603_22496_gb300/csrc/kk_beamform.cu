// kk_beamform.cu -- KK image formation, Eq. (KK), with compounding.
//
//   B_j(ix, iz) = sum_{p in group j} lerp(y_p, s_p(ix, iz)),
//   s_p(ix, iz) = A_p ix + B_p iz + C_p   (samples; affine because both the
//   transmit delay s_i.r/c and the receive delay s_o.r/c are linear in r,
//   Section II-F's LUT decomposition taken to its limit).
//
// Design (gather-bound; tensor cores do not apply):
//  * one CTA per 32x32 pixel tile (and per slice of the pair list when the
//    grid has too few tiles to fill the GPU); 4 warps, lane = x offset,
//    8 z rows per thread;
//  * pairs are processed in stages: for each pair of a stage the CTA stages
//    the window of y_p that its tile can touch into shared memory as
//    (y[k], y[k+1] - y[k]) so one 16-byte load gives a linear interpolation;
//    entries outside [0, T-2] are zero, which implements the record-end rule;
//  * delays: the 32.32 fixed-point coefficients give, per (warp, pair), the
//    integer sample of a reference pixel and its fraction; each pixel then
//    adds A dx + B dz (|.| <= ~20 samples) in FP32, so no FP32 rounding ever
//    touches an absolute delay;
//  * floor() is a round-down add of 1.5 * 2^23 (no conversion instruction);
//    the integer lands in the mantissa and indexes the staged window;
//  * sums are two-level: per stage, then across stages (FP32).
// Index bound: with W0 = floor(min_tile s) - 1 and the staged window length
// >= span + 4 (span = (|A| + B) * 31), every read index lies in [0, win).
#include "kk_internal.h"

namespace kk {

namespace {

constexpr int kMaxStage = 32;

struct __align__(8) WarpPair {
  unsigned off;  // byte offset of entry (k_ref - W0) minus the floor magic
  float phi;     // fraction of the reference pixel's delay
};

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

__global__ void __launch_bounds__(kGatherThreads)
    k_kk_gather(const float2 *__restrict__ rf_theta, int T, const int32_t *__restrict__ bf_row,
                const long long *__restrict__ bfA, const long long *__restrict__ bfB,
                const long long *__restrict__ bfC, const float *__restrict__ bfAf,
                const float *__restrict__ bfBf, const int32_t *__restrict__ group_start, int J,
                int nx, int nz, int tiles_x, int win, int stage, int split,
                float2 *__restrict__ out, float *__restrict__ I, int compound) {
  extern __shared__ float4 sw[];  // [stage][win] staged (y, dy) entries
  __shared__ WarpPair s_wp[4][kMaxStage];
  __shared__ float2 s_ab[kMaxStage];
  __shared__ int s_w0[kMaxStage];
  __shared__ int s_row[kMaxStage];

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x;
  const int sidx = blockIdx.y;
  const int ix0 = (tile % tiles_x) * kTileX;
  const int iz0 = (tile / tiles_x) * kTileZ;
  const int ix = ix0 + lane;
  const int izb = iz0 + warp * kRowsPerThread;
  const float dl = (float)(lane - 16);

  float2 sumB[kRowsPerThread];
  float Isum[kRowsPerThread];
#pragma unroll
  for (int r = 0; r < kRowsPerThread; ++r) {
    sumB[r] = make_float2(0.f, 0.f);
    Isum[r] = 0.f;
  }

  for (int g = 0; g < J; ++g) {
    const int gb = group_start[g], ge = group_start[g + 1];
    const int n = ge - gb;
    const int pb = gb + (int)(((long long)n * sidx) / split);
    const int pe = gb + (int)(((long long)n * (sidx + 1)) / split);
    float2 acc[kRowsPerThread];
#pragma unroll
    for (int r = 0; r < kRowsPerThread; ++r) acc[r] = make_float2(0.f, 0.f);

    for (int ps = pb; ps < pe; ps += stage) {
      const int ns = min(stage, pe - ps);
      __syncthreads();  // previous stage fully consumed
      {
        const int j = tid & 31, w = tid >> 5;
        if (j < ns) {
          const int p = ps + j;
          const long long A = __ldg(bfA + p), Bq = __ldg(bfB + p), Cq = __ldg(bfC + p);
          const long long smin = Cq + Bq * (long long)iz0 + A * (long long)(A >= 0 ? ix0 : ix0 + kTileX - 1);
          const int w0 = (int)(smin >> 32) - 1;
          const long long sref = Cq + Bq * (long long)(iz0 + w * kRowsPerThread + kRowsPerThread / 2) +
                                 A * (long long)(ix0 + 16);
          const int kref = (int)(sref >> 32);
          WarpPair wp;
          wp.phi = (float)(unsigned)(sref & 0xffffffffLL) * 0x1p-32f;
          wp.off = (unsigned)(j * win + (kref - w0)) * 16u - (unsigned)kFloorMagicBits * 16u;
          s_wp[w][j] = wp;
          if (w == 0) {
            s_ab[j] = make_float2(__ldg(bfAf + p), __ldg(bfBf + p));
            s_w0[j] = w0;
            s_row[j] = __ldg(bf_row + p);
          }
        }
      }
      __syncthreads();
      // stage windows: warp w stages pairs w, w+4, ...; lanes walk the window
      for (int j = warp; j < ns; j += kGatherThreads / 32) {
        const int w0 = s_w0[j];
        const float2 *y = rf_theta + (size_t)s_row[j] * T;
        float4 *dst = sw + j * win;
        for (int m = lane; m < win; m += 32) {
          const int k = w0 + m;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if ((unsigned)k <= (unsigned)(T - 2)) {
            const float2 a = __ldg(y + k), b = __ldg(y + k + 1);
            v = make_float4(a.x, a.y, b.x - a.x, b.y - a.y);
          }
          dst[m] = v;
        }
      }
      __syncthreads();
      float2 sacc[kRowsPerThread];
#pragma unroll
      for (int r = 0; r < kRowsPerThread; ++r) sacc[r] = make_float2(0.f, 0.f);
      const char *swb = reinterpret_cast<const char *>(sw);
      for (int j = 0; j < ns; ++j) {
        const float2 ab = s_ab[j];
        const WarpPair wp = s_wp[warp][j];
        const float base = fmaf(ab.x, dl, wp.phi);
#pragma unroll
        for (int r = 0; r < kRowsPerThread; ++r) {
          const float s = fmaf(ab.y, (float)(r - kRowsPerThread / 2), base);
          const float t = __fadd_rd(s, kFloorMagic);
          const float f = s - (t - kFloorMagic);
          const unsigned addr = wp.off + ((unsigned)__float_as_int(t) << 4);
          const float4 e = *reinterpret_cast<const float4 *>(swb + addr);
          sacc[r].x += fmaf(f, e.z, e.x);
          sacc[r].y += fmaf(f, e.w, e.y);
        }
      }
#pragma unroll
      for (int r = 0; r < kRowsPerThread; ++r) acc[r] = f2add(acc[r], sacc[r]);
    }
    // group finished: write B_j (or this slice's partial of it)
    float2 *dst = out + ((size_t)sidx * J + g) * (size_t)nx * nz;
#pragma unroll
    for (int r = 0; r < kRowsPerThread; ++r) {
      const int iz = izb + r;
      if (ix < nx && iz < nz) dst[(size_t)iz * nx + ix] = acc[r];
      sumB[r] = f2add(sumB[r], acc[r]);
      Isum[r] = fmaf(acc[r].x, acc[r].x, fmaf(acc[r].y, acc[r].y, Isum[r]));
    }
  }
  if (split == 1 && I != nullptr && compound != KK_COMPOUND_NONE) {
#pragma unroll
    for (int r = 0; r < kRowsPerThread; ++r) {
      const int iz = izb + r;
      if (ix < nx && iz < nz) {
        const float v = (compound == KK_COMPOUND_COHERENT)
                            ? fmaf(sumB[r].x, sumB[r].x, sumB[r].y * sumB[r].y)
                            : Isum[r];
        I[(size_t)iz * nx + ix] = v;
      }
    }
  }
}

// Sum the pair-slice partials in slice order and compound.
__global__ void k_kk_reduce(const float2 *__restrict__ part, int split, int J, int npix,
                            float2 *__restrict__ B, float *__restrict__ I, int compound) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= npix) return;
  float2 sb = make_float2(0.f, 0.f);
  float si = 0.f;
  for (int g = 0; g < J; ++g) {
    float2 a = make_float2(0.f, 0.f);
    for (int s = 0; s < split; ++s) a = f2add(a, part[((size_t)s * J + g) * npix + q]);
    B[(size_t)g * npix + q] = a;
    sb = f2add(sb, a);
    si = fmaf(a.x, a.x, fmaf(a.y, a.y, si));
  }
  if (I != nullptr && compound != KK_COMPOUND_NONE)
    I[q] = (compound == KK_COMPOUND_COHERENT) ? fmaf(sb.x, sb.x, sb.y * sb.y) : si;
}

}  // namespace

cudaError_t launch_kk_gather(const kk_plan &p, const float2 *rf_theta, float2 *B, float *I,
                             float2 *partial, cudaStream_t s) {
  const size_t smem = sizeof(float4) * (size_t)p.bf_stage * p.bf_win;
  cudaFuncSetAttribute(k_kk_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const dim3 grid(p.tiles_x * p.tiles_z, p.bf_split);
  float2 *dst = (p.bf_split > 1) ? partial : B;
  k_kk_gather<<<grid, kGatherThreads, smem, s>>>(
      rf_theta, p.T, p.t.bf_row, p.t.bf_A, p.t.bf_B, p.t.bf_C, p.t.bf_Af, p.t.bf_Bf,
      p.t.group_start, p.J, p.grid.nx, p.grid.nz, p.tiles_x, p.bf_win, p.bf_stage, p.bf_split, dst,
      I, p.compound);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || p.bf_split == 1) return e;
  const int npix = p.grid.nx * p.grid.nz;
  k_kk_reduce<<<(npix + 255) / 256, 256, 0, s>>>(partial, p.bf_split, p.J, npix, B, I, p.compound);
  return cudaGetLastError();
}

}  // namespace kk
