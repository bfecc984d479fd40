// das_beamform.cu -- CPWC delay-and-sum reference, Eq. (DAS).
//
//   B(ix, iz) = sum_{i,l} a_l(ix, iz) lerp(y_il, s_in(i; ix, iz) + R_l(ix, iz)),
//   a_l = receive-aperture weight (1 for the full aperture), applied once
//   per (pixel, element, stage) to the stage's partial sum,
//   s_in = fs (x sin theta_i + z cos theta_i) / c     (affine, 32.32 fixed point)
//   R_l  = fs sqrt((x - u_l)^2 + z^2) / c              (per pixel and element)
//
// Same tile, staging and floor scheme as the KK gather.  The receive delay
// R_l is not affine, so it is computed once per (pixel, element) in
// double-float arithmetic (FP32 hi + lo words; square root with one Newton
// correction), split into an integer and a fraction, and reused across all
// transmit angles: the transmit loop is the inner loop, so this costs
// ~30 FP32 operations per pixel per element against N gathers.
// Index bound: W0 = floor(min s_in) + floor(min R) - 2 over the tile and the
// staged window length >= span_in + span_out + 6 keep every read in [0, win).
//
// Two kernels:
//  * k_das_gather_staged (windows of up to 256 entries, i.e. pixels up to
//    about 0.3 mm at 20 MHz): 32 x 16 tiles, 4 warps of 4 rows; channels
//    (i, l) in stages of 4-16 transmits of one element; the raw samples of
//    stage s+1 are loaded into registers while stage s is gathered (as in the
//    KK gather), the per-channel tables are double-buffered, and the receive
//    delay of the thread's pixels is recomputed only when the element
//    changes;
//  * k_das_gather (any window): 32 x 32 tiles, synchronous staging.
#include "kk_internal.h"

namespace kk {

namespace {

constexpr int kMaxStage = 32;

#ifdef KK_DEBUG_BOUNDS
// failed staged-window index checks of this file's gathers
static __device__ unsigned g_bounds_das = 0;
#endif

struct __align__(8) WarpChan {
  unsigned off;
  float phi;
};

__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return make_float2(s, e);
}

// (a_hi + a_lo) - (b_hi + b_lo)
__device__ __forceinline__ float2 df_sub(float2 a, float2 b) {
  float2 s = two_sum(a.x, -b.x);
  s.y += a.y - b.y;
  const float h = s.x + s.y;
  return make_float2(h, s.y - (h - s.x));
}

// (h + l)^2 as double-float
__device__ __forceinline__ float2 df_sqr(float2 a) {
  const float p = a.x * a.x;
  float e = fmaf(a.x, a.x, -p);
  e = fmaf(2.f * a.x, a.y, e);
  return make_float2(p, e);
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float2 s = two_sum(a.x, b.x);
  s.y += a.y + b.y;
  const float h = s.x + s.y;
  return make_float2(h, s.y - (h - s.x));
}

// Receive-aperture weight of an element at lateral offset d (samples) from a
// pixel at depth z (samples): t = 2 F d / z, boxcar 1 for t <= 1, Hann
// (1 + cos(pi t)) / 2 for t <= 1, 0 beyond; two_f = 0 is the full aperture.
__device__ __forceinline__ float aperture_weight(float d, float z, float two_f, int window) {
  if (two_f <= 0.f) return 1.f;
  const float t = two_f * d / z;
  if (!(t <= 1.f)) return 0.f;
  return window == KK_APERTURE_HANN ? 0.5f * (1.f + cospif(t)) : 1.f;
}

__global__ void __launch_bounds__(kGatherThreads)
    k_das_gather(const float2 *__restrict__ y, int N, int L, int T, const long long *__restrict__ dA,
                 const long long *__restrict__ dB, const long long *__restrict__ dC,
                 const float *__restrict__ dAf, const float *__restrict__ dBf,
                 const float2 *__restrict__ xs, const float2 *__restrict__ zs,
                 const float2 *__restrict__ us, int nx, int nz, int tiles_x, int win, int stage,
                 int split, float two_f, int window, float2 *__restrict__ B, float *__restrict__ I) {
  extern __shared__ float4 sw[];
  __shared__ WarpChan s_wc[4][kMaxStage];
  __shared__ float2 s_ab[kMaxStage];
  __shared__ int s_w0[kMaxStage];
  __shared__ int s_row[kMaxStage];

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x;
  const int ix0 = (tile % tiles_x) * kTileX;
  const int iz0 = (tile / tiles_x) * kTileZ;
  const int ix = ix0 + lane;
  const int izb = iz0 + warp * kRowsPerThread;
  const float dl = (float)(lane - 16);

  const float2 xq = __ldg(xs + ix);
  float2 z2[kRowsPerThread];
#pragma unroll
  for (int r = 0; r < kRowsPerThread; ++r) z2[r] = df_sqr(__ldg(zs + izb + r));
  const float xlo = __ldg(xs + ix0).x, xhi = __ldg(xs + ix0 + kTileX - 1).x;
  const float zlo = __ldg(zs + iz0).x;

  float2 acc[kRowsPerThread];
#pragma unroll
  for (int r = 0; r < kRowsPerThread; ++r) acc[r] = make_float2(0.f, 0.f);

  const int sidx = blockIdx.y;
  const int lb = (int)(((long long)L * sidx) / split), le = (int)(((long long)L * (sidx + 1)) / split);
  for (int l = lb; l < le; ++l) {
    const float2 u = __ldg(us + l);
    // receive delay of this thread's pixels: integer part (x16 bytes) + fraction
    const float2 dx2 = df_sqr(df_sub(xq, u));
    unsigned kout16[kRowsPerThread];
    float fout[kRowsPerThread], aw[kRowsPerThread];
#pragma unroll
    for (int r = 0; r < kRowsPerThread; ++r) {
      aw[r] = aperture_weight(fabsf(xq.x - u.x), __ldg(zs + izb + r).x, two_f, window);
      const float2 S = df_add(dx2, z2[r]);
      const float rh = sqrtf(S.x);
      const float t = fmaf(-rh, rh, S.x) + S.y;
      const float corr = (rh > 0.f) ? t / (2.f * rh) : 0.f;
      const float kf = floorf(rh);
      kout16[r] = (unsigned)(int)kf * 16u;
      fout[r] = (rh - kf) + corr;
    }
    // smallest receive delay over the tile (lower bound for the window)
    const float xc = fminf(fmaxf(u.x, xlo), xhi) - u.x;
    const int kout_min = (int)floorf(sqrtf(fmaf(xc, xc, zlo * zlo)));

    for (int ps = 0; ps < N; ps += stage) {
      const int ns = min(stage, N - ps);
      __syncthreads();
      {
        const int j = tid & 31, w = tid >> 5;
        if (j < ns) {
          const int i = ps + j;
          const long long A = __ldg(dA + i), Bq = __ldg(dB + i), Cq = __ldg(dC + i);
          const long long smin = Cq + Bq * (long long)iz0 + A * (long long)(A >= 0 ? ix0 : ix0 + kTileX - 1);
          const int w0 = (int)(smin >> 32) + kout_min - 2;
          const long long sref = Cq + Bq * (long long)(iz0 + w * kRowsPerThread + kRowsPerThread / 2) +
                                 A * (long long)(ix0 + 16);
          const int kref = (int)(sref >> 32);
          WarpChan wc;
          wc.phi = (float)(unsigned)(sref & 0xffffffffLL) * 0x1p-32f;
          wc.off = (unsigned)(j * win + (kref - w0)) * 16u - (unsigned)kFloorMagicBits * 16u;
          s_wc[w][j] = wc;
          if (w == 0) {
            s_ab[j] = make_float2(__ldg(dAf + i), __ldg(dBf + i));
            s_w0[j] = w0;
            s_row[j] = i * L + l;
          }
        }
      }
      __syncthreads();
      for (int j = warp; j < ns; j += kGatherThreads / 32) {
        const int w0 = s_w0[j];
        const float2 *yr = y + (size_t)s_row[j] * T;
        float4 *dst = sw + j * win;
        for (int m = lane; m < win; m += 32) {
          const int k = w0 + m;
          float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
          if ((unsigned)k <= (unsigned)(T - 2)) {
            const float2 a = __ldg(yr + k), b = __ldg(yr + k + 1);
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
        const WarpChan wc = s_wc[warp][j];
        const float base = fmaf(ab.x, dl, wc.phi);
#pragma unroll
        for (int r = 0; r < kRowsPerThread; ++r) {
          const float s = fmaf(ab.y, (float)(r - kRowsPerThread / 2), base) + fout[r];
          const float t = __fadd_rd(s, kFloorMagic);
          const float f = s - (t - kFloorMagic);
          const unsigned addr = wc.off + kout16[r] + ((unsigned)__float_as_int(t) << 4);
          float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
          if (KK_IN_BOUNDS(g_bounds_das, (unsigned)((int)(addr >> 4) - j * win) < (unsigned)win))
            e = *reinterpret_cast<const float4 *>(swb + addr);
          sacc[r].x += fmaf(f, e.z, e.x);
          sacc[r].y += fmaf(f, e.w, e.y);
        }
      }
#pragma unroll
      for (int r = 0; r < kRowsPerThread; ++r) {
        acc[r].x = fmaf(aw[r], sacc[r].x, acc[r].x);
        acc[r].y = fmaf(aw[r], sacc[r].y, acc[r].y);
      }
    }
  }
  // split == 1: final image; otherwise this element slice's partial image
  float2 *dst = B + (size_t)sidx * nx * nz;
#pragma unroll
  for (int r = 0; r < kRowsPerThread; ++r) {
    const int iz = izb + r;
    if (ix < nx && iz < nz) {
      dst[(size_t)iz * nx + ix] = acc[r];
      if (split == 1 && I != nullptr) I[(size_t)iz * nx + ix] = fmaf(acc[r].x, acc[r].x, acc[r].y * acc[r].y);
    }
  }
}

// Per-slice terms of the volumetric (2D-array) form: the transmit delay's
// step per y slice (32.32 samples per slice, per transmit), the slices' y
// and the elements' y (fs / c units, as (hi, lo)), and the xz tiles per slice.
struct DasVolArgs {
  const long long *dY;
  const float2 *ys, *us_y;
  int ny, tiles_xz;
};

// Staged-window DAS gather for windows of at most 256 entries (see above).
// Entries E[k] = (y[k], y[k+1] - y[k]) (zero outside [0, T-2]): one 16-byte
// load and two FMAs per pixel-pair.  VOL: 2D array over a volume; the block
// index also runs over y slices, each tile lies in one slice (an [nz][nx]
// plane of the [ny][nz][nx] image), the transmit delay gains dY * slice and
// the receive distance the squared y offset of slice and element.
template <int STAGE, int NPT, int MINB, bool VOL = false>
__global__ void __launch_bounds__(kGatherThreads, MINB)
    k_das_gather_staged(const float2 *__restrict__ y, int N, int L, int T, const long long *__restrict__ dA,
                        const long long *__restrict__ dB, const long long *__restrict__ dC,
                        const float *__restrict__ dAf, const float *__restrict__ dBf,
                        const float2 *__restrict__ xs, const float2 *__restrict__ zs,
                        const float2 *__restrict__ us, int nx, int nz, int tiles_x, int win, int split,
                        float two_f, int window, float2 *__restrict__ B, float *__restrict__ I,
                        const DasVolArgs va) {
  constexpr int ROWS = 4, TZ = 16;
  constexpr int PPW = STAGE / 4;   // channels staged by each warp
  constexpr int QPP = NPT / PPW;   // entries per lane per staged channel
  static_assert(QPP * PPW == NPT && STAGE % 4 == 0 && STAGE <= 32, "stage shape");
  extern __shared__ float4 sw[];   // [STAGE][win]
  __shared__ WarpChan s_wc[2][4][STAGE];
  __shared__ float2 s_ab[2][STAGE];
  __shared__ int s_w0[2][STAGE];
  __shared__ int s_row[2][STAGE];

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  int tile = blockIdx.x;
  [[maybe_unused]] int slice = 0;
  size_t plane = (size_t)nx * nz;  // one image (all slices) per pair slice of the split
  if constexpr (VOL) {
    slice = tile / va.tiles_xz;
    tile -= slice * va.tiles_xz;
    plane *= (size_t)va.ny;
    B += (size_t)slice * nx * nz;
    if (I != nullptr) I += (size_t)slice * nx * nz;
  }
  const int ix0 = (tile % tiles_x) * kTileX;
  const int iz0 = (tile / tiles_x) * TZ;
  const int ix = ix0 + lane;
  const int izb = iz0 + warp * ROWS;
  const float dl = (float)(lane - 16);
  const float2 xq = __ldg(xs + ix);
  float2 z2[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) z2[r] = df_sqr(__ldg(zs + izb + r));
  const float xlo = __ldg(xs + ix0).x, xhi = __ldg(xs + ix0 + kTileX - 1).x;
  const float zlo = __ldg(zs + iz0).x;
  [[maybe_unused]] float2 ysl = make_float2(0.f, 0.f);  // this slice's y (fs / c units)
  if constexpr (VOL) ysl = __ldg(va.ys + slice);

  float2 acc[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) acc[r] = make_float2(0.f, 0.f);

  const int sidx = blockIdx.y;
  const int lb = (int)(((long long)L * sidx) / split), le = (int)(((long long)L * (sidx + 1)) / split);
  const int spl = (N + STAGE - 1) / STAGE;  // stages per element
  const int nq = (le - lb) * spl;

  // tables of stage q into buffer b_: transmits ps.. of element l
#define DAS_TABLES(Q, B_)                                                                             \
  {                                                                                                   \
    const int l_ = lb + (Q) / spl, ps_ = ((Q) % spl) * STAGE, ns_ = min(STAGE, N - ps_);             \
    if (lane < ns_) {                                                                                 \
      const float2 u_ = __ldg(us + l_);                                                               \
      const float xc_ = fminf(fmaxf(u_.x, xlo), xhi) - u_.x;                                          \
      float r2_ = fmaf(xc_, xc_, zlo * zlo);                                                          \
      if constexpr (VOL) {                                                                            \
        const float yc_ = ysl.x - __ldg(va.us_y + l_).x;                                              \
        r2_ = fmaf(yc_, yc_, r2_);                                                                    \
      }                                                                                               \
      const int kmin_ = (int)floorf(sqrtf(r2_));                                                      \
      const int i_ = ps_ + lane;                                                                      \
      const long long A_ = __ldg(dA + i_), Bq_ = __ldg(dB + i_);                                      \
      const long long Cq_ = __ldg(dC + i_) + (VOL ? __ldg(va.dY + i_) * (long long)slice : 0LL);      \
      const long long smin_ = Cq_ + Bq_ * (long long)iz0 + A_ * (long long)(A_ >= 0 ? ix0 : ix0 + kTileX - 1); \
      const int w0_ = (int)(smin_ >> 32) + kmin_ - 2;                                                 \
      const long long sref_ = Cq_ + Bq_ * (long long)(iz0 + warp * ROWS + ROWS / 2) + A_ * (long long)(ix0 + 16); \
      const int kref_ = (int)(sref_ >> 32);                                                           \
      WarpChan wc_;                                                                                   \
      wc_.phi = (float)(unsigned)(sref_ & 0xffffffffLL) * 0x1p-32f;                                   \
      wc_.off = (unsigned)(lane * win + (kref_ - w0_)) * 16u - (unsigned)kFloorMagicBits * 16u;       \
      s_wc[B_][warp][lane] = wc_;                                                                     \
      if (warp == 0) {                                                                                \
        s_ab[B_][lane] = make_float2(__ldg(dAf + i_), __ldg(dBf + i_));                                \
        s_w0[B_][lane] = w0_;                                                                         \
        s_row[B_][lane] = i_ * L + l_;                                                                \
      }                                                                                               \
    }                                                                                                 \
  }
  // raw samples of stage q (tables in buffer b_) into registers
#define DAS_LOAD_RAW(Q, B_)                                                                          \
  {                                                                                                  \
    const int ns_ = min(STAGE, N - ((Q) % spl) * STAGE);                                             \
    _Pragma("unroll") for (int u = 0; u < PPW; ++u) {                                                \
      const int j = warp + 4 * u;                                                                    \
      const int jj = j < ns_ ? j : 0;                                                                \
      const float2 *yr = y + (size_t)s_row[B_][jj] * T;                                              \
      const int w0 = s_w0[B_][jj];                                                                   \
      _Pragma("unroll") for (int i = 0; i < QPP; ++i) {                                              \
        const int m = lane + 32 * i;                                                                 \
        const int k = w0 + m;                                                                        \
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);                                 \
        if (j < ns_ && m < win && (unsigned)k <= (unsigned)(T - 2)) {                                \
          a = __ldg(yr + k);                                                                         \
          b = __ldg(yr + k + 1);                                                                     \
        }                                                                                            \
        raw0[u * QPP + i] = a;                                                                       \
        raw1[u * QPP + i] = b;                                                                       \
      }                                                                                              \
    }                                                                                                \
  }

  float2 raw0[NPT], raw1[NPT];
  int buf = 0;
  if (nq > 0) {
    DAS_TABLES(0, 0);
    __syncthreads();
    DAS_LOAD_RAW(0, 0);
  }
  int cur_l = -1;
  float fo[ROWS];     // receive delay of this thread's pixels minus kl16 / 16
  unsigned kl16 = 0;  // integer receive delay of the thread's first row, x 16 bytes
  const char *swb = reinterpret_cast<const char *>(sw);
  for (int q = 0; q < nq; ++q) {
    const int l = lb + q / spl;
    const int ns = min(STAGE, N - (q % spl) * STAGE);
    __syncthreads();  // everyone is done gathering from sw
#pragma unroll
    for (int u = 0; u < PPW; ++u) {
      const int j = warp + 4 * u;
#pragma unroll
      for (int i = 0; i < QPP; ++i) {
        const int m = lane + 32 * i;
        if (j < ns && m < win) {
          const float2 a = raw0[u * QPP + i], b = raw1[u * QPP + i];
          sw[(size_t)j * win + m] = make_float4(a.x, a.y, b.x - a.x, b.y - a.y);
        }
      }
    }
    if (q + 1 < nq) DAS_TABLES(q + 1, buf ^ 1);
    __syncthreads();  // entries of this stage and tables of the next visible
    if (q + 1 < nq) DAS_LOAD_RAW(q + 1, buf ^ 1);  // in flight during the gathers
    if (l != cur_l) {
      // receive delay of this thread's pixels for element l: the integer
      // delay of its first row (kl, folded into the per-channel offset, so a
      // lerp adds no integer) plus a small remainder per row (integer part
      // exact, fraction from the double-float root)
      cur_l = l;
      const float2 u = __ldg(us + l);
      float2 dx2 = df_sqr(df_sub(xq, u));
      if constexpr (VOL) dx2 = df_add(dx2, df_sqr(df_sub(ysl, __ldg(va.us_y + l))));
      int kl = 0;
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const float2 S = df_add(dx2, z2[r]);
        const float rh = sqrtf(S.x);
        const float t = fmaf(-rh, rh, S.x) + S.y;
        const float corr = (rh > 0.f) ? t / (2.f * rh) : 0.f;
        const float kf = floorf(rh);
        if (r == 0) kl = (int)kf;
        fo[r] = (float)((int)kf - kl) + ((rh - kf) + corr);
      }
      kl16 = (unsigned)kl * 16u;
    }
    float2 sacc[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) sacc[r] = make_float2(0.f, 0.f);
    // two rows per packed (f32x2) instruction: the scalar form's IEEE
    // operations in the same order, at half the issue slots
    const float2 magic2 = make_float2(kFloorMagic, kFloorMagic);
    const float2 nmagic2 = make_float2(-kFloorMagic, -kFloorMagic);
    const float2 neg1 = make_float2(-1.f, -1.f);
#pragma unroll 2
    for (int j = 0; j < ns; ++j) {
      const float2 ab = s_ab[buf][j];
      const WarpChan wc = s_wc[buf][warp][j];
      const float base = fmaf(ab.x, dl, wc.phi);
      const unsigned offl = wc.off + kl16;
      const float2 b2 = make_float2(ab.y, ab.y), base2 = make_float2(base, base);
#pragma unroll
      for (int r = 0; r < ROWS; r += 2) {
        const float2 s = __fadd2_rn(
            __ffma2_rn(b2, make_float2((float)(r - ROWS / 2), (float)(r + 1 - ROWS / 2)), base2),
            make_float2(fo[r], fo[r + 1]));
        const float2 t = __fadd2_rd(s, magic2);                        // floor in the mantissa
        const float2 f = __ffma2_rn(__fadd2_rn(t, nmagic2), neg1, s);  // s - floor(s)
        const unsigned addr0 = offl + ((unsigned)__float_as_int(t.x) << 4);
        const unsigned addr1 = offl + ((unsigned)__float_as_int(t.y) << 4);
        float4 e0 = make_float4(0.f, 0.f, 0.f, 0.f), e1 = e0;
        if (KK_IN_BOUNDS(g_bounds_das, (unsigned)((int)(addr0 >> 4) - j * win) < (unsigned)win))
          e0 = *reinterpret_cast<const float4 *>(swb + addr0);
        if (KK_IN_BOUNDS(g_bounds_das, (unsigned)((int)(addr1 >> 4) - j * win) < (unsigned)win))
          e1 = *reinterpret_cast<const float4 *>(swb + addr1);
        sacc[r] = __fadd2_rn(sacc[r], __ffma2_rn(make_float2(f.x, f.x), make_float2(e0.z, e0.w),
                                                 make_float2(e0.x, e0.y)));
        sacc[r + 1] = __fadd2_rn(sacc[r + 1], __ffma2_rn(make_float2(f.y, f.y), make_float2(e1.z, e1.w),
                                                         make_float2(e1.x, e1.y)));
      }
    }
    if (two_f > 0.f) {
      // receive-aperture weight of element l at this thread's pixels
      const float d = fabsf(xq.x - __ldg(us + l).x);
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const float aw = aperture_weight(d, __ldg(zs + izb + r).x, two_f, window);
        acc[r].x = fmaf(aw, sacc[r].x, acc[r].x);
        acc[r].y = fmaf(aw, sacc[r].y, acc[r].y);
      }
    } else {
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        acc[r].x += sacc[r].x;
        acc[r].y += sacc[r].y;
      }
    }
    buf ^= 1;
  }
#undef DAS_TABLES
#undef DAS_LOAD_RAW
  float2 *dst = B + (size_t)sidx * plane;
#pragma unroll
  for (int r = 0; r < ROWS; ++r) {
    const int iz = izb + r;
    if (ix < nx && iz < nz) {
      dst[(size_t)iz * nx + ix] = acc[r];
      if (split == 1 && I != nullptr) I[(size_t)iz * nx + ix] = fmaf(acc[r].x, acc[r].x, acc[r].y * acc[r].y);
    }
  }
}

// Sum element-slice partials in slice order.
__global__ void k_das_reduce(const float2 *__restrict__ part, int split, int npix,
                             float2 *__restrict__ B, float *__restrict__ I) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= npix) return;
  float2 a = make_float2(0.f, 0.f);
  for (int s = 0; s < split; ++s) {
    const float2 v = part[(size_t)s * npix + q];
    a.x += v.x;
    a.y += v.y;
  }
  B[q] = a;
  if (I != nullptr) I[q] = fmaf(a.x, a.x, a.y * a.y);
}

}  // namespace

namespace {
template <int STAGE, int NPT>
cudaError_t launch_staged(const kk_plan &p, const float2 *y, float2 *dst, float *I, cudaStream_t s) {
  constexpr int MINB = 7;
  const size_t smem = sizeof(float4) * (size_t)STAGE * p.bf_win;
  // volumetric plans: the slice terms cost registers, one CTA per SM fewer
  auto k = p.vol ? k_das_gather_staged<STAGE, NPT, MINB - 1, true> : k_das_gather_staged<STAGE, NPT, MINB, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  DasVolArgs va{p.t.das_Y, p.t.ys, p.t.us_y, p.ny, p.tiles_x * p.tiles_z};
  const dim3 grid(p.tiles_x * p.tiles_z * p.ny, p.bf_split);
  k<<<grid, kGatherThreads, smem, s>>>(y, p.N, p.L, p.T, p.t.das_A, p.t.das_B, p.t.das_C, p.t.das_Af,
                                       p.t.das_Bf, p.t.xs, p.t.zs, p.t.us, p.grid.nx, p.grid.nz, p.tiles_x,
                                       p.bf_win, p.bf_split, p.das_two_f, p.das_window, dst, I, va);
  return cudaGetLastError();
}
}  // namespace

// launch shape of the staged DAS gather for a window: stage 16 / 8 / 4
// transmits with 2 / 4 / 8 staged entries per lane and channel; 0 when the
// window is wider than 256 entries (the synchronous kernel takes it)
int das_staged_stage(int win) {
  const int q = gather_entries_per_lane(win);
  if (q == 1 || q == 2) return 16;
  if (q == 4) return 8;
  if (q == 8) return 4;
  return 0;
}

#ifdef KK_DEBUG_BOUNDS
cudaError_t take_bounds_das(unsigned long long *n) {
  unsigned v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_bounds_das, sizeof(v));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bounds_das, &zero, sizeof(zero));
  *n = v;
  return e;
}
#endif

cudaError_t launch_das_gather(const kk_plan &p, const float2 *y, float2 *B, float *I,
                              float2 *partial, cudaStream_t s) {
  float2 *dst = p.bf_split > 1 ? partial : B;
  cudaError_t e;
  if (p.bf_rows == 4) {
    const int q = gather_entries_per_lane(p.bf_win);
    switch (p.bf_stage) {
      case 16: e = q == 1 ? launch_staged<16, 4>(p, y, dst, I, s) : launch_staged<16, 8>(p, y, dst, I, s); break;
      case 8: e = launch_staged<8, 8>(p, y, dst, I, s); break;
      case 4: e = launch_staged<4, 8>(p, y, dst, I, s); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    if (p.vol) return cudaErrorInvalidConfiguration;  // the plan refuses such volumes
    const size_t smem = sizeof(float4) * (size_t)p.bf_stage * p.bf_win;
    cudaFuncSetAttribute(k_das_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const dim3 grid(p.tiles_x * p.tiles_z, p.bf_split);
    k_das_gather<<<grid, kGatherThreads, smem, s>>>(
        y, p.N, p.L, p.T, p.t.das_A, p.t.das_B, p.t.das_C, p.t.das_Af, p.t.das_Bf, p.t.xs, p.t.zs,
        p.t.us, p.grid.nx, p.grid.nz, p.tiles_x, p.bf_win, p.bf_stage, p.bf_split, p.das_two_f,
        p.das_window, dst, I);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess || p.bf_split == 1) return e;
  const int npix = p.grid.nx * p.grid.nz * p.ny;
  k_das_reduce<<<(npix + 255) / 256, 256, 0, s>>>(partial, p.bf_split, npix, B, I);
  return cudaGetLastError();
}

}  // namespace kk
