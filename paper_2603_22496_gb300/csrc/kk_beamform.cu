// kk_beamform.cu -- KK image formation, Eq. (KK), with compounding.
//
//   B_j(ix, iz) = sum_{p in group j} lerp(y_p, s_p(ix, iz)),
//   s_p(ix, iz) = A_p ix + B_p iz + C_p   (samples; affine because both the
//   transmit delay s_i.r/c and the receive delay s_o.r/c are linear in r,
//   Section II-F's LUT decomposition taken to its limit).
//
// Design (gather-bound; tensor cores do not apply):
//  * one CTA per 32 x (4 ROWS) pixel tile (and per slice of the pair list
//    when the grid has too few tiles to fill the GPU); 4 warps, lane = x
//    offset, ROWS z rows per thread;
//  * pairs are processed in stages of STAGE pairs: for each pair the CTA
//    stages the window of y_p its tile can touch into shared memory as
//    16-byte entries E[k] = (y[k], y[k+1] - y[k]), so one load and two FMAs
//    give a linear interpolation y[k] + f (y[k+1] - y[k]); E[k] = 0 outside
//    k in [0, T-2], which implements the record-end rule exactly;
//  * staging goes through registers: lane m of a warp reads y[k] and y[k+1]
//    and writes E[k], so a warp's 16-byte stores are contiguous (no bank
//    conflicts); the loads of stage s+1 are issued before the gathers of
//    stage s, so their latency hides behind the gathers;
//  * delays: the 32.32 fixed-point coefficients give, per (warp, pair), the
//    integer sample of a reference pixel and its fraction; each pixel then
//    adds A dx + B dz (|.| <= ~20 samples) in FP32, so no FP32 rounding ever
//    touches an absolute delay;
//  * floor() is a round-down add of 1.5 * 2^23 (no conversion instruction);
//    the integer lands in the mantissa and indexes the staged window;
//  * sums are two-level: per stage, then across stages (FP32).
// Index bound: with W0 = floor(min_tile s) - 1 and a staged window of
// win >= span + 4 entries (span = |A| 31 + B (TZ - 1)), every read index lies
// in [0, win).
#include <type_traits>

#include "kk_internal.h"

namespace kk {

namespace {

// Everything a warp needs for one pair, read with one broadcast 16-byte load.
struct __align__(16) WarpPair {
  float a, b;    // delay slopes along x and z (samples per pixel)
  float phi;     // fraction of the warp's reference pixel delay
  unsigned off;  // byte offset of entry (k_ref - W0) minus the floor magic
};

struct __align__(8) PairSrc {
  int w0;   // first staged sample
  int row;  // row of rf_theta
};

// Per-pair inputs of the delay tables, copied asynchronously one stage ahead.
struct __align__(8) PairIn {
  long long A, B, C;  // 32.32 fixed-point delay coefficients
  float af, bf;       // FP32 slopes
  int row;
  int pad;
};

// volumetric plans: also the 32.32 delay per y slice
struct __align__(8) PairInVol : PairIn {
  long long Y;
};

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

#ifdef KK_DEBUG_BOUNDS
// failed staged-window index checks of this file's gathers
static __device__ unsigned g_bounds_kk = 0;
#endif

// Per-pair state of the delay tables, double-buffered by stage.
template <int STAGE, bool VOL = false>
struct GatherSmem {
  WarpPair wp[2][4][STAGE];
  PairSrc src[2][STAGE];
  typename std::conditional<VOL, PairInVol, PairIn>::type in[2][STAGE];
};

// One tile (and pair slice) of KK image formation; shared by the per-plan
// kernel and the batched persistent kernel.  VOL: the tile index also runs
// over y slices (slice = tile / tiles_xz); every delay gains the pair's
// per-slice term Y * slice, and the slice is one [nz][nx] plane of the
// [J][ny][nz][nx] output (of the [ny][nz][nx] intensity).
template <int ROWS, int STAGE, int NPT, bool MULTI, bool VOL = false>
__device__ __forceinline__ void gather_tile(const GatherArgs &a, int tile, int sidx, float4 *sw,
                                            GatherSmem<STAGE, VOL> &sm,
                                            const GatherVolArgs *va = nullptr) {
  const float2 *__restrict__ rf_theta = a.rf_theta;
  const int T = a.T;
  const int32_t *__restrict__ bf_row = a.bf_row;
  const long long *__restrict__ bfA = a.bfA;
  const long long *__restrict__ bfB = a.bfB;
  const long long *__restrict__ bfC = a.bfC;
  const float *__restrict__ bfAf = a.bfAf;
  const float *__restrict__ bfBf = a.bfBf;
  const int32_t *__restrict__ group_start = a.group_start;
  const int J = a.J, nx = a.nx, nz = a.nz, tiles_x = a.tiles_x, win = a.win, split = a.split;
  float2 *__restrict__ out = a.out;
  float *__restrict__ I = a.I;
  const int compound = a.compound;
  // volumetric plans: slice of this tile and its per-pair delay term
  [[maybe_unused]] long long vol_slice = 0;
  if constexpr (VOL) {
    const int sl = tile / va->tiles_xz;
    tile -= sl * va->tiles_xz;
    vol_slice = sl;
    out += (size_t)sl * nx * nz;          // plane `sl` of each [ny][nz][nx] image
    if (I != nullptr) I += (size_t)sl * nx * nz;
  }
  auto &s_wp = sm.wp;
  auto &s_src = sm.src;
  auto &s_in = sm.in;
  static_assert(STAGE <= 32 && STAGE % 4 == 0, "one table thread per (pair, warp)");
  static_assert(ROWS % 2 == 0, "rows are processed in packed pairs");
  static_assert(NPT <= kMaxStagedEntries, "staged entries held in registers");
  constexpr int TZ = 4 * ROWS;
  constexpr int PPW = STAGE / 4;          // pairs staged by each warp
  constexpr int QPP = NPT / PPW;          // entries per lane per staged pair
  static_assert(QPP * PPW == NPT, "NPT must be a multiple of STAGE / 4");
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tj = tid & 31, tw = tid >> 5;  // table thread: pair tj, warp reference tw
  const int ix0 = (tile % tiles_x) * kTileX;
  const int iz0 = (tile / tiles_x) * TZ;
  const int ix = ix0 + lane;
  const int izb = iz0 + warp * ROWS;
  const float dl = (float)(lane - 16);

  // ---- stage schedule: groups in order, this CTA's slice of each group ----
  int g = 0, pe = 0, ps = 0;
  auto enter_group = [&](int gg) {
    for (g = gg; g < J; ++g) {
      const int gb = group_start[g];
      const unsigned n = (unsigned)(group_start[g + 1] - gb);
      ps = gb + (int)((n * (unsigned)sidx) / (unsigned)split);
      pe = gb + (int)((n * (unsigned)(sidx + 1)) / (unsigned)split);
      if (pe > ps) return;
    }
  };

  // image accumulators (with several groups, each group's image is written
  // out when the group ends; the compounded intensity reads them back at the
  // end, so no running compound state is held through the pair loop)
  float2 acc[ROWS];
#pragma unroll
  for (int r = 0; r < ROWS; ++r) acc[r] = make_float2(0.f, 0.f);
  int gw = 0;  // next group whose image is written

  float2 raw0[NPT], raw1[NPT];  // y[k], y[k+1] of this lane's staged entries

  enter_group(0);
  int cur_g = g, cur_p = ps, cur_n = (g < J) ? min(STAGE, pe - ps) : 0;
  int nxt_g = J, nxt_p = 0, nxt_n = 0;
  int buf = 0;

  // per-pair inputs of a stage (NS pairs from P0) into s_in[B_], asynchronously
#define KK_FETCH(P0, NS, B_)                           \
  if (tw == 0 && tj < (NS)) {                          \
    const int p_ = (P0) + tj;                          \
    auto *d_ = &s_in[B_][tj];                          \
    cp_async8(&d_->A, bfA + p_);                       \
    cp_async8(&d_->B, bfB + p_);                       \
    cp_async8(&d_->C, bfC + p_);                       \
    if constexpr (VOL) cp_async8(&d_->Y, va->bfY + p_); \
    cp_async4(&d_->af, bfAf + p_);                     \
    cp_async4(&d_->bf, bfBf + p_);                     \
    cp_async4(&d_->row, bf_row + p_);                  \
  }                                                    \
  cp_async_commit();
  // tables of a stage (NS pairs, inputs in s_in[B_]) into buffer B_
#define KK_TABLES(NS, B_)                                                                        \
  if (tj < (NS)) {                                                                               \
    auto in = s_in[B_][tj];                                                                      \
    if constexpr (VOL) in.C += in.Y * vol_slice;                                                 \
    const long long smin = in.C + in.B * (long long)iz0 +                                        \
                           in.A * (long long)(in.A >= 0 ? ix0 : ix0 + kTileX - 1);               \
    const int w0 = (int)(smin >> 32) - 1;                                                        \
    const long long sref = in.C + in.B * (long long)(iz0 + tw * ROWS + ROWS / 2) +               \
                           in.A * (long long)(ix0 + 16);                                         \
    const int kref = (int)(sref >> 32);                                                          \
    WarpPair wp;                                                                                 \
    wp.a = in.af;                                                                                \
    wp.b = in.bf;                                                                                \
    wp.phi = (float)(unsigned)(sref & 0xffffffffLL) * 0x1p-32f;                                  \
    wp.off = (unsigned)(tj * win + (kref - w0)) * 16u - (unsigned)kFloorMagicBits * 16u;         \
    s_wp[B_][tw][tj] = wp;                                                                       \
    if (tw == 0) s_src[B_][tj] = PairSrc{w0, in.row};                                            \
  }
  // raw samples of a stage (NS pairs, tables in buffer B_) into registers:
  // warp w stages pairs w, w+4, ...; lane handles entries m = lane + 32 i
#define KK_LOAD_RAW(NS, B_)                                                        \
  _Pragma("unroll") for (int u = 0; u < PPW; ++u) {                                \
    const int j = warp + 4 * u;                                                    \
    const PairSrc src = s_src[B_][j < (NS) ? j : 0];                               \
    const float2 *y = rf_theta + (size_t)src.row * T;                              \
    _Pragma("unroll") for (int i = 0; i < QPP; ++i) {                              \
      const int m = lane + 32 * i;                                                 \
      const int k = src.w0 + m;                                                    \
      float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);                 \
      if (j < (NS) && m < win && (unsigned)k <= (unsigned)(T - 2)) {               \
        a = __ldg(y + k);                                                          \
        b = __ldg(y + k + 1);                                                      \
      }                                                                            \
      raw0[u * QPP + i] = a;                                                       \
      raw1[u * QPP + i] = b;                                                       \
    }                                                                              \
  }

  if (cur_g < J) {
    KK_FETCH(cur_p, cur_n, 0);
    ps = cur_p + cur_n;
    if (ps >= pe) enter_group(cur_g + 1);
    nxt_g = g;
    nxt_p = ps;
    nxt_n = (g < J) ? min(STAGE, pe - ps) : 0;
    if (nxt_g < J) { KK_FETCH(nxt_p, nxt_n, 1); }
    cp_async_wait_all();
    __syncthreads();
    KK_TABLES(cur_n, 0);
    __syncthreads();
    KK_LOAD_RAW(cur_n, 0);
  }
  const char *swb = reinterpret_cast<const char *>(sw);
  while (cur_g < J) {
    cp_async_wait_all();  // inputs of the next stage have landed
    __syncthreads();      // everyone is done gathering from sw
    // entries E[k] = (y[k], y[k+1] - y[k]) of this stage (zero outside [0, T-2])
#pragma unroll
    for (int u = 0; u < PPW; ++u) {
      const int j = warp + 4 * u;
#pragma unroll
      for (int i = 0; i < QPP; ++i) {
        const int m = lane + 32 * i;
        if (j < cur_n && m < win) {
          const float2 a = raw0[u * QPP + i], b = raw1[u * QPP + i];
          sw[(size_t)j * win + m] = make_float4(a.x, a.y, b.x - a.x, b.y - a.y);
        }
      }
    }
    if (nxt_g < J) { KK_TABLES(nxt_n, buf ^ 1); }
    // schedule and per-pair inputs of the stage after next (in flight below)
    int n2_g = J, n2_p = 0, n2_n = 0;
    if (nxt_g < J) {
      ps = nxt_p + nxt_n;
      if (ps >= pe) enter_group(nxt_g + 1);
      n2_g = g;
      n2_p = ps;
      n2_n = (g < J) ? min(STAGE, pe - ps) : 0;
      if (n2_g < J) { KK_FETCH(n2_p, n2_n, buf); }
    }
    __syncthreads();  // entries of this stage and tables of the next visible
    if (nxt_g < J) { KK_LOAD_RAW(nxt_n, buf ^ 1); }  // in flight during the gathers

    while (gw < cur_g) {
      float2 *dst = out + ((size_t)sidx * J + gw) * (size_t)nx * nz * (VOL ? va->ny : 1);
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const int iz = izb + r;
        if (ix < nx && iz < nz) dst[(size_t)iz * nx + ix] = acc[r];
        if constexpr (MULTI) acc[r] = make_float2(0.f, 0.f);
      }
      ++gw;
    }
    float2 sacc[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) sacc[r] = make_float2(0.f, 0.f);
    const WarpPair *tab = s_wp[buf][warp];
    // two rows per packed (f32x2) instruction: the scalar form's IEEE
    // operations in the same order, at half the issue slots
    const float2 magic2 = make_float2(kFloorMagic, kFloorMagic);
    const float2 nmagic2 = make_float2(-kFloorMagic, -kFloorMagic);
    const float2 neg1 = make_float2(-1.f, -1.f);
#pragma unroll 1
    for (int j = 0; j < cur_n; ++j) {
      const WarpPair wp = tab[j];
      const float base = fmaf(wp.a, dl, wp.phi);
      const float2 b2 = make_float2(wp.b, wp.b), base2 = make_float2(base, base);
#pragma unroll
      for (int r = 0; r < ROWS; r += 2) {
        const float2 s = __ffma2_rn(b2, make_float2((float)(r - ROWS / 2), (float)(r + 1 - ROWS / 2)), base2);
        const float2 t = __fadd2_rd(s, magic2);                        // floor in the mantissa
        const float2 f = __ffma2_rn(__fadd2_rn(t, nmagic2), neg1, s);  // s - floor(s)
        const unsigned addr0 = wp.off + ((unsigned)__float_as_int(t.x) << 4);
        const unsigned addr1 = wp.off + ((unsigned)__float_as_int(t.y) << 4);
        float4 e0 = make_float4(0.f, 0.f, 0.f, 0.f), e1 = e0;
        if (KK_IN_BOUNDS(g_bounds_kk, (unsigned)((int)(addr0 >> 4) - j * win) < (unsigned)win))
          e0 = *reinterpret_cast<const float4 *>(swb + addr0);
        if (KK_IN_BOUNDS(g_bounds_kk, (unsigned)((int)(addr1 >> 4) - j * win) < (unsigned)win))
          e1 = *reinterpret_cast<const float4 *>(swb + addr1);
        sacc[r] = __fadd2_rn(sacc[r], __ffma2_rn(make_float2(f.x, f.x), make_float2(e0.z, e0.w),
                                                 make_float2(e0.x, e0.y)));
        sacc[r + 1] = __fadd2_rn(sacc[r + 1], __ffma2_rn(make_float2(f.y, f.y), make_float2(e1.z, e1.w),
                                                         make_float2(e1.x, e1.y)));
      }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) acc[r] = f2add(acc[r], sacc[r]);
    cur_g = nxt_g;
    cur_p = nxt_p;
    cur_n = nxt_n;
    nxt_g = n2_g;
    nxt_p = n2_p;
    nxt_n = n2_n;
    buf ^= 1;
  }
#undef KK_FETCH
#undef KK_TABLES
#undef KK_LOAD_RAW
  while (gw < J) {
    float2 *dst = out + ((size_t)sidx * J + gw) * (size_t)nx * nz * (VOL ? va->ny : 1);
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int iz = izb + r;
      if (ix < nx && iz < nz) dst[(size_t)iz * nx + ix] = acc[r];
      if constexpr (MULTI) acc[r] = make_float2(0.f, 0.f);
    }
    ++gw;
  }
  if (split == 1 && I != nullptr && compound != KK_COMPOUND_NONE) {
    const size_t plane = (size_t)nx * nz * (VOL ? va->ny : 1);
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int iz = izb + r;
      if (ix < nx && iz < nz) {
        float v;
        if constexpr (MULTI) {
          // this thread's own group images, in group order (split == 1: slice 0)
          float2 sb = make_float2(0.f, 0.f);
          float si = 0.f;
          for (int g2 = 0; g2 < J; ++g2) {
            const float2 b = out[(size_t)g2 * plane + (size_t)iz * nx + ix];
            sb = f2add(sb, b);
            si = fmaf(b.x, b.x, fmaf(b.y, b.y, si));
          }
          v = (compound == KK_COMPOUND_COHERENT) ? fmaf(sb.x, sb.x, sb.y * sb.y) : si;
        } else {
          v = fmaf(acc[r].x, acc[r].x, acc[r].y * acc[r].y);   // one group: |B|^2
        }
        I[(size_t)iz * nx + ix] = v;
      }
    }
  }
}

template <int ROWS, int STAGE, int NPT, int MINB, bool MULTI>
__global__ void __launch_bounds__(kGatherThreads, MINB) k_kk_gather(const GatherArgs a) {
  extern __shared__ float4 sw[];  // [STAGE][win] staged entries
  __shared__ GatherSmem<STAGE> sm;
  gather_tile<ROWS, STAGE, NPT, MULTI>(a, blockIdx.x, blockIdx.y, sw, sm);
}

// Volumetric plans: tiles of every y slice in one grid.
template <int ROWS, int STAGE, int NPT, int MINB, bool MULTI>
__global__ void __launch_bounds__(kGatherThreads, MINB)
    k_kk_gather_vol(const GatherArgs a, const GatherVolArgs v) {
  extern __shared__ float4 sw[];
  __shared__ GatherSmem<STAGE, true> sm;
  gather_tile<ROWS, STAGE, NPT, MULTI, true>(a, blockIdx.x, blockIdx.y, sw, sm, &v);
}

// Batched form: a persistent grid pulls (frame, tile) work items, largest
// frames first, from an atomic counter until the list is exhausted.
template <int ROWS, int STAGE, int NPT, int MINB>
__global__ void __launch_bounds__(kGatherThreads, MINB)
    k_kk_gather_batch(const GatherArgs *__restrict__ frames, const int2 *__restrict__ items,
                      int n_items, int *__restrict__ counter) {
  extern __shared__ float4 sw[];
  __shared__ GatherSmem<STAGE> sm;
  __shared__ int s_item;
  for (;;) {
    __syncthreads();  // previous item fully done with shared memory
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const int2 w = items[it];
    const GatherArgs a = frames[w.x];
    gather_tile<ROWS, STAGE, NPT, true>(a, w.y, 0, sw, sm);
  }
}

// Batched form, volumetric frames: the same persistent loop over (frame,
// tile) items, tiles running over every y slice of the frame.
template <int ROWS, int STAGE, int NPT, int MINB>
__global__ void __launch_bounds__(kGatherThreads, MINB)
    k_kk_gather_batch_vol(const GatherArgs *__restrict__ frames, const GatherVolArgs *__restrict__ vols,
                          const int2 *__restrict__ items, int n_items, int *__restrict__ counter) {
  extern __shared__ float4 sw[];
  __shared__ GatherSmem<STAGE, true> sm;
  __shared__ int s_item;
  for (;;) {
    __syncthreads();  // previous item fully done with shared memory
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const int2 w = items[it];
    const GatherArgs a = frames[w.x];
    const GatherVolArgs v = vols[w.x];
    gather_tile<ROWS, STAGE, NPT, true, true>(a, w.y, 0, sw, sm, &v);
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

template <int ROWS, int STAGE, int NPT>
cudaError_t launch_cfg(const kk_plan &p, const float2 *rf_theta, float2 *dst, float *I,
                       cudaStream_t s) {
  // registers held to 72 for ROWS <= 4 (7 CTAs of 128 threads per SM; 8
  // CTAs at 64 registers spill) and to 102 for ROWS = 8 (5 CTAs)
  constexpr int MB = ROWS <= 4 ? 7 : 5;
  const size_t smem = sizeof(float4) * (size_t)STAGE * p.bf_win;
  const dim3 grid(p.tiles_x * p.tiles_z * p.ny, p.bf_split);
  cudaError_t e;
  if (p.vol) {
    // the slice term costs registers: one CTA per SM fewer than the 2D kernel, without spills
    constexpr int MBV = MB - 1;
    auto k = (p.J > 1) ? k_kk_gather_vol<ROWS, STAGE, NPT, MBV, true> : k_kk_gather_vol<ROWS, STAGE, NPT, MBV, false>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kGatherThreads, smem, s>>>(gather_args(p, rf_theta, dst, I), gather_vol_args(p));
  } else {
    auto k = (p.J > 1) ? k_kk_gather<ROWS, STAGE, NPT, MB, true> : k_kk_gather<ROWS, STAGE, NPT, MB, false>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kGatherThreads, smem, s>>>(gather_args(p, rf_theta, dst, I));
  }
  return cudaGetLastError();
}

// entries per lane needed to stage win entries of STAGE pairs; a lane holds
// at most kMaxStagedEntries of them in registers
template <int ROWS, int STAGE>
cudaError_t launch_rs(const kk_plan &p, const float2 *rf_theta, float2 *dst, float *I,
                      cudaStream_t s) {
  constexpr int PPW = STAGE / 4;
  const int q = gather_entries_per_lane(p.bf_win);
  if constexpr (PPW * 1 <= kMaxStagedEntries) {
    if (q == 1) return launch_cfg<ROWS, STAGE, PPW * 1>(p, rf_theta, dst, I, s);
  }
  if constexpr (PPW * 2 <= kMaxStagedEntries) {
    if (q == 2) return launch_cfg<ROWS, STAGE, PPW * 2>(p, rf_theta, dst, I, s);
  }
  if constexpr (PPW * 4 <= kMaxStagedEntries) {
    if (q <= 4) return launch_cfg<ROWS, STAGE, PPW * 4>(p, rf_theta, dst, I, s);
  }
  if constexpr (PPW * 8 <= kMaxStagedEntries) {
    if (q <= 8) return launch_cfg<ROWS, STAGE, PPW * 8>(p, rf_theta, dst, I, s);
  }
  return cudaErrorInvalidConfiguration;
}

}  // namespace

GatherArgs gather_args(const kk_plan &p, const float2 *rf_theta, float2 *dst, float *I) {
  GatherArgs a;
  a.rf_theta = rf_theta;
  a.T = p.T;
  a.bf_row = p.t.bf_row;
  a.bfA = p.t.bf_A;
  a.bfB = p.t.bf_B;
  a.bfC = p.t.bf_C;
  a.bfAf = p.t.bf_Af;
  a.bfBf = p.t.bf_Bf;
  a.group_start = p.t.group_start;
  a.J = p.J;
  a.nx = p.grid.nx;
  a.nz = p.grid.nz;
  a.tiles_x = p.tiles_x;
  a.win = p.bf_win;
  a.split = p.bf_split;
  a.out = dst;
  a.I = I;
  a.compound = p.compound;
  return a;
}

GatherVolArgs gather_vol_args(const kk_plan &p) {
  GatherVolArgs v;
  v.bfY = p.t.bf_Y;
  v.ny = p.ny;
  v.tiles_xz = p.tiles_x * p.tiles_z;
  return v;
}

template <int ROWS, int STAGE, int NPT>
static cudaError_t batch_cfg(const GatherArgs *frames, const GatherVolArgs *vols, const int2 *items,
                             int n_items, int *counter, int max_win, int grid, cudaStream_t s) {
  const size_t smem = sizeof(float4) * (size_t)STAGE * max_win;
  if (vols != nullptr) {
    // the slice term costs registers: one CTA per SM fewer, as for one volume
    auto k = k_kk_gather_batch_vol<ROWS, STAGE, NPT, (ROWS <= 4 ? 6 : 4)>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kGatherThreads, smem, s>>>(frames, vols, items, n_items, counter);
    return cudaGetLastError();
  }
  auto k = k_kk_gather_batch<ROWS, STAGE, NPT, (ROWS <= 4 ? 7 : 5)>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kGatherThreads, smem, s>>>(frames, items, n_items, counter);
  return cudaGetLastError();
}

template <int ROWS, int STAGE>
static cudaError_t batch_rs(const GatherArgs *frames, const GatherVolArgs *vols, const int2 *items, int n_items,
                            int *counter, int max_win, int grid, cudaStream_t s) {
  constexpr int PPW = STAGE / 4;
  const int q = gather_entries_per_lane(max_win);
  if constexpr (PPW * 1 <= kMaxStagedEntries) {
    if (q == 1) return batch_cfg<ROWS, STAGE, PPW>(frames, vols, items, n_items, counter, max_win, grid, s);
  }
  if constexpr (PPW * 2 <= kMaxStagedEntries) {
    if (q == 2) return batch_cfg<ROWS, STAGE, PPW * 2>(frames, vols, items, n_items, counter, max_win, grid, s);
  }
  if constexpr (PPW * 4 <= kMaxStagedEntries) {
    if (q <= 4) return batch_cfg<ROWS, STAGE, PPW * 4>(frames, vols, items, n_items, counter, max_win, grid, s);
  }
  if constexpr (PPW * 8 <= kMaxStagedEntries) {
    if (q <= 8) return batch_cfg<ROWS, STAGE, PPW * 8>(frames, vols, items, n_items, counter, max_win, grid, s);
  }
  return cudaErrorInvalidConfiguration;
}

cudaError_t launch_kk_gather_batch(int rows, int stage, const GatherArgs *frames, const GatherVolArgs *vols,
                                   const int2 *items, int n_items, int *counter, int max_win, int grid,
                                   cudaStream_t s) {
  switch (rows * 100 + stage) {
    case 204: return batch_rs<2, 4>(frames, vols, items, n_items, counter, max_win, grid, s);
    case 208: return batch_rs<2, 8>(frames, vols, items, n_items, counter, max_win, grid, s);
    case 216: return batch_rs<2, 16>(frames, vols, items, n_items, counter, max_win, grid, s);
    case 404: return batch_rs<4, 4>(frames, vols, items, n_items, counter, max_win, grid, s);
    case 408: return batch_rs<4, 8>(frames, vols, items, n_items, counter, max_win, grid, s);
    case 416: return batch_rs<4, 16>(frames, vols, items, n_items, counter, max_win, grid, s);
    case 804: return batch_rs<8, 4>(frames, vols, items, n_items, counter, max_win, grid, s);
    case 808: return batch_rs<8, 8>(frames, vols, items, n_items, counter, max_win, grid, s);
    case 816: return batch_rs<8, 16>(frames, vols, items, n_items, counter, max_win, grid, s);
    default: return cudaErrorInvalidConfiguration;
  }
}

#ifdef KK_DEBUG_BOUNDS
cudaError_t take_bounds_kk(unsigned long long *n) {
  unsigned v = 0, zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_bounds_kk, sizeof(v));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bounds_kk, &zero, sizeof(zero));
  *n = v;
  return e;
}
#endif

int gather_entries_per_lane(int win) {
  const int q = (win + 31) / 32;
  return q <= 1 ? 1 : (q <= 2 ? 2 : (q <= 4 ? 4 : (q <= 8 ? 8 : 0)));
}

bool gather_config_supported(int rows, int stage, int win) {
  if (!((rows == 2 || rows == 4 || rows == 8) && (stage == 4 || stage == 8 || stage == 16))) return false;
  const int q = gather_entries_per_lane(win);
  return q > 0 && (stage / 4) * q <= kMaxStagedEntries;
}

cudaError_t launch_kk_gather(const kk_plan &p, const float2 *rf_theta, float2 *B, float *I,
                             float2 *partial, cudaStream_t s) {
  float2 *dst = (p.bf_split > 1) ? partial : B;
  cudaError_t e;
  const int key = p.bf_rows * 100 + p.bf_stage;
  switch (key) {
    case 204: e = launch_rs<2, 4>(p, rf_theta, dst, I, s); break;
    case 208: e = launch_rs<2, 8>(p, rf_theta, dst, I, s); break;
    case 216: e = launch_rs<2, 16>(p, rf_theta, dst, I, s); break;
    case 404: e = launch_rs<4, 4>(p, rf_theta, dst, I, s); break;
    case 408: e = launch_rs<4, 8>(p, rf_theta, dst, I, s); break;
    case 416: e = launch_rs<4, 16>(p, rf_theta, dst, I, s); break;
    case 804: e = launch_rs<8, 4>(p, rf_theta, dst, I, s); break;
    case 808: e = launch_rs<8, 8>(p, rf_theta, dst, I, s); break;
    case 816: e = launch_rs<8, 16>(p, rf_theta, dst, I, s); break;
    default: return cudaErrorInvalidConfiguration;
  }
  if (e != cudaSuccess || p.bf_split == 1) return e;
  const int npix = p.grid.nx * p.grid.nz * p.ny;
  k_kk_reduce<<<(npix + 255) / 256, 256, 0, s>>>(partial, p.bf_split, p.J, npix, B, I, p.compound);
  return cudaGetLastError();
}

}  // namespace kk
