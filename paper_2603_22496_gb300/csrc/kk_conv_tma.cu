// kk_conv_tma.cu -- the refiner's convolutions with TMA-fed operands:
// forward / backward-data (K-major) and weight gradient (MN-major) on
// tcgen05 with TMEM accumulators, for the shapes whose 128-pixel (64-pixel
// for the weight gradient) tiles are whole row segments or whole rows of one
// image -- every level of the encoder-decoder on 256 x 256 images.  Other
// shapes use the cp.async-gathered kernels of kk_conv_tc.cu.
//
// Operands land in the swizzled canonical layouts (the tensor map's swizzle
// matches the descriptor's layout type: rows of 128 / 64 / 32 bytes ->
// SWIZZLE_128B / 64B / 32B, codes 2 / 4 / 6 in the descriptor), so each copy
// is a wide box:
//   forward A  X [n][h][w][c] as (c, w, h, n), box {KC, bw, bh, 1}: one chunk
//              = KC channels of a bw x bh = 128-pixel tile at tap offset
//              (kw - 1, kh - 1); the image border comes from the zero fill.
//              K-major, rows = pixels, SBO = 8 rows, K step = 32 bytes.
//   forward B  W [cout][9 cin] as (9 cin, cout), box {KC, N}; K-major.
//   wgrad   A  X as above, box {AC, bw, bh, 1} with bw x bh = 64 pixels:
//              MN-major atoms of AC = 64 / 32 / 16 channels (one tap each);
//              LBO = atom stride, SBO = 8 pixel rows, K step = 2 SBO.
//   wgrad   B  dY [P][cout] as (cout, P), box {AC, 64}; MN-major atoms.
// One thread issues a chunk's copies (lanes of warp 0 when there are
// several), all completing on the stage's mbarrier (expect_tx = its bytes).
// Weight gradient: warp 0 issues the copies, warp 1's lane 0 the MMAs, all
// four warps run the epilogue.  Every wait is bounded; a CTA that gives up records
// KK_ERR_TIMEOUT, waits (bounded) for the copies it issued, frees its TMEM
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "kk_internal.h"
#include "kk_nn.h"
#include "kk_tc.h"
#include "kk_tma.h"

namespace kk {
namespace nn {
namespace {

using namespace kk::tc;

constexpr int kMaxStages = 8;
constexpr int kStageBudget = 40 * 1024;  // ring of about 40 KB: several CTAs per SM
constexpr int kTileM = 128;
constexpr int kMaxN = 256;
constexpr int kThreads = 128;
constexpr int kWgK = 64;

__device__ int g_tma_status;

using kk::tma::encoder;
using kk::tma::EncodeFn;

// swizzle of a row of `ch` bf16 channels (32 / 64 / 128 bytes) and the
// matching descriptor layout code
CUtensorMapSwizzle swizzle_of(int ch) {
  return ch == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : ch == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
}
__host__ __device__ constexpr uint32_t layout_code(int ch) { return ch == 64 ? 2u : ch == 32 ? 4u : 6u; }
// the largest of 64 / 32 / 16 dividing c (c is a multiple of 16)
int atom_channels(int c) { return c % 64 == 0 ? 64 : c % 32 == 0 ? 32 : 16; }

// bf16 tiled tensor map; dims innermost first, strides (bytes) of dims 1..rank-1
bool make_map(CUtensorMap *m, const void *base, int rank, const cuuint64_t *dims, const cuuint64_t *strides,
              const cuuint32_t *box, CUtensorMapSwizzle sw) {
  EncodeFn f = encoder();
  if (!f) return false;
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void *>(base), dims, strides, box, es,
           CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// X [n][h][w][c] as (c, w, h, n), box {bc, bw, bh, 1}, rows of bc channels
bool map_nhwc(CUtensorMap *m, const Tensor4 &x, int bc, int bw, int bh) {
  const cuuint64_t dims[4] = {(cuuint64_t)x.c, (cuuint64_t)x.w, (cuuint64_t)x.h, (cuuint64_t)x.n};
  const cuuint64_t strides[3] = {(cuuint64_t)x.c * 2, (cuuint64_t)x.w * x.c * 2, (cuuint64_t)x.h * x.w * x.c * 2};
  const cuuint32_t box[4] = {(cuuint32_t)bc, (cuuint32_t)bw, (cuuint32_t)bh, 1};
  return make_map(m, x.p, 4, dims, strides, box, swizzle_of(bc));
}

// [rows][cols] bf16 row-major as (cols, rows), box {bc, br}
bool map_2d(CUtensorMap *m, const void *base, int rows, int cols, int bc, int br) {
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)bc, (cuuint32_t)br};
  return make_map(m, base, 2, dims, strides, box, swizzle_of(bc));
}

__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap *m, int c0, int c1, int c2, int c3,
                                       uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
using kk::tma::tma_2d;
// shared-memory descriptor with a layout (swizzle) code
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
  return smem_desc(saddr, lbo, sbo) | ((uint64_t)layout << 61);
}
using kk::tma::mbar_expect_tx;
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// pixel tile t of `tp` pixels (whole row segments or whole rows): image, first row, first column
__device__ __forceinline__ void tile_origin(int t, int tp, int H, int W, int bw, int &img, int &h0, int &w0) {
  const int per_img = H * W / tp;
  img = t / per_img;
  const int loc = t - img * per_img;
  if (bw == W) {
    h0 = loc * (tp / W);
    w0 = 0;
  } else {
    const int per_row = W / bw;
    h0 = loc / per_row;
    w0 = (loc - h0 * per_row) * bw;
  }
}

struct TmaConvArgs {
  int n, h, w, cin, cout, bw;
  const float *bias;
  int relu;
  __nv_bfloat16 *y;
  float *yf;
  int *status;
};

// Forward / backward-data convolution, persistent: 1-4 CTAs per SM (as many
// as TMEM holds with two accumulators each) loop over (pixel tile, channel
// tile) items with one continuous copy ring each (up to 16 stages, about
// 200 KB per SM) and two TMEM accumulators, so that the epilogue of one item
// overlaps the MMAs of the next.  Warp 0 issues the
// copies, warp 1's lane 0 the MMAs, warps 2-5 run the epilogue (warp w reads
// TMEM lane quarter w % 4).  Barriers: full / empty per stage; acc_full[b]
// (MMA commit) and acc_empty[b] (the 128 epilogue threads) per accumulator.
constexpr int kPersThreads = 192;
constexpr int kPersMaxStages = 16;
constexpr int kPersBudget = 200 * 1024;

// HALO (one-row tiles of 128 pixels): a stage is one channel chunk -- one
// copy of the tile's 3 input rows x 130 pixels (box {KC, 130, 3, 1} at
// (c0, w0 - 1, h0 - 1)) plus the nine taps' weight tiles -- and tap (kh, kw)
// reads A from row kh * 130 + kw of that halo tile (rows are packed densely,
// so a tap is a whole-row shift of the descriptor start within the swizzled
// tile).  Each input pixel then crosses L2 about 3 times per layer, not 9.
constexpr int kHaloW = kTileM + 2;
constexpr int kHaloRows = 3 * kHaloW;
__host__ __device__ constexpr uint32_t halo_bytes(int KC) {
  return (uint32_t)((kHaloRows * KC * 2 + 1023) / 1024 * 1024);
}

template <int KC, bool HALO>
__global__ void __launch_bounds__(kPersThreads)
    k_conv3x3_tma_pers(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW,
                       const TmaConvArgs a, const int N, const int S, const int n_items, const int n_ntiles) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[kPersMaxStages], empty_bar[kPersMaxStages];
  __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  constexpr uint32_t A_BYTES = HALO ? halo_bytes(KC) : kTileM * KC * 2;
  constexpr uint32_t ROW = KC * 2;
  constexpr uint32_t LAYOUT = layout_code(KC);
  const uint32_t B_BYTES = (uint32_t)N * KC * 2;
  const uint32_t STAGE = A_BYTES + (HALO ? 9u : 1u) * B_BYTES;
  const uint32_t STAGE_TX = (HALO ? (uint32_t)kHaloRows * ROW : A_BYTES) + (HALO ? 9u : 1u) * B_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cpt = a.cin / KC;
  const int nK = HALO ? cpt : 9 * cpt;
  int *status = a.status ? a.status : &g_tma_status;

  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;
  if (warp == 0) {
    tmem_alloc(&tmem_slot, 2 * ncols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int q = 0; q < S; ++q) {
      mbar_init(&full_bar[q], 1);
      mbar_init(&empty_bar[q], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], 128);
    }
    mbar_init(&done_bar, 1);
    s_abort = 0;
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t sbase = smem_u32(smem);

  if (warp == 0) {
    // ---- copies: every chunk of every item of this CTA through one ring ----
    int g = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
      const int tile = it / n_ntiles, n0 = (it - tile * n_ntiles) * N;
      int img, h0, w0;
      tile_origin(tile, kTileM, a.h, a.w, a.bw, img, h0, w0);
      for (int k = 0; k < nK; ++k, ++g) {
        const int s = g % S;
        int go = 1;
        if (lane == 0) {
          if (g >= S && !mbar_wait(&empty_bar[s], (uint32_t)((g / S) - 1) & 1u)) go = 0;
          if (go) {
            mbar_expect_tx(&full_bar[s], STAGE_TX);
            const uint32_t sA = sbase + (uint32_t)s * STAGE;
            if constexpr (HALO) {
              const int c0 = k * KC;
              tma_4d(sA, &tmX, c0, w0 - 1, h0 - 1, img, &full_bar[s]);
              for (int tap = 0; tap < 9; ++tap)
                tma_2d(sA + A_BYTES + (uint32_t)tap * B_BYTES, &tmW, tap * a.cin + c0, n0, &full_bar[s]);
            } else {
              const int tap = k / cpt, c0 = (k - tap * cpt) * KC;
              const int kh = tap / 3, kw = tap - kh * 3;
              tma_4d(sA, &tmX, c0, w0 + kw - 1, h0 + kh - 1, img, &full_bar[s]);
              tma_2d(sA + A_BYTES, &tmW, tap * a.cin + c0, n0, &full_bar[s]);
            }
          }
        }
        go = __shfl_sync(0xffffffffu, go, 0);
        if (!go) {
          s_abort = 1;
          ok = false;
          break;
        }
      }
    }
    // no copy may still be in flight at exit (bounded waits)
    if (lane == 0)
      for (int j = max(0, g - S); j < g; ++j) mbar_wait(&full_bar[j % S], (uint32_t)(j / S) & 1u);
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMAs: item li accumulates into TMEM buffer li & 1 ----
    if (lane == 0) {
      const uint32_t idesc = instr_desc(1u /* bf16 */, kTileM, (uint32_t)N);
      int g = 0, li = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++li) {
        const int b = li & 1;
        if (li >= 2 && !mbar_wait(&acce_bar[b], (uint32_t)((li >> 1) - 1) & 1u)) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)b * ncols;
        for (int k = 0; k < nK; ++k, ++g) {
          const int s = g % S;
          if (!mbar_wait(&full_bar[s], (uint32_t)(g / S) & 1u)) {
            s_abort = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sA = sbase + (uint32_t)s * STAGE, sB = sA + A_BYTES;
          if constexpr (HALO) {
            for (int tap = 0; tap < 9; ++tap) {
              const int kh = tap / 3, kw = tap - kh * 3;
              const uint32_t sAt = sA + (uint32_t)(kh * kHaloW + kw) * ROW;
              const uint32_t sBt = sB + (uint32_t)tap * B_BYTES;
#pragma unroll
              for (int kk = 0; kk < KC / 16; ++kk) {
                const uint64_t ad = smem_desc_sw(sAt + (uint32_t)kk * 32, 16, 8 * ROW, LAYOUT);
                const uint64_t bd = smem_desc_sw(sBt + (uint32_t)kk * 32, 16, 8 * ROW, LAYOUT);
                mma_bf16(acc, ad, bd, idesc, (k | tap | kk) != 0 ? 1u : 0u);
              }
            }
          } else {
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
              const uint64_t ad = smem_desc_sw(sA + (uint32_t)kk * 32, 16, 8 * ROW, LAYOUT);
              const uint64_t bd = smem_desc_sw(sB + (uint32_t)kk * 32, 16, 8 * ROW, LAYOUT);
              mma_bf16(acc, ad, bd, idesc, (k | kk) != 0 ? 1u : 0u);
            }
          }
          mma_commit(&empty_bar[s]);
        }
        if (ok) mma_commit(&accf_bar[b]);
      }
      mma_commit(&done_bar);  // arrives when every MMA issued above has completed
    }
    __syncwarp();
  } else {
    // ---- epilogue: warps 2-5, TMEM lane quarter warp % 4 ----
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int li = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x, ++li) {
      const int b = li & 1;
      if (!mbar_wait(&accf_bar[b], (uint32_t)(li >> 1) & 1u)) {
        s_abort = 1;
        break;
      }
      tc_fence_after();
      const int tile = it / n_ntiles, n0 = (it - tile * n_ntiles) * N;
      const size_t p = (size_t)tile * kTileM + row;
      const uint32_t trow = tmem + (uint32_t)b * ncols + ((uint32_t)(q * 32) << 16);
      for (int c = 0; c < N; c += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c, v);
        const int co = n0 + c;
        if (co >= a.cout) continue;
        if (a.bias) {
#pragma unroll
          for (int u = 0; u < 16; ++u) v[u] += __ldg(a.bias + co + u);
        }
        if (a.relu) {
#pragma unroll
          for (int u = 0; u < 16; ++u) v[u] = fmaxf(v[u], 0.f);
        }
        if (a.y) {
          uint4 *dst = reinterpret_cast<uint4 *>(a.y + p * a.cout + co);
          dst[0] = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                              pack_bf16x2(v[6], v[7]));
          dst[1] = make_uint4(pack_bf16x2(v[8], v[9]), pack_bf16x2(v[10], v[11]), pack_bf16x2(v[12], v[13]),
                              pack_bf16x2(v[14], v[15]));
        }
        if (a.yf) {
          float4 *dst = reinterpret_cast<float4 *>(a.yf + p * a.cout + co);
#pragma unroll
          for (int u = 0; u < 4; ++u) dst[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
        }
      }
      tc_fence_before();
      mbar_arrive(&acce_bar[b]);
    }
  }
  __syncthreads();
  if (warp == 0) {
    const bool done = mbar_wait(&done_bar, 0);
    if ((!done || s_abort) && lane == 0) atomicExch(status, (int)KK_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 2 * ncols);
}

struct TmaWgradArgs {
  int n, h, w, cin, cout, bw;
  int chunks_per_split, n_chunks;
  int aca, acb;  // channels per MN atom of A (X) and B (dY): 64, 32 or 16
  float *part;
  int *status;
};

__global__ void __launch_bounds__(kThreads)
    k_wgrad_tma(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmD,
                const TmaWgradArgs a, const int N, const int S) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  constexpr uint32_t A_BYTES = kWgK * kTileM * 2;
  const uint32_t B_BYTES = (uint32_t)kWgK * N * 2;
  const int nB = N / a.acb;  // B atoms per chunk
  const uint32_t atomA = (uint32_t)kWgK * a.aca * 2, atomB = (uint32_t)kWgK * a.acb * 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Ncol = 9 * a.cin;
  const int r0 = blockIdx.x * kTileM, n0 = blockIdx.y * N;
  const int cb = blockIdx.z * a.chunks_per_split, ce = min(a.n_chunks, cb + a.chunks_per_split);
  const int nK = max(0, ce - cb);
  const int validA = (min(kTileM, Ncol - r0) + a.aca - 1) / a.aca;  // atoms holding rows < Ncol
  const uint32_t STAGE = A_BYTES + B_BYTES;
  const uint32_t TX = (uint32_t)validA * atomA + B_BYTES;
  int *status = a.status ? a.status : &g_tma_status;

  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;
  if (warp == 0) {
    tmem_alloc(&tmem_slot, ncols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    s_abort = 0;
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t sbase = smem_u32(smem);

  if (warp == 0) {
    // lane j < nA owns A atom j (one tap, aca channels) for every chunk
    int gdh = 0, gdw = 0, gc = 0;
    if (lane < validA) {
      const int r = r0 + a.aca * lane;
      const int tap = r / a.cin;
      gc = r - tap * a.cin;
      gdh = tap / 3 - 1;
      gdw = tap % 3 - 1;
    }
    int issued = 0;
    for (int k = 0; k < nK; ++k) {
      const int s = k % S;
      int go = 1;
      if (lane == 0) {
        if (k >= S && !mbar_wait(&empty_bar[s], (uint32_t)((k / S) - 1) & 1u)) go = 0;
        if (go) mbar_expect_tx(&full_bar[s], TX);
      }
      go = __shfl_sync(0xffffffffu, go, 0);
      if (!go) {
        s_abort = 1;
        break;
      }
      const int c = cb + k;
      int img, h0, w0;
      tile_origin(c, kWgK, a.h, a.w, a.bw, img, h0, w0);
      const uint32_t sA = sbase + (uint32_t)s * STAGE, sB = sA + A_BYTES;
      if (lane < validA) tma_4d(sA + (uint32_t)lane * atomA, &tmX, gc, w0 + gdw, h0 + gdh, img, &full_bar[s]);
      if (lane >= 16 && lane < 16 + nB) {
        const int g = lane - 16;
        tma_2d(sB + (uint32_t)g * atomB, &tmD, n0 + g * a.acb, c * kWgK, &full_bar[s]);
      }
      issued = k + 1;
    }
    if (lane == 0)
      for (int j = std::max(0, issued - S); j < issued; ++j) mbar_wait(&full_bar[j % S], (uint32_t)(j / S) & 1u);
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc(1u /* bf16 */, kTileM, (uint32_t)N) | (1u << 15) | (1u << 16);
      for (int k = 0; k < nK; ++k) {
        const int s = k % S;
        if (!mbar_wait(&full_bar[s], (uint32_t)(k / S) & 1u)) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sA = sbase + (uint32_t)s * STAGE, sB = sA + A_BYTES;
#pragma unroll
        for (int q = 0; q < kWgK / 16; ++q) {
          const uint32_t sboA = 16u * a.aca, sboB = 16u * a.acb;  // 8 pixel rows
          const uint64_t ad = smem_desc_sw(sA + (uint32_t)q * 2 * sboA, atomA, sboA, layout_code(a.aca));
          const uint64_t bd = smem_desc_sw(sB + (uint32_t)q * 2 * sboB, atomB, sboB, layout_code(a.acb));
          mma_bf16(tmem, ad, bd, idesc, (k | q) != 0 ? 1u : 0u);
        }
        mma_commit(&empty_bar[s]);
      }
      mma_commit(&done_bar);
    }
    __syncwarp();
  }

  __syncwarp();
  const bool done = mbar_wait(&done_bar, 0);
  tc_fence_after();
  __syncthreads();
  if (!done || s_abort) {
    if (tid == 0) atomicExch(status, (int)KK_ERR_TIMEOUT);
  } else {
    const int r = r0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    float *dst = a.part + (size_t)blockIdx.z * ((size_t)a.cout * Ncol);
    for (int c = 0; c < N; c += 16) {
      float v[16];
      tmem_ld16(trow + (uint32_t)c, v);
      if (r >= Ncol) continue;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int co = n0 + c + q;
        if (co < a.cout) dst[(size_t)co * Ncol + r] = nK > 0 ? v[q] : 0.f;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// 3..8 stages: about 40 KB of ring, at most 200 KB
inline int ring_stages(size_t bytes) {
  int S = (int)std::max<size_t>(3, std::min<size_t>(kMaxStages, kStageBudget / bytes));
  while (S > 2 && (size_t)S * bytes > 200 * 1024) --S;
  return S;
}

// tile width / height for tp-pixel tiles, or false when the shape does not tile
bool tile_shape(int H, int W, int tp, int &bw, int &bh) {
  if (W % tp == 0) {
    bw = tp;
    bh = 1;
    return true;
  }
  if (tp % W == 0 && H % (tp / W) == 0) {
    bw = W;
    bh = tp / W;
    return true;
  }
  return false;
}

int sm_count() {
  int dev = 0, n = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

template <int KC, bool HALO>
cudaError_t launch_fwd(const CUtensorMap &mx, const CUtensorMap &mw, const TmaConvArgs &a, int N, int tiles,
                       cudaStream_t s) {
  // persistent CTAs per SM: as many as TMEM holds (2 accumulators each), at
  // most 4; halo stages are larger, so at most 2 CTAs with 2+ stages each
  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;
  const size_t stage = HALO ? (size_t)halo_bytes(KC) + 9 * (size_t)N * KC * 2
                            : (size_t)kTileM * KC * 2 + (size_t)N * KC * 2;
  int cps = std::max(1, std::min(4, (int)(512 / (2 * ncols))));
  if (HALO)  // two stages per CTA at least: as many CTAs as fit in the shared-memory budget
    cps = std::max(1, std::min(cps, (int)(kPersBudget / (2 * stage))));
  const int S = (int)std::max<size_t>(HALO ? 2 : 3, std::min<size_t>(kPersMaxStages, kPersBudget / cps / stage));
  const size_t smem = (size_t)S * stage;
  auto k = k_conv3x3_tma_pers<KC, HALO>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int n_ntiles = (a.cout + N - 1) / N;
  const int n_items = tiles * n_ntiles;
  const int grid = std::min(n_items, cps * sm_count());
  k<<<grid, kPersThreads, smem, s>>>(mx, mw, a, N, S, n_items, n_ntiles);
  return cudaGetLastError();
}

}  // namespace

bool conv3x3_tma(const Tensor4 &x, const __nv_bfloat16 *w, int cout, const float *bias, bool relu,
                 __nv_bfloat16 *y, float *yf, int *status, cudaStream_t s, cudaError_t *err) {
  int bw, bh;
  if (!tile_shape(x.h, x.w, kTileM, bw, bh) || x.c % 16 || cout % 16) return false;
  int KC = atom_channels(x.c);
  int N = std::min(cout, kMaxN);
  const long tiles = (long)x.n * x.h * x.w / kTileM;
  while (N > 32 && N % 32 == 0 && tiles * ((cout + N - 1) / N) < 304) N /= 2;
  CUtensorMap mx, mw;
  // one-row tiles read a halo tile per chunk of at most 32 channels (wider
  // inputs in 32-channel chunks), while a stage of nine weight tiles fits
  const bool halo = bh == 1 && (KC <= 32 || x.c % 32 == 0) && N <= 64;
  if (halo && KC > 32) KC = 32;
  if (!map_nhwc(&mx, x, KC, halo ? kHaloW : bw, halo ? 3 : bh) || !map_2d(&mw, w, cout, 9 * x.c, KC, N))
    return false;
  TmaConvArgs a{x.n, x.h, x.w, x.c, cout, bw, bias, relu ? 1 : 0, y, yf, status};
  if (KC == 64)
    *err = launch_fwd<64, false>(mx, mw, a, N, (int)tiles, s);
  else if (KC == 32)
    *err = halo ? launch_fwd<32, true>(mx, mw, a, N, (int)tiles, s) : launch_fwd<32, false>(mx, mw, a, N, (int)tiles, s);
  else
    *err = halo ? launch_fwd<16, true>(mx, mw, a, N, (int)tiles, s) : launch_fwd<16, false>(mx, mw, a, N, (int)tiles, s);
  return true;
}

bool wgrad_tma(const Tensor4 &x, const __nv_bfloat16 *dy, int cout, float *part, int splits, int pix_per_split,
               int *status, cudaStream_t s, cudaError_t *err) {
  int bw, bh;
  if (!tile_shape(x.h, x.w, kWgK, bw, bh) || x.c % 16 || cout % 16 || pix_per_split % kWgK) return false;
  const int P = x.n * x.h * x.w;
  const int n_chunks = P / kWgK;
  const int per = pix_per_split / kWgK;  // chunks per split
  const int N = std::min(cout, kMaxN);
  const int aca = atom_channels(x.c), acb = atom_channels(N);
  CUtensorMap mx, md;
  if (!map_nhwc(&mx, x, aca, bw, bh) || !map_2d(&md, dy, P, cout, acb, kWgK)) return false;
  TmaWgradArgs a{x.n, x.h, x.w, x.c, cout, bw, per, n_chunks, aca, acb, part, status};
  const size_t stage = (size_t)kWgK * kTileM * 2 + (size_t)kWgK * N * 2;
  const int S = ring_stages(stage);
  const size_t smem = (size_t)S * stage;
  cudaError_t e = cudaFuncSetAttribute(k_wgrad_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) {
    dim3 grid((9 * x.c + kTileM - 1) / kTileM, (cout + N - 1) / N, splits);
    k_wgrad_tma<<<grid, kThreads, smem, s>>>(mx, md, a, N, S);
    e = cudaGetLastError();
  }
  *err = e;
  return true;
}

cudaError_t tma_status(int *out) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_tma_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tma_status, &zero, sizeof(int));
  return e;
}

}  // namespace nn
}  // namespace kk
