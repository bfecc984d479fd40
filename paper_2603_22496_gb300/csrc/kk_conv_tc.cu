// kk_conv_tc.cu -- 3x3 convolution (forward and backward-data) of the
// learned refiner as an implicit GEMM on the 5th-generation tensor cores:
// tcgen05.mma (BF16 operands, FP32 accumulator in TMEM), operands gathered
// into shared memory by cp.async.
//
//   D[p][co] = sum_{tap, ci} X[p + tap][ci] W[co][tap][ci]
//   M = 128 output pixels per CTA, N = output channels (<= 256 per CTA),
//   K = 9 taps x Cin, in chunks of KC = min(64, Cin) channels of one tap.
//
// A chunk's operands in the no-swizzle K-major canonical layout (core
// matrix = 8 rows x 16 bytes):
//   A: [K slice j of 8 channels][pixel p] 16 bytes each -> K-adjacent core
//      matrices 2048 bytes apart (LBO), M-adjacent 128 bytes (SBO);
//   B: [K slice j][output channel n] 16 bytes each -> LBO = 16 N, SBO = 128.
// The im2col gather is one 16-byte cp.async per (pixel, slice); taps outside
// the image are zero-filled by the copy (source size 0).
//
// Warp roles: warps 0-3 gather chunks into a ring of S = 4..8 stages (about
// 96 KB) and afterwards run the epilogue (warp w owns TMEM lanes 32w..32w+31
// = pixels); warp 4's lane 0 issues the MMAs.  Stage handshake: a producer
// thread keeps S - 1 chunks of copies in flight; when it has issued chunk k
// it waits for its own copies of chunk k - S + 1 (cp.async.wait_group), makes
// them visible to the tensor core (fence.proxy.async) and arrives on
// full[stage]; the MMA thread
// waits on full, issues KC/16 MMAs and commits to empty[stage], which the
// producers wait on before they refill the stage.  Every wait is bounded; on
// a timeout the CTA records KK_ERR_TIMEOUT, waits for its own copies and
// MMAs (bounded), frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "kk_internal.h"
#include "kk_nn.h"
#include "kk_tc.h"

namespace kk {
namespace nn {
namespace {

using namespace kk::tc;

constexpr int kMaxStages = 8;    // stage ring: 4..8 stages, about 96 KB of shared memory
constexpr int kStageBudget = 96 * 1024;
constexpr int kTileM = 128;
constexpr int kMaxN = 256;
constexpr int kProducers = 128;  // warps 0-3
constexpr int kThreads = 160;    // + the MMA warp

__device__ int g_conv_status;    // status of layer-level launches without a status word

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// wait until at most n (0..7) groups are pending
__device__ __forceinline__ void cp_async_wait_pending(int n) {
  switch (n) {
    case 0: cp_async_wait<0>(); break;
    case 1: cp_async_wait<1>(); break;
    case 2: cp_async_wait<2>(); break;
    case 3: cp_async_wait<3>(); break;
    case 4: cp_async_wait<4>(); break;
    case 5: cp_async_wait<5>(); break;
    case 6: cp_async_wait<6>(); break;
    default: cp_async_wait<7>(); break;
  }
}
// stages of a ring whose stage takes `bytes`
inline int ring_stages(size_t bytes) {
  return (int)std::max<size_t>(4, std::min<size_t>(kMaxStages, kStageBudget / bytes));
}
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

struct ConvArgs {
  const __nv_bfloat16 *x;
  int n, h, w, cin;
  const __nv_bfloat16 *wt;  // [cout][3][3][cin]
  int cout;
  const float *bias;        // nullable
  int relu;
  __nv_bfloat16 *y;         // nullable, [pixels][cout]
  float *yf;                // nullable
  int *status;              // nullable -> g_conv_status
};

template <int KC>
__global__ void __launch_bounds__(kThreads) k_conv3x3_tc(const ConvArgs a, const int N, const int S) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  constexpr int SL = KC / 8;  // 16-byte K slices per chunk
  constexpr uint32_t A_BYTES = kTileM * KC * 2;
  const uint32_t B_BYTES = (uint32_t)N * KC * 2;
  const uint32_t STAGE = A_BYTES + B_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int P = a.n * a.h * a.w;
  const int m0 = blockIdx.x * kTileM, n0 = blockIdx.y * N;
  const int cpt = a.cin / KC;  // chunks per tap
  const int nK = 9 * cpt;
  int *status = a.status ? a.status : &g_conv_status;

  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;
  if (warp == 0) {
    tmem_alloc(&tmem_slot, ncols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], kProducers);
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

  if (warp < 4) {
    // ---------------- producers: im2col gather of A, weights of B --------------
    const int p = m0 + tid;
    int pn = 0, ph = 0, pw = 0;
    if (p < P) {
      pn = p / (a.h * a.w);
      const int r = p - pn * a.h * a.w;
      ph = r / a.w;
      pw = r - ph * a.w;
    }
    bool ok = true;
    int k = 0;
    for (; k < nK; ++k) {
      const int s = k % S;
      if (k >= S && !mbar_wait(&empty_bar[s], (uint32_t)((k / S) - 1) & 1u)) {
        ok = false;
        break;
      }
      const int tap = k / cpt, c0 = (k - tap * cpt) * KC;
      const int kh = tap / 3, kw = tap - kh * 3;
      const int hh = ph + kh - 1, ww = pw + kw - 1;
      const bool valid = p < P && hh >= 0 && hh < a.h && ww >= 0 && ww < a.w;
      const __nv_bfloat16 *src = valid ? a.x + (((size_t)pn * a.h + hh) * a.w + ww) * a.cin + c0 : a.x;
      const uint32_t sA = sbase + (uint32_t)s * STAGE;
#pragma unroll
      for (int j = 0; j < SL; ++j)
        cp_async16(sA + (uint32_t)j * (kTileM * 16) + (uint32_t)tid * 16, src + 8 * j, valid ? 16u : 0u);
      const uint32_t sB = sA + A_BYTES;
      for (int r = tid; r < N; r += kProducers) {
        const int co = n0 + r;
        const bool vb = co < a.cout;
        const __nv_bfloat16 *wsrc = vb ? a.wt + ((size_t)co * 9 + tap) * a.cin + c0 : a.wt;
#pragma unroll
        for (int j = 0; j < SL; ++j)
          cp_async16(sB + (uint32_t)j * ((uint32_t)N * 16) + (uint32_t)r * 16, wsrc + 8 * j, vb ? 16u : 0u);
      }
      cp_async_commit();
      // keep S - 1 chunks in flight: wait for the oldest, publish it
      if (k >= S - 1) {
        cp_async_wait_pending(S - 1);
        fence_async_smem();
        mbar_arrive(&full_bar[(k - (S - 1)) % S]);
      }
    }
    cp_async_wait<0>();
    fence_async_smem();
    if (ok) {
      for (int j = std::max(0, nK - (S - 1)); j < nK; ++j) mbar_arrive(&full_bar[j % S]);
    } else {
      s_abort = 1;
    }
  } else if (warp == 4) {
    // ---------------- MMA issuer (one thread) -----------------------------------
    if (lane == 0) {
    const uint32_t idesc = instr_desc(1u /* bf16 */, kTileM, (uint32_t)N);
    int k = 0;
    for (; k < nK; ++k) {
      const int s = k % S;
      if (!mbar_wait(&full_bar[s], (uint32_t)(k / S) & 1u)) {
        s_abort = 1;
        break;
      }
      tc_fence_after();
      const uint32_t sA = sbase + (uint32_t)s * STAGE, sB = sA + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < KC / 16; ++kk) {
        const uint64_t ad = smem_desc(sA + (uint32_t)kk * 2 * (kTileM * 16), kTileM * 16, 128);
        const uint64_t bd = smem_desc(sB + (uint32_t)kk * 2 * ((uint32_t)N * 16), (uint32_t)N * 16, 128);
        mma_bf16(tmem, ad, bd, idesc, (k | kk) != 0 ? 1u : 0u);
      }
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&done_bar);  // arrives when every MMA issued above has completed
    }
    __syncwarp();
  }

  // ---------------- epilogue -----------------------------------------------------
  if (warp < 4) {
    __syncwarp();
    const bool done = mbar_wait(&done_bar, 0);
    tc_fence_after();
    if (!done || s_abort) {
      if (tid == 0) atomicExch(status, (int)KK_ERR_TIMEOUT);
    } else {
      const int row = warp * 32 + lane;
      const int p = m0 + row;
      const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
      for (int c = 0; c < N; c += 16) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c, v);
        const int co = n0 + c;
        if (p >= P || co >= a.cout) continue;
        if (a.bias) {
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] += __ldg(a.bias + co + q);
        }
        if (a.relu) {
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = fmaxf(v[q], 0.f);
        }
        if (a.y) {
          uint4 *dst = reinterpret_cast<uint4 *>(a.y + (size_t)p * a.cout + co);
          dst[0] = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                              pack_bf16x2(v[6], v[7]));
          dst[1] = make_uint4(pack_bf16x2(v[8], v[9]), pack_bf16x2(v[10], v[11]), pack_bf16x2(v[12], v[13]),
                              pack_bf16x2(v[14], v[15]));
        }
        if (a.yf) {
          float4 *dst = reinterpret_cast<float4 *>(a.yf + (size_t)p * a.cout + co);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores:
//   D[r][co] = sum_p X[p + tap(r)][ci(r)] dY[p][co],  r = tap * cin + ci
// M = 128 rows r per CTA, N = cout (<= 256), K = the CTA's pixel range in
// chunks of 64.  Both operands are MN-major (channels contiguous, as NHWC
// stores them): core matrix = 8 pixels (K) x 16 bytes (8 channels);
//   A: [pixel group h][row group g][pixel % 8] -> LBO (K) = 16 x 128 bytes, SBO (M) = 128
//   B: [pixel group h][cout group g][pixel % 8] -> LBO (K) = N / 8 x 128,   SBO (N) = 128
// One 16-byte cp.async per (pixel, 8-channel group); taps outside the image
// and pixels outside the range are zero-filled.  The CTA writes its partial
// sums to part[split][co][r] (plain stores; reduced in split order later).
// ---------------------------------------------------------------------------
constexpr int kWgK = 64;  // pixels per chunk

struct WgradArgs {
  const __nv_bfloat16 *x;
  int n, h, w, cin;
  const __nv_bfloat16 *dy;
  int cout;
  int pix_per_split;
  float *part;  // [split][cout * 9 * cin + cout]
  int *status;
};

__global__ void __launch_bounds__(kThreads) k_wgrad_tc(const WgradArgs a, const int N, const int S) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  constexpr uint32_t A_BYTES = kWgK * kTileM * 2;
  const uint32_t B_BYTES = (uint32_t)kWgK * N * 2;
  const uint32_t STAGE = A_BYTES + B_BYTES;
  const int NG = N / 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int P = a.n * a.h * a.w;
  const int Ncol = 9 * a.cin;
  const int r0 = blockIdx.x * kTileM, n0 = blockIdx.y * N;
  const int pb = blockIdx.z * a.pix_per_split, pe = min(P, pb + a.pix_per_split);
  const int nK = (pe - pb + kWgK - 1) / kWgK;
  int *status = a.status ? a.status : &g_conv_status;

  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;
  if (warp == 0) {
    tmem_alloc(&tmem_slot, ncols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], kProducers);
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

  if (warp < 4) {
    const int kk = tid % kWgK;   // this thread's pixel within a chunk
    const int g0 = tid / kWgK;   // first of its row / cout groups (stride 2)
    bool ok = true;
    for (int k = 0; k < nK; ++k) {
      const int s = k % S;
      if (k >= S && !mbar_wait(&empty_bar[s], (uint32_t)((k / S) - 1) & 1u)) {
        ok = false;
        break;
      }
      const int p = pb + k * kWgK + kk;
      const bool pv = p < pe;
      int pn = 0, ph = 0, pw = 0;
      if (pv) {
        pn = p / (a.h * a.w);
        const int rr = p - pn * a.h * a.w;
        ph = rr / a.w;
        pw = rr - ph * a.w;
      }
      const uint32_t sA = sbase + (uint32_t)s * STAGE;
      const uint32_t rowoff = (uint32_t)(kk >> 3) * (kTileM / 8 * 128) + (uint32_t)(kk & 7) * 16;
      for (int g = g0; g < kTileM / 8; g += 2) {
        const int r = r0 + 8 * g;
        const int tap = r / a.cin, ci = r - tap * a.cin;
        const int kh = tap / 3, kw = tap - kh * 3;
        const int hh = ph + kh - 1, ww = pw + kw - 1;
        const bool v = pv && r < Ncol && hh >= 0 && hh < a.h && ww >= 0 && ww < a.w;
        const __nv_bfloat16 *src = v ? a.x + (((size_t)pn * a.h + hh) * a.w + ww) * a.cin + ci : a.x;
        cp_async16(sA + rowoff + (uint32_t)g * 128, src, v ? 16u : 0u);
      }
      const uint32_t sB = sA + A_BYTES;
      const uint32_t boff = (uint32_t)(kk >> 3) * ((uint32_t)NG * 128) + (uint32_t)(kk & 7) * 16;
      for (int g = g0; g < NG; g += 2) {
        const int co = n0 + 8 * g;
        const bool v = pv && co < a.cout;
        const __nv_bfloat16 *src = v ? a.dy + (size_t)p * a.cout + co : a.dy;
        cp_async16(sB + boff + (uint32_t)g * 128, src, v ? 16u : 0u);
      }
      cp_async_commit();
      // keep S - 1 chunks in flight: wait for the oldest, publish it
      if (k >= S - 1) {
        cp_async_wait_pending(S - 1);
        fence_async_smem();
        mbar_arrive(&full_bar[(k - (S - 1)) % S]);
      }
    }
    cp_async_wait<0>();
    fence_async_smem();
    if (ok) {
      for (int j = std::max(0, nK - (S - 1)); j < nK; ++j) mbar_arrive(&full_bar[j % S]);
    } else {
      s_abort = 1;
    }
  } else if (warp == 4) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc(1u /* bf16 */, kTileM, (uint32_t)N) | (1u << 15) | (1u << 16);
      const uint32_t lboA = kTileM / 8 * 128, lboB = (uint32_t)NG * 128;
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
          const uint64_t ad = smem_desc(sA + (uint32_t)q * 2 * lboA, lboA, 128);
          const uint64_t bd = smem_desc(sB + (uint32_t)q * 2 * lboB, lboB, 128);
          mma_bf16(tmem, ad, bd, idesc, (k | q) != 0 ? 1u : 0u);
        }
        mma_commit(&empty_bar[s]);
      }
      mma_commit(&done_bar);
    }
    __syncwarp();
  }

  if (warp < 4) {
    __syncwarp();
    const bool done = mbar_wait(&done_bar, 0);
    tc_fence_after();
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
          // an empty range leaves the accumulator unwritten: store zeros
          if (co < a.cout) dst[(size_t)co * Ncol + r] = nK > 0 ? v[q] : 0.f;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// Bias gradient partials: out[b * cout + co] = sum over pixel block b of
// dY[p][co]; 8-channel groups x pixel phases per block, fixed-order tree
// over the phases.
constexpr int kBiasThreads = 256;
__global__ void __launch_bounds__(kBiasThreads)
    k_bias_part(const __nv_bfloat16 *__restrict__ dy, int P, int cout, int pix_per_block, float *__restrict__ out) {
  __shared__ float red[kBiasThreads][8];
  const int groups = cout / 8;                 // <= 32 (cout <= 256)
  const int phases = kBiasThreads / groups;
  const int g = threadIdx.x % groups, ph = threadIdx.x / groups;
  const int pb = blockIdx.x * pix_per_block, pe = min(P, pb + pix_per_block);
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (ph < phases)
    for (int p = pb + ph; p < pe; p += phases) {
      const uint4 v = *reinterpret_cast<const uint4 *>(dy + (size_t)p * cout + 8 * g);
      const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 f = __bfloat1622float2(h2[q]);
        acc[2 * q] += f.x;
        acc[2 * q + 1] += f.y;
      }
    }
#pragma unroll
  for (int q = 0; q < 8; ++q) red[threadIdx.x][q] = acc[q];
  __syncthreads();
  if ((int)threadIdx.x < groups) {
    float s8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int h = 0; h < phases; ++h)
#pragma unroll
      for (int q = 0; q < 8; ++q) s8[q] += red[h * groups + threadIdx.x][q];
#pragma unroll
    for (int q = 0; q < 8; ++q) out[(size_t)blockIdx.x * cout + 8 * threadIdx.x + q] = s8[q];
  }
}

template <int KC>
cudaError_t launch(const ConvArgs &a, int N, cudaStream_t s) {
  const size_t stage = (size_t)kTileM * KC * 2 + (size_t)N * KC * 2;
  const int S = ring_stages(stage);
  const size_t smem = (size_t)S * stage;
  cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int P = a.n * a.h * a.w;
  dim3 grid((P + kTileM - 1) / kTileM, (a.cout + N - 1) / N);
  k_conv3x3_tc<KC><<<grid, kThreads, smem, s>>>(a, N, S);
  return cudaGetLastError();
}

}  // namespace

// Tensor-core form of conv3x3 (same contract).  N per CTA = cout up to 256.
cudaError_t conv3x3_tc(const Tensor4 &x, const __nv_bfloat16 *w, int cout, const float *bias, bool relu,
                       __nv_bfloat16 *y, float *yf, int *status, cudaStream_t s) {
  cudaError_t err = cudaSuccess;
  if (conv3x3_tma(x, w, cout, bias, relu, y, yf, status, s, &err)) return err;
  ConvArgs a{x.p, x.n, x.h, x.w, x.c, w, cout, bias, relu ? 1 : 0, y, yf, status};
  // N per CTA: all output channels (up to 256), halved while the grid has
  // fewer than two CTAs per SM (low-resolution layers)
  int N = std::min(cout, kMaxN);
  const long tiles_m = ((long)x.n * x.h * x.w + kTileM - 1) / kTileM;
  while (N > 32 && N % 32 == 0 && tiles_m * ((cout + N - 1) / N) < 304) N /= 2;
  if (x.c % 64 == 0) return launch<64>(a, N, s);
  if (x.c % 32 == 0) return launch<32>(a, N, s);
  return launch<16>(a, N, s);  // cin is a multiple of 16
}

// Pixel splits of the weight gradient: about 2 x 152 CTAs in all (a fixed
// count, so that results do not depend on the device), at least 8 chunks of
// 64 pixels per split (fewer, larger partial sums for the low-resolution
// layers, whose weight tensors are the largest).
int wgrad_splits(const Tensor4 &x, int cout) {
  const int P = x.n * x.h * x.w;
  const int tiles = ((9 * x.c + kTileM - 1) / kTileM) * ((cout + kMaxN - 1) / kMaxN);
  int want = std::max(1, (304 + tiles - 1) / tiles);
  want = std::min(want, std::max(1, P / (8 * kWgK)));
  const int per = ((P + want - 1) / want + kWgK - 1) / kWgK * kWgK;
  return (P + per - 1) / per;
}

// pixel blocks of the bias partials: about 8 pixels per thread (256
// threads = cout / 8 channel groups x pixel phases), at most 2048 blocks
int bias_blocks(int pixels, int cout) {
  const long work = (long)pixels * (cout / 8);
  return (int)std::max<long>(1, std::min<long>(2048, (work + 2047) / 2048));
}

size_t wgrad_part_floats(const Tensor4 &x, int cout) {
  return (size_t)wgrad_splits(x, cout) * ((size_t)cout * 9 * x.c) +
         (size_t)bias_blocks(x.n * x.h * x.w, cout) * cout;
}

cudaError_t conv3x3_wgrad(const Tensor4 &x, const __nv_bfloat16 *dy, int cout, float *part, int *n_split,
                          int *n_bias, int *status, cudaStream_t s) {
  const int P = x.n * x.h * x.w;
  const int splits = wgrad_splits(x, cout);
  const int per = ((P + splits - 1) / splits + kWgK - 1) / kWgK * kWgK;
  const int N = std::min(cout, kMaxN);
  const int nb = bias_blocks(P, cout);
  const int bper = (P + nb - 1) / nb;
  float *bpart = part + (size_t)splits * cout * 9 * x.c;
  *n_split = splits;
  *n_bias = nb;
  cudaError_t err = cudaSuccess;
  if (wgrad_tma(x, dy, cout, part, splits, per, status, s, &err)) {
    if (err != cudaSuccess) return err;
    k_bias_part<<<nb, kBiasThreads, 0, s>>>(dy, P, cout, bper, bpart);
    return cudaGetLastError();
  }
  WgradArgs a{x.p, x.n, x.h, x.w, x.c, dy, cout, per, part, status};
  const size_t stage = (size_t)kWgK * kTileM * 2 + (size_t)kWgK * N * 2;
  const int S = ring_stages(stage);
  const size_t smem = (size_t)S * stage;
  cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((9 * x.c + kTileM - 1) / kTileM, (cout + N - 1) / N, splits);
  k_wgrad_tc<<<grid, kThreads, smem, s>>>(a, N, S);
  k_bias_part<<<nb, kBiasThreads, 0, s>>>(dy, P, cout, bper, bpart);
  return cudaGetLastError();
}

// status word of layer-level launches: read and reset
cudaError_t conv_status(int *out) {
  int zero = 0, t = 0;
  cudaError_t e = cudaMemcpyFromSymbol(out, g_conv_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_conv_status, &zero, sizeof(int));
  if (e == cudaSuccess) e = tma_status(&t);
  if (e == cudaSuccess && *out == 0) *out = t;
  return e;
}

}  // namespace nn
}  // namespace kk
