// kk_shear_tc.cu -- the far-field decomposition contraction on the 5th-
// generation tensor cores (tcgen05, TMEM accumulators): BF16, FP16 and
// FP8-e4m3 operand forms with FP32 accumulation.
//
// Per frequency bin k the decomposition is the complex product (Eq.
// (compression) applied through the Fourier shift theorem, Section II-F)
//     Y[k][i][o] = sum_l X[k][i][l] W[k][o][l],  W = exp(+2 pi i k phi[o][l]).
// It is run as a real GEMM D = A B^T with
//     A row (o, re) = [ Wr[o][l], -Wi[o][l] ]_l     A row (o, im) = [ Wi, Wr ]_l
//     B row i       = [ Xr[i][l],  Xi[i][l] ]_l     (K index = 2 l + component)
// so D[(o, re)][i] = Re Y, D[(o, im)][i] = Im Y.  B is the spectrum in its own
// interleaved layout; A is generated on chip from the shear phases rounded to
// 0.32 fixed-point turns (angle error < 8e-7 rad, far below these forms'
// operand rounding)
// (never stored in HBM).
//
// Each CTA (two warpgroups, two CTAs per SM) takes one bin at a time: it
// copies B into shared memory, then for each tile of 64 receive angles (128
// rows of A) generates A, one thread issues K/16 (K/32 for FP8) tcgen05.mma
// into a TMEM accumulator of 128 lanes x N columns, commits to an mbarrier,
// and the eight warps read the accumulator back (tcgen05.ld; warp w reads
// lane quarter w % 4) and store Y.
//
// Shared-memory operands use the no-swizzle K-major canonical layout: 8-row x
// 16-byte core matrices, K-adjacent core matrices 128 bytes apart (LBO), 8-row
// groups KC*ES/16*... apart (SBO = 16 bytes x K-cores x 8).
//
// FP8: the scale is per column (k, i) of X -- it factors out of the sum over
// elements; X is rounded to e4m3 as X / s with s = max_l |X| / 448, W is
// stored as 64 W (|W| <= 1, clear of e4m3 subnormals), and the FP32 result is
// multiplied by s / 64 in the epilogue.  Each operand is held as two e4m3
// terms, hi = e4m3(v) and lo = e4m3(v - hi), and the accumulator takes
// A_hi B_hi + A_hi B_lo + A_lo B_hi: one e4m3 term per operand (three mantissa
// bits) leaves the image about 2e-2 from the FP64 result, the two-term form
// about 5e-4.
//
// Every wait is bounded (%globaltimer): on timeout the CTA records
// KK_ERR_TIMEOUT in the plan's status word, frees its TMEM and returns.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kk_internal.h"
#include "kk_tc.h"
#include "kk_tma.h"

namespace kk {

namespace {

using namespace kk::tc;

constexpr int kTcThreads = 256;        // two warpgroups
constexpr int kKC = 256;                 // K elements per pass (128 array elements)
constexpr int kRowsM = 128;              // rows of A per tile (64 receive angles)
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}
__device__ __forceinline__ uint32_t pack_f16(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}
// two floats -> two e4m3 bytes (round to nearest, saturate), low byte = a
__device__ __forceinline__ uint32_t pack_e4m3x2(float a, float b) {
  uint16_t r;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(b), "f"(a));
  return r;
}

// two e4m3 bytes (low byte first) -> two floats (exact: e4m3 is a subset of f16)
__device__ __forceinline__ float2 e4m3x2_to_float2(uint32_t v) {
  uint32_t h;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h) : "h"((uint16_t)v));
  return __half22float2(*reinterpret_cast<const __half2 *>(&h));
}
// two-term e4m3 split of two floats: a ~ hi + lo with lo = e4m3(a - hi); the
// residual is exact in FP32 (hi lies within a factor two of a, or is zero)
__device__ __forceinline__ void split_e4m3x2(float a, float b, uint32_t &hi, uint32_t &lo) {
  hi = pack_e4m3x2(a, b);
  const float2 h = e4m3x2_to_float2(hi);
  lo = pack_e4m3x2(a - h.x, b - h.y);
}

template <int KIND>
struct Fmt {
  static constexpr int ES = (KIND == 2) ? 1 : 2;        // bytes per operand element
  static constexpr int KSTEP = (KIND == 2) ? 32 : 16;   // K per MMA instruction
  static constexpr uint32_t code = (KIND == 0) ? 1u : 0u;  // BF16 = 1, F16 = 0, E4M3 = 0
  static constexpr int EPC = 16 / ES;                   // elements per 16-byte core row
};

// byte offset of element (row, k) in a K-major no-swizzle tile of kKC columns
template <int ES>
__device__ __forceinline__ uint32_t core_off(int row, int kbyte) {
  constexpr uint32_t SBO = (uint32_t)(kKC * ES / 16) * 128u;
  return (uint32_t)(row >> 3) * SBO + (uint32_t)(kbyte >> 4) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(kbyte & 15);
}

// ---- pipelined form (BF16 / FP16, up to 96 transmits) -----------------------
// One persistent CTA per SM walks its bins; each bin is ceil(Mu / 64) items
// (tiles of 128 rows of A).  Operands use the 128-byte-swizzled K-major
// layout in chunks of 64 elements (128 rows / NP rows x 128 bytes, 16-byte
// units XOR-ed with the row index within each 8-row group):
//   B (the bin's spectrum rows) by 2D bulk copies of the [F * Nu][2L] spectra,
//     box {64, NP}, into two stages one bin ahead (rows past Nu are the next
//     bin's and only reach discarded outputs; past the last bin they are the
//     copy's zero fill);
//   A generated on chip from the shear phases (0.32 fixed-point turns).
// Arithmetic and K order equal k_shear_tc's.  The work is split over warp
// roles that meet only at mbarriers (no CTA-wide barrier in the main loop):
//   * 16 producer warps generate A one 64-element K chunk (128 rows x 128
//     bytes) at a time into a ring of kT3Slots chunk slots (two tiles), from
//     shear phases read through the cache (the ring leaves no room for them);
//   * one thread issues the bins' 2D bulk copies of B (up to four stages, as
//     many bins ahead as shared memory holds) and, per chunk, the four MMAs, committing each chunk's slot back
//     to the producers and each item's accumulator to the epilogue;
//   * 8 epilogue warps read the TMEM accumulators (up to four, in turn) and store Y.
constexpr int kT3MaxNP = 96;
// A producer reuses a slot after the MMAs that read it have completed; the
// issuer starts an item's MMAs once its accumulator has been drained.
// Every wait is bounded; a role that gives up raises the CTA's abort flag,
// which every other wait also watches.
constexpr int kT3Producers = 512;
constexpr int kT3Epi = 256;
constexpr int kT3Threads = kT3Producers + 32 + kT3Epi;
constexpr int kT3Slots = 8;
constexpr int kT3MaxB = 4;   // B stages (bins in flight), as many as shared memory holds
constexpr int kT3MaxAcc = 4;

template <int KIND>
__global__ void __launch_bounds__(kT3Threads, 1)
    k_shear_tc3(const __grid_constant__ CUtensorMap xmap, const uint32_t *__restrict__ phase, int F, int L,
                int Nu, int Mu, int NP, int nb, float yscale, float2 *__restrict__ Y, int *__restrict__ status) {
  static_assert(KIND == 0 || KIND == 1, "BF16 / FP16 forms");
  constexpr uint32_t CH_BYTES = (uint32_t)kRowsM * 128u;  // one chunk of A: 16 KB
  constexpr uint32_t SBO = 1024u;                         // 8 rows x 128 bytes
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t afull[kT3Slots], aempty[kT3Slots], bfull[kT3MaxB], bempty[kT3MaxB], accfull[kT3MaxAcc],
      accempty[kT3MaxAcc], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nch = (2 * L + 63) / 64;                       // chunks holding data (<= 4)
  const uint32_t B_BYTES = (uint32_t)nch * (uint32_t)NP * 128u;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t sA = sbase;                               // ring of chunk slots
  const uint32_t sB0 = sbase + kT3Slots * CH_BYTES;        // nb B stages
  const int ntile = (Mu + kRowsM / 2 - 1) / (kRowsM / 2);
  const int nbins = (int)blockIdx.x < F ? (F - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nitems = nbins * ntile;
  uint32_t ncols = 32;
  while ((int)ncols < NP) ncols <<= 1;
  // as many accumulators as the SM's 512 TMEM columns hold (up to four), so
  // the MMAs can run that many tiles ahead of the epilogue
  const int nacc = (int)min(512u / ncols, (uint32_t)kT3MaxAcc);
  if (warp == 0) {
    tmem_alloc(&tmem_slot, nacc * ncols);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int q = 0; q < kT3Slots; ++q) {
      mbar_init(&afull[q], kT3Producers / 32);   // one arrival per producer warp
      mbar_init(&aempty[q], 1);
    }
    for (int q = 0; q < kT3MaxB; ++q) {
      mbar_init(&bfull[q], 1);
      mbar_init(&bempty[q], 1);
    }
    for (int q = 0; q < kT3MaxAcc; ++q) {
      mbar_init(&accfull[q], 1);
      mbar_init(&accempty[q], kT3Epi / 32);      // one arrival per epilogue warp
    }
    mbar_init(&drain, 1);
    s_abort = 0;
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int *abort_flag = &s_abort;
  // bounded wait that also gives up when another role has aborted
  auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
    if (mbar_try_wait(bar, parity)) return true;  // the timer is read only when the wait is real
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity)) {
      if (*abort_flag || globaltimer() - t0 > kWaitNs) {
        *abort_flag = 1;
        return false;
      }
    }
    return true;
  };
  auto bin_of = [&](int jj) { return (int)blockIdx.x + jj * (int)gridDim.x; };
  if (warp < kT3Producers / 32) {
    // ---- producers: chunk c of item n's A into slot (n nch + c) % kT3Slots;
    // thread = (row pair ol, 16-byte unit u) of a chunk; two chunks per step
    // (eight W values in flight) ----
    const int ol = tid >> 3, u = tid & 7;
    const int R0 = 2 * ol, R1 = R0 + 1;
    bool ok = true;
    for (int n = 0; ok && n < nitems; ++n) {
      const int jj = n / ntile, t = n - jj * ntile;
      const uint32_t k32 = (uint32_t)bin_of(jj);
      const int o = t * (kRowsM / 2) + ol;
      for (int c = 0; ok && c < nch; c += 2) {
        const int nc2 = min(2, nch - c);
        uint4 re[2], im[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int l0 = 32 * (c + h) + 4 * u;
          uint4 p4 = make_uint4(0u, 0u, 0u, 0u);
          if (h < nc2 && o < Mu && l0 < L) p4 = __ldg(reinterpret_cast<const uint4 *>(phase + (size_t)o * L + l0));
          const uint32_t ph4[4] = {p4.x, p4.y, p4.z, p4.w};
          float wr[4], wi[4];
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            wr[qq] = wi[qq] = 0.f;
            if (h < nc2 && o < Mu && l0 + qq < L) {
              const uint32_t ph = ph4[qq] * k32;                            // k phi mod 1 turn
              const float ang = (float)(int)ph * 1.4629180792671596e-09f;  // 2 pi / 2^32
              float sn, cs;
              __sincosf(ang, &sn, &cs);
              wr[qq] = cs;
              wi[qq] = sn;
            }
          }
          if constexpr (KIND == 0) {
            re[h] = make_uint4(pack_bf16(wr[0], -wi[0]), pack_bf16(wr[1], -wi[1]), pack_bf16(wr[2], -wi[2]),
                               pack_bf16(wr[3], -wi[3]));
            im[h] = make_uint4(pack_bf16(wi[0], wr[0]), pack_bf16(wi[1], wr[1]), pack_bf16(wi[2], wr[2]),
                               pack_bf16(wi[3], wr[3]));
          } else {
            re[h] = make_uint4(pack_f16(wr[0], -wi[0]), pack_f16(wr[1], -wi[1]), pack_f16(wr[2], -wi[2]),
                               pack_f16(wr[3], -wi[3]));
            im[h] = make_uint4(pack_f16(wi[0], wr[0]), pack_f16(wi[1], wr[1]), pack_f16(wi[2], wr[2]),
                               pack_f16(wi[3], wr[3]));
          }
        }
        for (int h = 0; h < nc2; ++h) {
          const int q = n * nch + c + h, s = q % kT3Slots;
          if (q >= kT3Slots) {
            // one lane waits for the slot, the warp follows its answer
            bool got = lane == 0 ? wait(&aempty[s], (uint32_t)((q / kT3Slots) - 1) & 1u) : true;
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!(ok = got)) break;
          }
          unsigned char *base = smem + (size_t)s * CH_BYTES;
          *reinterpret_cast<uint4 *>(base + R0 * 128 + ((u ^ (R0 & 7)) << 4)) = re[h];
          *reinterpret_cast<uint4 *>(base + R1 * 128 + ((u ^ (R1 & 7)) << 4)) = im[h];
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&afull[s]);
        }
      }
    }
  } else if (warp == kT3Producers / 32) {
    // ---- one thread: copies of B and the MMAs ----
    if (lane == 0) {
      const uint32_t idesc = instr_desc(Fmt<KIND>::code, kRowsM, (uint32_t)NP);
      auto issue_b = [&](int jj) {
        const uint32_t dst = sB0 + (uint32_t)(jj % nb) * B_BYTES;
        tma::mbar_expect_tx(&bfull[jj % nb], B_BYTES);
        for (int c = 0; c < nch; ++c)
          tma::tma_2d(dst + (uint32_t)c * (uint32_t)NP * 128u, &xmap, 64 * c, bin_of(jj) * Nu, &bfull[jj % nb]);
      };
      int issued = 0, waited = 0;
      while (issued < nb && issued < nbins) issue_b(issued++);
      bool ok = true;
      for (int jj = 0; ok && jj < nbins; ++jj) {
        if (jj >= 1 && jj + nb - 1 < nbins) {
          // stage (jj - 1) % nb held bin jj - 1: refill it with bin jj + nb - 1
          // once that bin's MMAs are done
          if (!(ok = wait(&bempty[(jj - 1) % nb], (uint32_t)((jj - 1) / nb) & 1u))) break;
          issue_b(issued++);
        }
        if (!(ok = wait(&bfull[jj % nb], (uint32_t)(jj / nb) & 1u))) break;
        waited = jj + 1;
        const uint32_t sB = sB0 + (uint32_t)(jj % nb) * B_BYTES;
        for (int t = 0; ok && t < ntile; ++t) {
          const int n = jj * ntile + t;
          if (n >= nacc && !(ok = wait(&accempty[n % nacc], (uint32_t)((n / nacc) - 1) & 1u))) break;
          const uint32_t acc = tmem + (uint32_t)(n % nacc) * ncols;
          for (int c = 0; ok && c < nch; ++c) {
            const int q = n * nch + c, s = q % kT3Slots;
            if (!(ok = wait(&afull[s], (uint32_t)(q / kT3Slots) & 1u))) break;
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t ad = smem_desc(sA + (uint32_t)s * CH_BYTES + (uint32_t)ks * 32u, 16, SBO) | (2ull << 61);
              const uint64_t bd =
                  smem_desc(sB + (uint32_t)c * (uint32_t)NP * 128u + (uint32_t)ks * 32u, 16, SBO) | (2ull << 61);
              mma<KIND>(acc, ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
            }
            mma_commit(&aempty[s]);
          }
          if (ok) mma_commit(&accfull[n % nacc]);
        }
        if (ok) mma_commit(&bempty[jj % nb]);
      }
      // every MMA this thread issued has completed (bounded), and so has
      // every copy it issued, before the CTA frees TMEM and exits
      mma_commit(&drain);
      mbar_wait(&drain, 0u);
      if (!ok) {
        atomicExch(status, (int)KK_ERR_TIMEOUT);
        for (int jb = waited; jb < issued; ++jb) mbar_wait(&bfull[jb % nb], (uint32_t)(jb / nb) & 1u);
      }
    }
  } else {
    // ---- epilogue: warp reads TMEM lane quarter warp % 4, column half ew / 4 ----
    const int ew = warp - (kT3Producers / 32 + 1);
    const int quarter = warp & 3, half = ew >> 2;
    const int r = quarter * 32 + lane;
    for (int n = 0; n < nitems; ++n) {
      const int jj = n / ntile, t = n - jj * ntile;
      const int k = bin_of(jj);
      bool ok = lane == 0 ? wait(&accfull[n % nacc], (uint32_t)(n / nacc) & 1u) : true;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      tc_fence_after();
      const int o = t * (kRowsM / 2) + (r >> 1), part = r & 1;
      const uint32_t trow = tmem + (uint32_t)(n % nacc) * ncols + ((uint32_t)(quarter * 32) << 16);
      float *Yf = reinterpret_cast<float *>(Y + (size_t)k * Nu * Mu);
      for (int c0 = 16 * half; c0 < NP; c0 += 32) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
        for (int qq = 0; qq < 16; ++qq) {
          const int i = c0 + qq;
          if (i < Nu && o < Mu) Yf[((size_t)i * Mu + o) * 2 + part] = v[qq] * yscale;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[n % nacc]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, nacc * ncols);
}

template <int KIND>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_shear_tc(const void *__restrict__ Xv, const uint32_t *__restrict__ phase, int F,
               int L, int Nu, int Mu, int NP, float yscale, float2 *__restrict__ Y,
               int *__restrict__ status) {
  using FM = Fmt<KIND>;
  constexpr int ES = FM::ES;
  constexpr uint32_t LBO = 128u;
  constexpr uint32_t SBO = (uint32_t)(kKC * ES / 16) * 128u;
  extern __shared__ __align__(1024) unsigned char smem[];
  // FP8 holds each operand as two terms (hi, lo): A_hi, A_lo, B_hi, B_lo
  constexpr int NT = (KIND == 2) ? 2 : 1;
  unsigned char *sA = smem;                                   // NT x kRowsM x kKC elements
  unsigned char *sB = smem + (size_t)NT * kRowsM * kKC * ES;  // NT x NP x kKC elements
  [[maybe_unused]] unsigned char *sAl = sA + (size_t)kRowsM * kKC * ES;
  [[maybe_unused]] unsigned char *sBl = sB + (size_t)NP * kKC * ES;
  float *sScale = reinterpret_cast<float *>(sB + (size_t)NT * NP * kKC * ES);  // [NP] (FP8)
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint32_t ncols = 32;
  while ((int)ncols < NP) ncols <<= 1;

  if (warp == 0) {
    tmem_alloc(&tmem_slot, ncols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = instr_desc(FM::code, kRowsM, (uint32_t)NP);
  uint32_t phase_bit = 0;
  bool ok = true;

  for (int k = blockIdx.x; k < F && ok; k += gridDim.x) {
    // ---- B: X[k][i][l] for i < NP (zero rows beyond Nu), l < L ----
    if constexpr (KIND == 2) {
      // FP16 spectra -> per-column scale -> e4m3
      const __half2 *Xk = reinterpret_cast<const __half2 *>(Xv) + (size_t)k * Nu * L;
      for (int i = warp; i < NP; i += kTcThreads / 32) {
        float m = 0.f;
        if (i < Nu)
          for (int l = lane; l < L; l += 32) {
            const float2 v = __half22float2(Xk[(size_t)i * L + l]);
            m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
          }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const float s = (m > 0.f) ? m / 448.f : 1.f;
        const float inv = 1.f / s;
        if (lane == 0) sScale[i] = s;
        // 16-byte core rows: 8 complex elements each
        for (int c = lane; c < kKC / 16; c += 32) {
          uint32_t w[4], wl[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int l0 = c * 8 + 2 * q;
            float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
            if (i < Nu && l0 < L) a = __half22float2(Xk[(size_t)i * L + l0]);
            if (i < Nu && l0 + 1 < L) b = __half22float2(Xk[(size_t)i * L + l0 + 1]);
            uint32_t ha, la, hb, lb;
            split_e4m3x2(a.x * inv, a.y * inv, ha, la);
            split_e4m3x2(b.x * inv, b.y * inv, hb, lb);
            w[q] = ha | (hb << 16);
            wl[q] = la | (lb << 16);
          }
          *reinterpret_cast<uint4 *>(sB + core_off<1>(i, c * 16)) = make_uint4(w[0], w[1], w[2], w[3]);
          *reinterpret_cast<uint4 *>(sBl + core_off<1>(i, c * 16)) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
        }
      }
    } else {
      // BF16 / FP16 spectra: one complex value is 4 bytes, so a 16-byte core
      // row holds 4 consecutive complex X
      const uint32_t *Xk = reinterpret_cast<const uint32_t *>(Xv) + (size_t)k * Nu * L;
      const bool vec = (L & 3) == 0;
#pragma unroll 4
      for (int e = tid; e < NP * (kKC / 8); e += kTcThreads) {
        const int i = e / (kKC / 8), c = e - i * (kKC / 8);
        const int l0 = c * 4;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (i < Nu && l0 < L) {
          if (vec) {
            v = *reinterpret_cast<const uint4 *>(Xk + (size_t)i * L + l0);
          } else {
            uint32_t t[4] = {0u, 0u, 0u, 0u};
            for (int q = 0; q < 4; ++q)
              if (l0 + q < L) t[q] = Xk[(size_t)i * L + l0 + q];
            v = make_uint4(t[0], t[1], t[2], t[3]);
          }
        }
        *reinterpret_cast<uint4 *>(sB + core_off<2>(i, c * 16)) = v;
      }
    }

    const uint32_t k32 = (uint32_t)k;
    const bool vecph = (L & 3) == 0;
    for (int m0 = 0; m0 < Mu && ok; m0 += kRowsM / 2) {
      // ---- A: rows (o, re) / (o, im) of W for o in [m0, m0 + 64) ----
      constexpr int EPC = FM::EPC;                       // elements per core row
      constexpr int LPR = EPC / 2;                       // array elements per core row
      const float wscale = (KIND == 2) ? 64.f : 1.f;
#pragma unroll 2
      for (int e = tid; e < (kRowsM / 2) * (kKC / EPC); e += kTcThreads) {
        const int ol = e / (kKC / EPC), c = e - ol * (kKC / EPC);
        const int o = m0 + ol;
        float wr[LPR], wi[LPR];
        uint32_t ph32[LPR];
        const int l0 = c * LPR;
        if (o < Mu && vecph && l0 + LPR <= L) {
          // LPR consecutive phases with 16-byte loads (row starts are 16-byte aligned)
          const uint4 *src = reinterpret_cast<const uint4 *>(phase + (size_t)o * L + l0);
#pragma unroll
          for (int h = 0; h < LPR / 4; ++h) {
            const uint4 u = __ldg(src + h);
            ph32[4 * h] = u.x;
            ph32[4 * h + 1] = u.y;
            ph32[4 * h + 2] = u.z;
            ph32[4 * h + 3] = u.w;
          }
        } else {
#pragma unroll
          for (int q = 0; q < LPR; ++q)
            ph32[q] = (o < Mu && l0 + q < L) ? __ldg(phase + (size_t)o * L + l0 + q) : 0u;
        }
#pragma unroll
        for (int q = 0; q < LPR; ++q) {
          const int l = l0 + q;
          wr[q] = wi[q] = 0.f;
          if (o < Mu && l < L) {
            const uint32_t ph = ph32[q] * k32;  // k phi mod 1 turn, 0.32 fixed point
            const float ang = (float)(int)ph * 1.4629180792671596e-09f;  // 2 pi / 2^32
            float sn, cs;
            __sincosf(ang, &sn, &cs);
            wr[q] = cs * wscale;
            wi[q] = sn * wscale;
          }
        }
        uint4 re, im;
        if constexpr (KIND == 2) {
          uint32_t r4[4], i4[4], rl4[4], il4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t h0, l0_, h1, l1, g0, m0_, g1, m1;
            split_e4m3x2(wr[2 * q], -wi[2 * q], h0, l0_);
            split_e4m3x2(wr[2 * q + 1], -wi[2 * q + 1], h1, l1);
            split_e4m3x2(wi[2 * q], wr[2 * q], g0, m0_);
            split_e4m3x2(wi[2 * q + 1], wr[2 * q + 1], g1, m1);
            r4[q] = h0 | (h1 << 16);
            rl4[q] = l0_ | (l1 << 16);
            i4[q] = g0 | (g1 << 16);
            il4[q] = m0_ | (m1 << 16);
          }
          re = make_uint4(r4[0], r4[1], r4[2], r4[3]);
          im = make_uint4(i4[0], i4[1], i4[2], i4[3]);
          *reinterpret_cast<uint4 *>(sAl + core_off<ES>(2 * ol, c * 16)) = make_uint4(rl4[0], rl4[1], rl4[2], rl4[3]);
          *reinterpret_cast<uint4 *>(sAl + core_off<ES>(2 * ol + 1, c * 16)) = make_uint4(il4[0], il4[1], il4[2], il4[3]);
        } else if constexpr (KIND == 0) {
          re = make_uint4(pack_bf16(wr[0], -wi[0]), pack_bf16(wr[1], -wi[1]), pack_bf16(wr[2], -wi[2]),
                          pack_bf16(wr[3], -wi[3]));
          im = make_uint4(pack_bf16(wi[0], wr[0]), pack_bf16(wi[1], wr[1]), pack_bf16(wi[2], wr[2]),
                          pack_bf16(wi[3], wr[3]));
        } else {
          re = make_uint4(pack_f16(wr[0], -wi[0]), pack_f16(wr[1], -wi[1]), pack_f16(wr[2], -wi[2]),
                          pack_f16(wr[3], -wi[3]));
          im = make_uint4(pack_f16(wi[0], wr[0]), pack_f16(wi[1], wr[1]), pack_f16(wi[2], wr[2]),
                          pack_f16(wi[3], wr[3]));
        }
        *reinterpret_cast<uint4 *>(sA + core_off<ES>(2 * ol, c * 16)) = re;
        *reinterpret_cast<uint4 *>(sA + core_off<ES>(2 * ol + 1, c * 16)) = im;
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        const int ksteps = (2 * L + FM::KSTEP - 1) / FM::KSTEP;
        // FP8: A_hi B_hi + A_hi B_lo + A_lo B_hi into one accumulator (the
        // lo x lo term is below the accumulation's own rounding)
#pragma unroll 1
        for (int t = 0; t < (KIND == 2 ? 3 : 1); ++t) {
          const uint32_t at = a0 + (t == 2 ? (uint32_t)(kRowsM * kKC * ES) : 0u);
          const uint32_t bt = b0 + (t == 1 ? (uint32_t)(NP * kKC * ES) : 0u);
#pragma unroll 1
          for (int s = 0; s < ksteps; ++s) {
            const uint32_t koff = (uint32_t)s * (FM::KSTEP * ES / 16) * LBO;
            mma<KIND>(tmem, smem_desc(at + koff, LBO, SBO), smem_desc(bt + koff, LBO, SBO), idesc,
                      (s > 0 || t > 0) ? 1u : 0u);
          }
        }
        mma_commit(&mbar);
      }
      // all threads wait for the accumulator
      const bool done = mbar_wait(&mbar, phase_bit);
      phase_bit ^= 1u;
      if (!done) {
        s_abort = 1;
        ok = false;
      }
      __syncthreads();
      if (s_abort) {
        ok = false;
        if (tid == 0) atomicExch(status, (int)KK_ERR_TIMEOUT);
        // wait (bounded) for the MMAs still in flight before TMEM is freed
        mbar_wait(&mbar, phase_bit ^ 1u);
        break;
      }
      tc_fence_after();
      // ---- epilogue: warp w reads TMEM lane quarter w % 4 (rows r = 32 (w % 4)
      // + lane -> (o, re|im)) and every other 16-column chunk from w / 4 ----
      const int quarter = warp & 3, half = warp >> 2;
      const int r = quarter * 32 + lane;
      const int o = m0 + (r >> 1), part = r & 1;
      const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
      float *Yf = reinterpret_cast<float *>(Y + (size_t)k * Nu * Mu);
      for (int c0 = 16 * half; c0 < NP; c0 += 32) {
        float v[16];
        tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int i = c0 + q;
          if (i < Nu && o < Mu) {
            float val = v[q] * yscale;
            if constexpr (KIND == 2) val *= sScale[i] * (1.f / 64.f);
            Yf[((size_t)i * Mu + o) * 2 + part] = val;
          }
        }
      }
      tc_fence_before();
      __syncthreads();  // accumulator read and A free before the next tile
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace

size_t tc_shear_smem_bytes(int precision, int NP) {
  const int ES = (precision == KK_PREC_F8E4M3) ? 1 : 2;
  const int NT = (precision == KK_PREC_F8E4M3) ? 2 : 1;   // FP8: hi and lo terms
  return (size_t)NT * kRowsM * kKC * ES + (size_t)NT * NP * kKC * ES + sizeof(float) * NP;
}

// spectra [F * Nu][2 L] 16-bit elements, box {64, NP}, 128-byte swizzle
static bool map_x(CUtensorMap *m, const void *X, int F, int Nu, int L, int NP, bool bf16) {
  tma::EncodeFn enc = tma::encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * L), (cuuint64_t)F * (cuuint64_t)Nu};
  const cuuint64_t strides[1] = {(cuuint64_t)(4 * L)};
  const cuuint32_t box[2] = {64, (cuuint32_t)NP};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(X),
             dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_shear_tc(const kk_plan &p, const void *X, float2 *Y, cudaStream_t s) {
  const int NP = ((p.Nu + 15) / 16) * 16;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
  if ((p.precision == KK_PREC_BF16 || p.precision == KK_PREC_F16) && NP <= kT3MaxNP && p.L % 4 == 0 &&
      ((uintptr_t)X % 16) == 0) {
    CUtensorMap m;
    if (map_x(&m, X, p.F, p.Nu, p.L, NP, p.precision == KK_PREC_BF16)) {
      const int nch = (2 * p.L + 63) / 64;
      const size_t bbytes = (size_t)nch * NP * 128;
      const size_t amax = (size_t)kT3Slots * kRowsM * 128;
      const int nb = (int)std::min<size_t>(kT3MaxB, (227 * 1024 - 1024 - amax) / bbytes);
      const size_t smem3 = amax + (size_t)nb * bbytes;
      const int grid3 = std::min(p.F, sms);
      auto k = p.precision == KK_PREC_BF16 ? k_shear_tc3<0> : k_shear_tc3<1>;
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3);
      if (e != cudaSuccess) return e;
      k<<<grid3, kT3Threads, smem3, s>>>(m, p.t.phase32, p.F, p.L, p.Nu, p.Mu, NP, nb, 1.f / p.x_scale, Y,
                                         p.t.status);
      return cudaGetLastError();
    }
  }
  const size_t smem = tc_shear_smem_bytes(p.precision, NP);
  const int grid = std::min(p.F, 2 * sms);
  cudaError_t e;
  switch (p.precision) {
    case KK_PREC_BF16: {
      auto k = k_shear_tc<0>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k<<<grid, kTcThreads, smem, s>>>(X, p.t.phase32, p.F, p.L, p.Nu, p.Mu, NP, 1.f / p.x_scale, Y,
                                       p.t.status);
      break;
    }
    case KK_PREC_F16: {
      auto k = k_shear_tc<1>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k<<<grid, kTcThreads, smem, s>>>(X, p.t.phase32, p.F, p.L, p.Nu, p.Mu, NP, 1.f / p.x_scale, Y,
                                       p.t.status);
      break;
    }
    case KK_PREC_F8E4M3: {
      auto k = k_shear_tc<2>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k<<<grid, kTcThreads, smem, s>>>(X, p.t.phase32, p.F, p.L, p.Nu, p.Mu, NP, 1.f / p.x_scale, Y,
                                       p.t.status);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace kk
