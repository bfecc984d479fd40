// kk_internal.h -- plan layout and launch declarations shared by the library's
// translation units.  Not part of the public ABI (see include/kkbeam.h).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/kkbeam.h"

namespace kk {

// Tile of the gather kernels: 32 pixels along x (one warp, lane = x offset)
// by 32 along z (4 warps x 8 rows per thread).
constexpr int kTileX = 32;
constexpr int kTileZ = 32;
constexpr int kRowsPerThread = 8;
constexpr int kGatherThreads = 128;

// 1.5 * 2^23: adding it with round-down leaves floor(s) in the low mantissa
// bits for |s| < 2^22.
constexpr float kFloorMagic = 12582912.0f;
constexpr int kFloorMagicBits = 0x4B400000;

// Supported FFT lengths for the analytic spectrum (F = T/2 points, complex).
bool fft_size_supported(int F);

// Radix plan of an F-point Stockham FFT: radices applied in order, each pass
// with Ns = product of earlier radices, twiddle table offsets per pass.
struct FftPlan {
  int F = 0;
  int npass = 0;
  int radix[12] = {};
  int ns[12] = {};
  int tw_off[12] = {};
  int tw_count = 0;
};
FftPlan make_fft_plan(int F);

// Device-side plan tables, all inside one allocation.
struct DevTables {
  // FFT
  float2 *fft_tw = nullptr;   // Stockham twiddles e^{-2 pi i r k / (Ns R)}
  float2 *rfft_w = nullptr;   // [F] e^{-2 pi i k / T}
  int32_t *tx_used = nullptr; // [Nu] row of rf for used transmit iu
  // decomposition
  unsigned long long *phase = nullptr; // [Mu][L] frac(D/T) * 2^64
  uint32_t *phase32 = nullptr;         // [Mu][L] the same, rounded to 0.32 turns (tensor-core forms)
  // separable volumetric contraction: per-bin phasors of the two axes
  // ([F][Wf [Lf][Mf] padded to even, Ws [Ls][parts * osn] zero padded]),
  // element slot in the staged grid, column of Y per receive combination
  float2 *sep_w = nullptr;
  int32_t *sep_slot = nullptr;         // [L] ls Lf + lf (f: the grid axis listed fastest)
  int32_t *sep_col = nullptr;          // [Ms][Mf] receive position (0..Mu-1)
  int32_t *pair_q = nullptr;           // [P] (caller order) column of Y
  // KK gather (pairs in group-sorted order)
  int32_t *bf_row = nullptr;           // [P] row of rf_theta
  long long *bf_A = nullptr, *bf_B = nullptr, *bf_C = nullptr; // 32.32 samples
  long long *bf_Y = nullptr;           // [P] 32.32 samples per y slice (volumetric)
  float *bf_Af = nullptr, *bf_Bf = nullptr;                    // samples per pixel
  float *pair_w = nullptr;             // [P] pair weights, caller's order (null: all 1)
  int32_t *group_start = nullptr;      // [J+1]
  // per rf_theta row (caller's pair order): the samples [lo, hi) the gather
  // can stage under any launch shape (linear-array KK plans)
  int2 *rec_range = nullptr;
  // DAS
  long long *das_A = nullptr, *das_B = nullptr, *das_C = nullptr; // [N] tau_in 32.32
  float *das_Af = nullptr, *das_Bf = nullptr;                     // [N]
  float2 *xs = nullptr;                // [nx] x fs / c as (hi, lo)
  float2 *zs = nullptr;                // [nz] z fs / c as (hi, lo)
  float2 *us = nullptr;                // [L]  u fs / c as (hi, lo)
  // volumetric DAS: transmit delay step per y slice (32.32), slice y and
  // element y (fs / c, as (hi, lo))
  long long *das_Y = nullptr;          // [N]
  float2 *ys = nullptr;                // [ny]
  float2 *us_y = nullptr;              // [L]
  int *status = nullptr;               // device status word (KK_OK or KK_ERR_TIMEOUT)
};

}  // namespace kk

struct kk_plan {
  bool is_das = false;
  int device = 0;
  int L = 0, N = 0, T = 0, F = 0, P = 0, J = 1, Nu = 0, Mu = 0;
  int compound = KK_COMPOUND_NONE;
  int rf_dtype = KK_RF_F32;
  int precision = KK_PREC_F32;
  kk_grid grid{};
  double c = 0, fs = 0;
  kk::FftPlan fft;
  kk::DevTables t;
  void *dev_block = nullptr;     // the one allocation holding DevTables
  size_t status_off = 0;
  std::vector<int32_t> h_group_start;
  // host copies of the pair tables (caller's pair order), for the streaming
  // decomposition: transmit position (0..Nu-1), receive position (0..Mu-1),
  // pair weight (empty without weights); used transmit rows (ascending)
  std::vector<int32_t> h_pair_tu, h_pair_ou, h_tx_used;
  std::vector<float> h_pair_w;
  // gather kernel configuration
  int bf_rows = 8;     // z rows per thread: tile = 32 x (4 * bf_rows) pixels
  int bf_win = 0;      // window entries staged per pair / channel
  int bf_stage = 0;    // pairs (KK) or transmits (DAS) per stage
  int bf_split = 1;    // pair-range splits (KK), partial images reduced after
  bool trim = false;   // the inverse stores only each record's rec_range
  size_t trim_bytes = 0;  // bytes the trimmed records store (16-byte sample pairs)
  int tiles_x = 0, tiles_z = 0;
  std::vector<double> h_bfA, h_bfB;  // per-pair delay slopes (samples per pixel)
  // workspace layout (bytes from the workspace base)
  size_t ws_X = 0, ws_Y = 0, ws_part = 0, ws_total = 0;
  double compression = 0;
  // FP16-stored spectra (F16 and F8E4M3 forms) are scaled by an exact power
  // of two, 2^-ceil(log2(2T)), so |X| <= 2 T 32768 stays below the FP16
  // maximum; the contraction's epilogue multiplies by 1 / x_scale
  float x_scale = 1.f;
  // DAS receive aperture: 2 F (0 = full aperture) and window (kk_aperture)
  float das_two_f = 0.f;
  int das_window = KK_APERTURE_BOXCAR;
  // volumetric plan: ny y-slices at y0 + iy dy, per-pair y slope of the
  // delay in bf_Y (32.32 samples per slice)
  bool vol = false;
  int ny = 1;
  // pair q's record comes from column q of Y (pairs listed transmit-major
  // over every used (transmit, receive) combination): the inverse needs no
  // column table and can stream Y tiles by TMA
  bool pair_q_identity = false;
  double y0 = 0, dy = 0;
  // separable FP32 contraction (0: the full form): element grid Lx x Ly,
  // receive product Mx x My, transmits per item; the elements are listed
  // y-fastest (else x-fastest, or in another order when not bulk)
  int sep_Lx = 0, sep_Ly = 0, sep_Mx = 0, sep_My = 0, sep_tpc = 0;
  bool sep_yfast = false, sep_bulk = false;
};

namespace kk {

// NVTX range over a host scope: the stages a call enqueues show up by name in
// a profiler's timeline (nvtx3 is header-only; with no tool attached a push
// or pop is one test of a function pointer).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Bounds-checked build: KK_IN_BOUNDS(counter, ok) counts a failed index check
// in the translation unit's device counter and yields ok (the caller skips
// the access); in the product build it is the constant true and the check is
// not compiled.  Each file with checks keeps its own counter, taken (read and
// reset) by the host functions below.
#ifdef KK_DEBUG_BOUNDS
#define KK_IN_BOUNDS(counter, ok) ::kk::bound_check(&(counter), (ok))
#ifdef __CUDACC__
__device__ __forceinline__ bool bound_check(unsigned *counter, bool ok) {
  if (!ok) atomicAdd(counter, 1u);
  return ok;
}
#endif
cudaError_t take_bounds_kk(unsigned long long *n);
cudaError_t take_bounds_das(unsigned long long *n);
#else
#define KK_IN_BOUNDS(counter, ok) true
#endif

// staged entries a lane of the gather kernels holds in registers
constexpr int kMaxStagedEntries = 8;
int gather_entries_per_lane(int win);
// stage (transmits) of the staged DAS gather for a window, 0 = window too wide
int das_staged_stage(int win);
bool gather_config_supported(int rows, int stage, int win);

// Arguments of one frame's KK gather (also the batched form's per-frame
// descriptor, copied to the device).
struct GatherArgs {
  const float2 *rf_theta;
  int T;
  const int32_t *bf_row;
  const long long *bfA, *bfB, *bfC;
  const float *bfAf, *bfBf;
  const int32_t *group_start;
  int J, nx, nz, tiles_x, win, split;
  float2 *out;
  float *I;
  int compound;
};

// Extra arguments of the volumetric gather (a second kernel parameter, so the
// linear-array kernel's argument block stays as it is).
struct GatherVolArgs {
  const long long *bfY;  // per-pair delay per y slice (32.32 samples)
  int ny, tiles_xz;      // y slices and tiles per slice
};

// Keeps the caller's current device and restores it on exit.
struct DeviceGuard {
  int old = -1;
  bool ok = true;
  explicit DeviceGuard(int dev);
  ~DeviceGuard();
};

// Checks shared by the KK image-formation entry points: a KK plan, non-null
// rf_theta and B, I present when the plan compounds, rf_theta 16-byte aligned.
kk_status check_beamform_args(const kk_plan *p, const void *rf_theta, const void *B, const float *I);

// spectrum -> contraction -> inverse of one frame on stream s (no checks)
// side_by_side: the launch shares the GPU with other frames' kernels (the
// batched form's graph), so the contraction picks its throughput shape
kk_status enqueue_decompose(const kk_plan *p, const void *rf, void *rf_theta, void *ws, cudaStream_t s,
                            bool side_by_side = false);
// KK image formation of one frame on stream s (no checks)
kk_status enqueue_beamform(const kk_plan *p, const void *rf_theta, void *B, float *I, void *ws, cudaStream_t s);
// the contraction of the plan's precision form: X [F][p.Nu][L] -> Y [F][p.Nu][Mu]
cudaError_t launch_shear(const kk_plan &p, const void *X, float2 *Y, cudaStream_t s, bool side_by_side = false);

// thread-local error message
void set_error(const std::string &msg);
kk_status cuda_fail(cudaError_t e, const char *what);

// ---- launches (each returns cudaGetLastError() after the launch) ----------
// X is complex FP32, BF16 or FP16 per the plan's precision (spectrum_bytes)
cudaError_t launch_spectrum(const kk_plan &p, const void *rf, void *X, int n_tx_rows,
                            const int32_t *tx_rows, cudaStream_t s);
// row r goes to row out_row[r] of out (nullable: r) scaled by row_w[r]
// (nullable: 1)
cudaError_t launch_inverse(const kk_plan &p, const float2 *Y, int ncol, const int32_t *col_of_row,
                           int nrow, float2 *out, cudaStream_t s, const float *row_w = nullptr,
                           const int32_t *out_row = nullptr);
cudaError_t launch_shear_f32(const kk_plan &p, const float2 *X, float2 *Y, cudaStream_t s,
                             bool side_by_side = false);
cudaError_t launch_shear_sep(const kk_plan &p, const float2 *X, float2 *Y, cudaStream_t s);
size_t sep_shear_smem_bytes(int L, int Lf, int Ls, int Mf, int Ms, int msp, int tpc, bool bulk);
// separable contraction's split of the slow-axis waves over thread parts:
// parts, and waves per part (2, 4, 8 or 16); Ws rows hold parts * osn entries
void sep_split(int Lf, int Ms, int tpc, int &parts, int &osn);
constexpr int kSepMaxSlowWaves = 16;
cudaError_t launch_shear_tc(const kk_plan &p, const void *X, float2 *Y, cudaStream_t s);
size_t tc_shear_smem_bytes(int precision, int NP);
// bytes of one complex spectrum value for the plan's precision: FP32 8,
// BF16 / FP16 4 (FP8 plans keep FP16 spectra and round to e4m3 per column)
inline int spectrum_bytes(int precision) { return precision == KK_PREC_F32 ? 8 : 4; }
cudaError_t launch_kk_gather(const kk_plan &p, const float2 *rf_theta, float2 *B, float *I,
                             float2 *partial, cudaStream_t s);
GatherArgs gather_args(const kk_plan &p, const float2 *rf_theta, float2 *dst, float *I);
GatherVolArgs gather_vol_args(const kk_plan &p);
// persistent gather over n_items (frame, tile) items; *counter must be 0;
// vols (per frame, indexed like frames) non-null: volumetric frames, whose
// tiles run over every y slice
cudaError_t launch_kk_gather_batch(int rows, int stage, const GatherArgs *frames, const GatherVolArgs *vols,
                                   const int2 *items, int n_items, int *counter, int max_win, int grid,
                                   cudaStream_t s);
cudaError_t launch_das_gather(const kk_plan &p, const float2 *y, float2 *B, float *I,
                              float2 *partial, cudaStream_t s);

}  // namespace kk
