// kk_shear.cu -- the far-field decomposition as a per-bin complex contraction
// (FP32 form, CUDA cores).
//
// Eq. (compression) shears every element's record by delta_l(theta_o) and sums
// over elements.  Section II-F applies the shear with the Fourier shift
// theorem, which makes the step, for every frequency bin k, a dense complex
// product of the (receive angle x element) phase matrix with the (element x
// transmit) spectra:
//     Y[k][i][o] = sum_l X[k][i][l] W[k][o][l],
//     W[k][o][l] = exp(+2 pi i k phi[o][l]),  phi = frac(fs delta_l(theta_o) / T).
// W is never stored: each CTA generates its tile on chip from the 0.64
// fixed-point phases (k * phi mod 2^64 is exact integer arithmetic), so the
// contraction reads only X from HBM and writes only Y.
//
// Four kernels, chosen by launch_shear_f32:
//   k_shear_sep         volumetric plans whose elements form a grid and whose
//                       receive waves form a product of x and y tilts (W
//                       factors per axis);
//   k_shear_f32n        up to 64 transmits in use (tile sized to Nu x Mu, the
//                       phasor stepped across four bins);
//   k_shear_f32n_split  the same tile on a problem too small to fill the GPU:
//                       one bin per CTA, the elements split over slices;
//   k_shear_f32         everything else.
#include "kk_internal.h"
#include "kk_tc.h"
#include "kk_tma.h"

#include <algorithm>

namespace kk {

namespace {

constexpr int kTO = 64;   // receive angles per CTA (16 threads x 4)
constexpr int kLC = 32;   // elements per chunk

template <int RI>
__global__ void __launch_bounds__(256) k_shear_f32(const float2 *__restrict__ X,
                                                   const unsigned long long *__restrict__ phase,
                                                   int L, int Nu, int Mu,
                                                   float2 *__restrict__ Y) {
  constexpr int TI = 16 * RI;
  __shared__ __align__(16) float2 Ws[kLC][kTO];
  __shared__ __align__(16) float2 Xs[kLC][TI + 1];
  const int k = blockIdx.x;
  const int o0 = blockIdx.y * kTO;
  const int i0 = blockIdx.z * TI;
  const int tid = threadIdx.x;
  const int tx = tid & 15;   // receive-angle group (4 each)
  const int ty = tid >> 4;   // transmit group (RI each)
  const unsigned long long kk64 = (unsigned long long)k;
  const float2 *Xk = X + (size_t)k * Nu * L;

  float2 acc[4][RI];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < RI; ++b) acc[a][b] = make_float2(0.f, 0.f);

  for (int l0 = 0; l0 < L; l0 += kLC) {
    // W tile [l][o]: exp(2 pi i * (k phi mod 1))
    for (int e = tid; e < kLC * kTO; e += 256) {
      const int ll = e / kTO, oo = e - ll * kTO;
      const int o = o0 + oo, l = l0 + ll;
      float2 w = make_float2(0.f, 0.f);
      if (o < Mu && l < L) {
        const unsigned long long ph = __ldg(phase + (size_t)o * L + l) * kk64;
        const int hi = (int)(ph >> 32);              // turns in [-1/2, 1/2) * 2^32
        float sn, cs;
        sincospif((float)hi * 0x1p-31f, &sn, &cs);   // angle = 2 pi turns
        w = make_float2(cs, sn);
      }
      Ws[ll][oo] = w;
    }
    // X tile [l][i]
    for (int e = tid; e < kLC * TI; e += 256) {
      const int ii = e / kLC, ll = e - ii * kLC;
      const int i = i0 + ii, l = l0 + ll;
      float2 x = make_float2(0.f, 0.f);
      if (i < Nu && l < L) x = Xk[(size_t)i * L + l];
      Xs[ll][ii] = x;
    }
    __syncthreads();
    const int lmax = min(kLC, L - l0);
    for (int ll = 0; ll < lmax; ++ll) {
      const float4 w01 = *reinterpret_cast<const float4 *>(&Ws[ll][tx * 4]);
      const float4 w23 = *reinterpret_cast<const float4 *>(&Ws[ll][tx * 4 + 2]);
      const float2 w[4] = {make_float2(w01.x, w01.y), make_float2(w01.z, w01.w),
                           make_float2(w23.x, w23.y), make_float2(w23.z, w23.w)};
      float2 x[RI];
#pragma unroll
      for (int b = 0; b < RI; ++b) x[b] = Xs[ll][ty * RI + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < RI; ++b) {
          acc[a][b].x = fmaf(w[a].x, x[b].x, acc[a][b].x);
          acc[a][b].x = fmaf(-w[a].y, x[b].y, acc[a][b].x);
          acc[a][b].y = fmaf(w[a].x, x[b].y, acc[a][b].y);
          acc[a][b].y = fmaf(w[a].y, x[b].x, acc[a][b].y);
        }
    }
    __syncthreads();
  }
  float2 *Yk = Y + (size_t)k * Nu * Mu;
#pragma unroll
  for (int b = 0; b < RI; ++b) {
    const int i = i0 + ty * RI + b;
    if (i >= Nu) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int o = o0 + tx * 4 + a;
      if (o < Mu) Yk[(size_t)i * Mu + o] = acc[a][b];
    }
  }
}

// Few transmits (Nu <= 64): a W element serves only Nu transmits, so its
// sin/cos, not the products, dominated the form above (and a 16 RI transmit
// tile was mostly padding).  This form takes TN = 8 .. 64 transmits
// and 4 AG receive angles (the tile with the least padded work), and KB
// consecutive bins: W of the first bin and
// E = exp(2 pi i phi) come from the fixed-point phases once per element
// chunk, later bins step W <- W E (one complex product), at most KB - 1
// steps from an exact value.
constexpr int kLCn = 32;   // elements per chunk
constexpr int kKBn = 4;    // bins per CTA, at most (fewer when the grid would not fill the GPU)
constexpr int kKBnMinPerSM = 8;   // four bins per CTA from this many CTAs per SM on (a lone frame)
constexpr int kKSn = 4;    // element slices per CTA, at most, in the one-bin form

template <int TN, int AG>
__global__ void __launch_bounds__(TN * AG, 768 / (TN * AG)) k_shear_f32n(const float2 *__restrict__ X,
                                                    const unsigned long long *__restrict__ phase,
                                                    int L, int Nu, int Mu, int F, int kbn,
                                                    float2 *__restrict__ Y) {
  constexpr int NT = TN * AG;    // threads: TN transmits x AG angle groups of 4
  constexpr int TO = 4 * AG;
  extern __shared__ __align__(16) float2 n_smem[];
  float2 (*Ws)[TO] = reinterpret_cast<float2 (*)[TO]>(n_smem);               // [kLCn][TO]
  float2 (*Es)[TO] = reinterpret_cast<float2 (*)[TO]>(n_smem + kLCn * TO);   // [kLCn][TO]
  float2 (*Xs)[TN + 1] = reinterpret_cast<float2 (*)[TN + 1]>(n_smem + 2 * kLCn * TO);
  const int k0 = blockIdx.x * kbn;
  const int nk = min(kbn, F - k0);
  const int o0 = blockIdx.y * TO;
  const int i0 = blockIdx.z * TN;
  const int tid = threadIdx.x;
  // transmit fastest across lanes: a warp reads 32 / TN angle groups of W
  // (one or two 128-byte runs) and TN neighbouring X values per element
  const int ty = tid % TN;   // transmit
  const int tx = tid / TN;   // angle group
  const unsigned long long kk64 = (unsigned long long)k0;

  float2 acc[kKBn][4];
#pragma unroll
  for (int b = 0; b < kKBn; ++b)
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[b][a] = make_float2(0.f, 0.f);

  auto phasor = [](unsigned long long ph) {
    const int hi = (int)(ph >> 32);   // turns in [-1/2, 1/2) * 2^32
    float sn, cs;
    sincospif((float)hi * 0x1p-31f, &sn, &cs);
    return make_float2(cs, sn);
  };

  for (int l0 = 0; l0 < L; l0 += kLCn) {
    for (int e = tid; e < kLCn * TO; e += NT) {
      const int ll = e / TO, oo = e - ll * TO;
      const int o = o0 + oo, l = l0 + ll;
      float2 w = make_float2(0.f, 0.f), r = make_float2(0.f, 0.f);
      if (o < Mu && l < L) {
        const unsigned long long ph = __ldg(phase + (size_t)o * L + l);
        w = phasor(ph * kk64);
        if (kbn > 1) r = phasor(ph);
      }
      Ws[ll][oo] = w;
      Es[ll][oo] = r;
    }
    const int lmax = min(kLCn, L - l0);
#pragma unroll
    for (int b = 0; b < kKBn; ++b) {
      if (b >= nk) break;
      if (b > 0) {
        for (int e = tid; e < kLCn * TO; e += NT) {
          const int ll = e / TO, oo = e - ll * TO;
          const float2 w = Ws[ll][oo], r = Es[ll][oo];
          Ws[ll][oo] = make_float2(fmaf(w.x, r.x, -w.y * r.y), fmaf(w.x, r.y, w.y * r.x));
        }
      }
      const float2 *Xk = X + (size_t)(k0 + b) * Nu * L;
      for (int e = tid; e < kLCn * TN; e += NT) {
        const int ii = e / kLCn, ll = e - ii * kLCn;
        const int i = i0 + ii, l = l0 + ll;
        Xs[ll][ii] = (i < Nu && l < L) ? Xk[(size_t)i * L + l] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      for (int ll = 0; ll < lmax; ++ll) {
        const float4 w01 = *reinterpret_cast<const float4 *>(&Ws[ll][tx * 4]);
        const float4 w23 = *reinterpret_cast<const float4 *>(&Ws[ll][tx * 4 + 2]);
        const float2 w[4] = {make_float2(w01.x, w01.y), make_float2(w01.z, w01.w),
                             make_float2(w23.x, w23.y), make_float2(w23.z, w23.w)};
        const float2 x = Xs[ll][ty];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          acc[b][a].x = fmaf(w[a].x, x.x, acc[b][a].x);
          acc[b][a].x = fmaf(-w[a].y, x.y, acc[b][a].x);
          acc[b][a].y = fmaf(w[a].x, x.y, acc[b][a].y);
          acc[b][a].y = fmaf(w[a].y, x.x, acc[b][a].y);
        }
      }
      __syncthreads();
    }
  }
  const int i = i0 + ty;
  if (i >= Nu) return;
#pragma unroll
  for (int b = 0; b < kKBn; ++b) {
    if (b >= nk) break;
    float2 *Yk = Y + ((size_t)(k0 + b) * Nu + i) * Mu;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int o = o0 + tx * 4 + a;
      if (o < Mu) Yk[o] = acc[b][a];
    }
  }
}

// One bin per CTA with the elements split over KS slices of TN x AG
// threads (KS = 2 .. 4): a problem too small to give every SM a few CTAs of
// the form above (the 8 x 16 vernier frame: 1024 bins x one angle tile of 32
// threads) spreads its sin/cos and products over KS times the warps.  Slice
// s takes the element chunks s, s + KS, ... with its own W and X tiles; the
// slices step together between CTA barriers (named barriers per slice would
// hold the SM to four CTAs), and the partial sums are added in slice order.
template <int TN, int AG>
__global__ void __launch_bounds__(4 * TN * AG) k_shear_f32n_split(const float2 *__restrict__ X,
                                                             const unsigned long long *__restrict__ phase,
                                                             int L, int Nu, int Mu, int ks,
                                                             float2 *__restrict__ Y) {
  constexpr int NS = TN * AG;    // threads per slice
  constexpr int TO = 4 * AG;
  constexpr int SL = kLCn * TO + kLCn * (TN + 1);   // float2 per slice
  extern __shared__ __align__(16) float2 n_smem[];
  const int s = threadIdx.x / NS, t = threadIdx.x - s * NS;
  float2 (*Ws)[TO] = reinterpret_cast<float2 (*)[TO]>(n_smem + s * SL);
  float2 (*Xs)[TN + 1] = reinterpret_cast<float2 (*)[TN + 1]>(n_smem + s * SL + kLCn * TO);
  const int k = blockIdx.x;
  const int o0 = blockIdx.y * TO;
  const int i0 = blockIdx.z * TN;
  const int ty = t % TN, tx = t / TN;
  const unsigned long long kk64 = (unsigned long long)k;
  const float2 *Xk = X + (size_t)k * Nu * L;

  float2 acc[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a] = make_float2(0.f, 0.f);
  for (int c0 = 0; c0 * kLCn < L; c0 += ks) {
    const int l0 = (c0 + s) * kLCn;   // this slice's chunk (none past the last)
    for (int e = t; e < kLCn * TO; e += NS) {
      const int ll = e / TO, oo = e - ll * TO;
      const int o = o0 + oo, l = l0 + ll;
      float2 w = make_float2(0.f, 0.f);
      if (o < Mu && l < L) {
        const int hi = (int)((__ldg(phase + (size_t)o * L + l) * kk64) >> 32);
        sincospif((float)hi * 0x1p-31f, &w.y, &w.x);
      }
      Ws[ll][oo] = w;
    }
    for (int e = t; e < kLCn * TN; e += NS) {
      const int ii = e / kLCn, ll = e - ii * kLCn;
      const int i = i0 + ii, l = l0 + ll;
      Xs[ll][ii] = (i < Nu && l < L) ? Xk[(size_t)i * L + l] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int lmax = min(kLCn, L - l0);
    for (int ll = 0; ll < lmax; ++ll) {
      const float4 w01 = *reinterpret_cast<const float4 *>(&Ws[ll][tx * 4]);
      const float4 w23 = *reinterpret_cast<const float4 *>(&Ws[ll][tx * 4 + 2]);
      const float2 w[4] = {make_float2(w01.x, w01.y), make_float2(w01.z, w01.w),
                           make_float2(w23.x, w23.y), make_float2(w23.z, w23.w)};
      const float2 x = Xs[ll][ty];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        acc[a].x = fmaf(w[a].x, x.x, acc[a].x);
        acc[a].x = fmaf(-w[a].y, x.y, acc[a].x);
        acc[a].y = fmaf(w[a].x, x.y, acc[a].y);
        acc[a].y = fmaf(w[a].y, x.x, acc[a].y);
      }
    }
    __syncthreads();
  }   // every slice is done with its tiles: they now hold the partial sums
  float2 *part = n_smem;   // [ks - 1][NS][4]
  if (s > 0) {
#pragma unroll
    for (int a = 0; a < 4; ++a) part[((size_t)(s - 1) * NS + t) * 4 + a] = acc[a];
  }
  __syncthreads();
  if (s > 0) return;
  for (int r = 1; r < ks; ++r)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float2 q = part[((size_t)(r - 1) * NS + t) * 4 + a];
      acc[a].x += q.x;
      acc[a].y += q.y;
    }
  const int i = i0 + ty;
  if (i >= Nu) return;
  float2 *Yk = Y + ((size_t)k * Nu + i) * Mu;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int o = o0 + tx * 4 + a;
    if (o < Mu) Yk[o] = acc[a];
  }
}

template <int TN, int AG>
cudaError_t launch_n(const kk_plan &p, const float2 *X, float2 *Y, cudaStream_t s, bool side_by_side) {
  constexpr int TO = 4 * AG;
  const size_t smem = sizeof(float2) * (2 * (size_t)kLCn * TO + (size_t)kLCn * (TN + 1));
  cudaError_t e =
      cudaFuncSetAttribute(k_shear_f32n<TN, AG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // bins per CTA: kKBn amortises each element chunk's sin/cos over four
  // bins, which pays where throughput counts: in the batched form, whose
  // frames' kernels share the GPU, from one four-bin CTA per SM, and for a
  // lone frame from kKBnMinPerSM per SM.  A smaller lone frame is latency
  // bound: it takes one bin per CTA with the elements split over up to kKSn
  // slices, so that its sin/cos and products spread over more warps.  Both
  // choices depend on the bins, receive angles and elements only, never on
  // the transmits in use: W of a bin is then formed and summed the same way
  // whatever transmit subset a call contracts (the streaming decomposition's
  // groups equal the whole frame bit for bit).
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
  const long long nominal = (long long)((p.F + kKBn - 1) / kKBn) * ((p.Mu + 15) / 16);
  const int kbn = nominal >= (long long)(side_by_side ? 1 : kKBnMinPerSM) * sms ? kKBn : 1;
  const int ks = kbn == 1 ? std::min(kKSn, (p.L + kLCn - 1) / kLCn) : 1;
  if (ks > 1) {
    constexpr size_t sl = sizeof(float2) * ((size_t)kLCn * TO + (size_t)kLCn * (TN + 1));
    const size_t smem_s = std::max(sl * ks, sizeof(float2) * 4 * TN * AG * (ks - 1));
    e = cudaFuncSetAttribute(k_shear_f32n_split<TN, AG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_s);
    // all of the SM's shared memory for CTAs (the vernier frame's 1024 CTAs
    // of 26 KB then fit in one wave, eight per SM)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_shear_f32n_split<TN, AG>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    const dim3 grid_s(p.F, (p.Mu + TO - 1) / TO, (p.Nu + TN - 1) / TN);
    k_shear_f32n_split<TN, AG><<<grid_s, TN * AG * ks, smem_s, s>>>(X, p.t.phase, p.L, p.Nu, p.Mu, ks, Y);
    return cudaGetLastError();
  }
  const dim3 grid((p.F + kbn - 1) / kbn, (p.Mu + TO - 1) / TO, (p.Nu + TN - 1) / TN);
  k_shear_f32n<TN, AG><<<grid, TN * AG, smem, s>>>(X, p.t.phase, p.L, p.Nu, p.Mu, p.F, kbn, Y);
  return cudaGetLastError();
}

template <int RI>
cudaError_t launch_ri(const kk_plan &p, const float2 *X, float2 *Y, cudaStream_t s) {
  const dim3 grid(p.F, (p.Mu + kTO - 1) / kTO, (p.Nu + 16 * RI - 1) / (16 * RI));
  k_shear_f32<RI><<<grid, 256, 0, s>>>(X, p.t.phase, p.L, p.Nu, p.Mu, Y);
  return cudaGetLastError();
}

// Separable form.  For a matrix array whose elements fill an Lx x Ly grid,
// u_l = ux[lx], v_l = vy[ly], and receive waves on a product of Mx x-tilts
// and My y-tilts, the volumetric shear delay splits per axis,
//     fs delta_l(o) / T = phx[ox][lx] + phy[oy][ly]  (mod 1),
// so W[o][l] = Wx[ox][lx] Wy[oy][ly] and the element sum of Eq. (compression)
// becomes two short contractions per bin and transmit.  With the element
// index l = ls Lf + lf (f the grid axis that varies fastest in the caller's
// element order, s the other):
//     Z[lf][os] = sum_ls X[ls][lf] Ws[os][ls],   Y[os][of] = sum_lf Z[lf][os] Wf[of][lf],
// (Ms Ls + Mf Ms) Lf complex products instead of Lf Ls Mf Ms.
//
// The phasors of every bin, Wf[k][lf][of] and Ws[k][ls][os], are built by
// the plan in FP64 (from the 0.64 fixed-point phases, k phi mod 1 exact) and
// stored per bin as one contiguous run, so an item needs no sin/cos.
//
// Persistent CTAs walk the (bin, transmit chunk) items.  A chunk's spectra
// X[k][i0 .. i0 + nt)[:] are one contiguous run: it and the bin's phasors
// are fetched by bulk copies into the other of two shared-memory stages
// while the current item is contracted (BULK; element orders that are not a
// row-major grid use a plain gather through the slot table and one stage).
// In the first contraction the lanes of a warp run along lf, so the
// unpadded rows are read without bank conflicts and the weights Ws[ls][os]
// are broadcasts; the threads left over take the slow-axis waves in parts of
// OSN (zero weights pad the last part), each thread summing every row.  Z
// goes to the stage's X buffer once every thread has read its rows, and the
// second contraction sums it over lf.
constexpr int kSepThreads = 256;

struct SepArgs {
  const float2 *X;
  const float2 *W;       // [F][wf + ws]: Wf [Lf][Mf] (padded to even), Ws [Ls][msp] (zero pad)
  const int32_t *slot;   // [L] ls Lf + lf (gather form)
  const int32_t *col;    // [Ms][Mf] receive position
  int L, Lf, Ls, Mf, Ms, msp, parts, Nu, Mu, tpc, chunks, n_items;
  float2 *Y;
  int *status;
};

__device__ __forceinline__ void cmac(float2 &acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// float2 counts of one stage: X / Z buffer, Wf, Ws (each a multiple of 2,
// so every part starts on 16 bytes)
struct SepLayout {
  int buf, wf, ws;
  __host__ __device__ SepLayout(int L, int Lf, int Ls, int Mf, int Ms, int msp, int tpc) {
    const int x = tpc * L, z = tpc * Lf * Ms;
    buf = ((x > z ? x : z) + 1) & ~1;
    wf = (Lf * Mf + 1) & ~1;
    ws = Ls * msp;
  }
  __host__ __device__ int stage() const { return buf + wf + ws; }
};

template <bool BULK, int OSN>
__global__ void __launch_bounds__(kSepThreads) k_shear_sep(const SepArgs a) {
  extern __shared__ __align__(16) float2 sep_smem[];
  __shared__ __align__(8) uint64_t bar[2];
  const SepLayout lay(a.L, a.Lf, a.Ls, a.Mf, a.Ms, a.msp, a.tpc);
  const int tid = threadIdx.x;
  if (BULK) {
    if (tid == 0) {
      tc::mbar_init(&bar[0], 1);
      tc::mbar_init(&bar[1], 1);
    }
    tc::mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int item, int b) {  // one thread
    const int k = item / a.chunks, i0 = (item - k * a.chunks) * a.tpc;
    const unsigned xb = (unsigned)(min(a.tpc, a.Nu - i0) * a.L * (int)sizeof(float2));
    const unsigned wb = (unsigned)((lay.wf + lay.ws) * (int)sizeof(float2));
    float2 *st = sep_smem + (size_t)b * lay.stage();
    tma::mbar_expect_tx(&bar[b], xb + wb);
    tma::bulk_1d(tc::smem_u32(st), a.X + ((size_t)k * a.Nu + i0) * a.L, xb, &bar[b]);
    tma::bulk_1d(tc::smem_u32(st + lay.buf), a.W + (size_t)k * (lay.wf + lay.ws), wb, &bar[b]);
  };
  int item = blockIdx.x;
  if (BULK && tid == 0 && item < a.n_items) issue(item, 0);
  for (int n = 0; item < a.n_items; item += gridDim.x, ++n) {
    const int b = BULK ? (n & 1) : 0;
    const int k = item / a.chunks, i0 = (item - k * a.chunks) * a.tpc;
    const int nt = min(a.tpc, a.Nu - i0);
    const bool next = item + (int)gridDim.x < a.n_items;
    float2 *Xs = sep_smem + (size_t)b * lay.stage();
    const float2 *Wf = Xs + lay.buf;   // [Lf][Mf]
    const float2 *Ws = Wf + lay.wf;    // [Ls][msp]: part h's waves at h OSN
    if (BULK) {
      if (tid == 0 && next) issue(item + gridDim.x, b ^ 1);
      const bool ok = tc::mbar_wait(&bar[b], (uint32_t)(n >> 1) & 1u);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicExch(a.status, (int)KK_ERR_TIMEOUT);
          tc::mbar_wait(&bar[b], (uint32_t)(n >> 1) & 1u);
          if (next) tc::mbar_wait(&bar[b ^ 1], (uint32_t)((n + 1) >> 1) & 1u);
        }
        return;
      }
    } else {
      const float2 *Xk = a.X + ((size_t)k * a.Nu + i0) * a.L;
      for (int e = tid; e < nt * a.L; e += kSepThreads) {
        const int t = e / a.L, l = e - t * a.L;
        Xs[(size_t)t * a.L + __ldg(a.slot + l)] = __ldg(Xk + e);
      }
      const float2 *Wk = a.W + (size_t)k * (lay.wf + lay.ws);
      for (int e = tid; e < lay.wf + lay.ws; e += kSepThreads) Xs[lay.buf + e] = __ldg(Wk + e);
      __syncthreads();
    }

    // first contraction: thread (part h, transmit t, lf) over every row ls
    // for the OSN slow-axis waves of part h (zero weights past Ms), so each
    // Z entry is one sum in a fixed order whatever the items hold
    const int lanes = nt * a.Lf;
    const bool worker = tid < a.parts * lanes;
    const int h = tid / lanes, r = tid - h * lanes;
    const int t = r / a.Lf, lf = r - t * a.Lf;
    float2 acc[OSN];
#pragma unroll
    for (int j = 0; j < OSN; ++j) acc[j] = make_float2(0.f, 0.f);
    if (worker) {
      const float2 *xc = Xs + (size_t)t * a.L + lf;
      const float4 *wc = reinterpret_cast<const float4 *>(Ws + h * OSN);
      const int wstep = a.msp / 2;
#pragma unroll 4
      for (int ls = 0; ls < a.Ls; ++ls) {
        const float2 x = xc[ls * a.Lf];
        const float4 *w = wc + ls * wstep;
#pragma unroll
        for (int j = 0; j < OSN / 2; ++j) {
          const float4 w2 = w[j];
          cmac(acc[2 * j], make_float2(w2.x, w2.y), x);
          cmac(acc[2 * j + 1], make_float2(w2.z, w2.w), x);
        }
      }
    }
    __syncthreads();  // every row of X read: Z may overwrite the buffer
    if (worker) {
      float2 *z = Xs + ((size_t)t * a.Lf + lf) * a.Ms;
#pragma unroll
      for (int j = 0; j < OSN; ++j)
        if (h * OSN + j < a.Ms) z[h * OSN + j] = acc[j];
    }
    // the stage is refilled by bulk copies two items on: order these
    // ordinary stores before the copies' asynchronous writes
    if (BULK) tc::fence_async_smem();
    __syncthreads();

    // second contraction: thread (t, os, of) over lf, four interleaved
    // partial sums (short dependency chains)
    float2 *Yk = a.Y + ((size_t)k * a.Nu + i0) * a.Mu;
    const int per_t = a.Ms * a.Mf;
    for (int e = tid; e < nt * per_t; e += kSepThreads) {
      const int t2 = e / per_t, r2 = e - t2 * per_t;
      const int os = r2 / a.Mf, of = r2 - os * a.Mf;
      float2 s4[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) s4[j] = make_float2(0.f, 0.f);
      const float2 *z = Xs + (size_t)t2 * a.Lf * a.Ms + os;
      const float2 *wf = Wf + of;
      int l2 = 0;
      for (; l2 + 4 <= a.Lf; l2 += 4) {
#pragma unroll
        for (int j = 0; j < 4; ++j) cmac(s4[j], wf[(l2 + j) * a.Mf], z[(l2 + j) * a.Ms]);
      }
      for (; l2 < a.Lf; ++l2) cmac(s4[0], wf[l2 * a.Mf], z[l2 * a.Ms]);
      Yk[(size_t)t2 * a.Mu + __ldg(a.col + r2)] =
          make_float2((s4[0].x + s4[1].x) + (s4[2].x + s4[3].x), (s4[0].y + s4[1].y) + (s4[2].y + s4[3].y));
    }
    __syncthreads();  // stage free for the copy issued at the next item
  }
}

}  // namespace

size_t sep_shear_smem_bytes(int L, int Lf, int Ls, int Mf, int Ms, int msp, int tpc, bool bulk) {
  return sizeof(float2) * (size_t)(bulk ? 2 : 1) * SepLayout(L, Lf, Ls, Mf, Ms, msp, tpc).stage();
}

void sep_split(int Lf, int Ms, int tpc, int &parts, int &osn) {
  parts = std::max(1, std::min(Ms, kSepThreads / (tpc * Lf)));
  const int need = (Ms + parts - 1) / parts;
  osn = need <= 2 ? 2 : need <= 4 ? 4 : need <= 8 ? 8 : 16;
}

cudaError_t launch_shear_sep(const kk_plan &p, const float2 *X, float2 *Y, cudaStream_t s) {
  SepArgs a;
  a.X = X;
  a.Y = Y;
  a.W = p.t.sep_w;
  a.status = p.t.status;
  a.slot = p.t.sep_slot;
  a.col = p.t.sep_col;
  a.L = p.L;
  a.Nu = p.Nu;
  a.Mu = p.Mu;
  a.Lf = p.sep_yfast ? p.sep_Ly : p.sep_Lx;
  a.Ls = p.sep_yfast ? p.sep_Lx : p.sep_Ly;
  a.Mf = p.sep_yfast ? p.sep_My : p.sep_Mx;
  a.Ms = p.sep_yfast ? p.sep_Mx : p.sep_My;
  a.tpc = p.sep_tpc;
  int osn = 0;
  sep_split(a.Lf, a.Ms, a.tpc, a.parts, osn);
  a.msp = a.parts * osn;
  a.chunks = (p.Nu + p.sep_tpc - 1) / p.sep_tpc;
  a.n_items = p.F * a.chunks;
  const bool bulk = p.sep_bulk && ((uintptr_t)X % 16) == 0;
  const size_t smem = sep_shear_smem_bytes(p.L, a.Lf, a.Ls, a.Mf, a.Ms, a.msp, a.tpc, bulk);
  void (*k)(SepArgs) = nullptr;
  switch (osn) {
    case 2: k = bulk ? k_shear_sep<true, 2> : k_shear_sep<false, 2>; break;
    case 4: k = bulk ? k_shear_sep<true, 4> : k_shear_sep<false, 4>; break;
    case 8: k = bulk ? k_shear_sep<true, 8> : k_shear_sep<false, 8>; break;
    default: k = bulk ? k_shear_sep<true, 16> : k_shear_sep<false, 16>; break;
  }
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int sms = 148, per_sm = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kSepThreads, smem);
  const int grid = std::max(1, std::min(a.n_items, sms * std::max(per_sm, 1)));
  k<<<grid, kSepThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_shear_f32(const kk_plan &p, const float2 *X, float2 *Y, cudaStream_t s, bool side_by_side) {
  if (p.sep_Lx > 0) return launch_shear_sep(p, X, Y, s);
  if (p.Nu <= 64) {
    // the tile (TN transmits x AG groups of 4 angles, 32 .. 256 threads)
    // with the least padded work per bin group, then the fewest CTAs
    int bt = 0, ba = 0;
    long long best = 0;
    for (int tn : {8, 16, 32, 64})
      for (int ag : {1, 2, 4, 8, 16, 32}) {
        if (tn * ag < 32 || tn * ag > 256) continue;
        const long long tiles = (long long)((p.Mu + 4 * ag - 1) / (4 * ag)) * ((p.Nu + tn - 1) / tn);
        const long long work = tiles * tn * ag;
        if (bt == 0 || work < best || (work == best && tn * ag > bt * ba)) {
          bt = tn;
          ba = ag;
          best = work;
        }
      }
    switch (bt * 100 + ba) {
      case 804: return launch_n<8, 4>(p, X, Y, s, side_by_side);
      case 808: return launch_n<8, 8>(p, X, Y, s, side_by_side);
      case 816: return launch_n<8, 16>(p, X, Y, s, side_by_side);
      case 832: return launch_n<8, 32>(p, X, Y, s, side_by_side);
      case 1602: return launch_n<16, 2>(p, X, Y, s, side_by_side);
      case 1604: return launch_n<16, 4>(p, X, Y, s, side_by_side);
      case 1608: return launch_n<16, 8>(p, X, Y, s, side_by_side);
      case 1616: return launch_n<16, 16>(p, X, Y, s, side_by_side);
      case 3201: return launch_n<32, 1>(p, X, Y, s, side_by_side);
      case 3202: return launch_n<32, 2>(p, X, Y, s, side_by_side);
      case 3204: return launch_n<32, 4>(p, X, Y, s, side_by_side);
      case 3208: return launch_n<32, 8>(p, X, Y, s, side_by_side);
      case 6401: return launch_n<64, 1>(p, X, Y, s, side_by_side);
      case 6402: return launch_n<64, 2>(p, X, Y, s, side_by_side);
      default: return launch_n<64, 4>(p, X, Y, s, side_by_side);
    }
  }
  const int ri = (p.Nu + 15) / 16;
  switch (ri) {
    case 1: return launch_ri<1>(p, X, Y, s);
    case 2: return launch_ri<2>(p, X, Y, s);
    case 3: return launch_ri<3>(p, X, Y, s);
    case 4: return launch_ri<4>(p, X, Y, s);
    default: return launch_ri<5>(p, X, Y, s);
  }
}

}  // namespace kk
