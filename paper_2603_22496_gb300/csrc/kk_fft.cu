// kk_fft.cu -- analytic spectrum (forward) and half-spectrum inverse.
//
// Section II-F of the paper: the RF records are made complex (analytic) by a
// temporal Fourier transform with the negative frequencies set to zero, and
// the receive shear of Eq. (compression) is applied in that frequency domain.
//
//  * k_spectrum: one T-sample real record per channel -> X[k] for k < F = T/2,
//    with weights h_0 = 1, h_k = 2 (the Nyquist bin is dropped).  The record
//    is packed as F complex points z[n] = x[2n] + i x[2n+1], transformed with
//    an F-point Stockham FFT in shared memory (radix-16 passes computed in
//    registers, then radix 4 / 2 / 3), and split into the T-point
//    spectrum by X[k] = E[k] + e^{-2 pi i k / T} O[k].
//    Output layout X[k][c] (bin-major) feeds the per-bin contraction.
//  * k_inverse: y[t] = (w/T) sum_{k<F} Y[k] e^{+2 pi i k t / T} for t < T
//    (w = the row's pair weight, 1 without weights),
//    computed as two F-point inverse transforms (even t from Y[k], odd t from
//    Y[k] e^{+2 pi i k / T}), written as one contiguous T-sample row.
//
// Each CTA transforms several records at once (C per CTA), so that a
// bin-major global access touches C consecutive complex values.  The
// transform runs in place in shared memory: every pass reads its butterfly
// inputs into registers, synchronises, then writes the outputs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kk_internal.h"
#include "kk_tma.h"

namespace kk {

// ---- radix plan (shared by host and device) --------------------------------
// passes of radix 16 first (computed in registers as 4 x 4), then 4, 2, 3
__host__ __device__ constexpr int fft_npass(int F) {
  int n = 0;
  while (F % 16 == 0) { F /= 16; ++n; }
  while (F % 4 == 0) { F /= 4; ++n; }
  while (F % 2 == 0) { F /= 2; ++n; }
  while (F % 3 == 0) { F /= 3; ++n; }
  return n;
}
__host__ __device__ constexpr int fft_radix(int F, int i) {
  int n = 0;
  while (F % 16 == 0) { if (n == i) return 16; F /= 16; ++n; }
  while (F % 4 == 0) { if (n == i) return 4; F /= 4; ++n; }
  while (F % 2 == 0) { if (n == i) return 2; F /= 2; ++n; }
  while (F % 3 == 0) { if (n == i) return 3; F /= 3; ++n; }
  return 1;
}
// Shared-memory position of point e of a transform: one padding slot per 32
// points, so that the radix-16 pass's stride-16 writes hit distinct banks.
__host__ __device__ constexpr int fft_pad(int e) { return e + (e >> 5); }
// row stride (complex points) of one transform in shared memory: 2 mod 16,
// so that 8 transforms x 2 neighbouring points read by a half-warp hit 16
// distinct 8-byte bank pairs
__host__ __device__ constexpr int fft_row(int F) { return F + F / 32 + 2; }
__host__ __device__ constexpr int fft_ns(int F, int i) {
  int ns = 1;
  for (int k = 0; k < i; ++k) ns *= fft_radix(F, k);
  return ns;
}
__host__ __device__ constexpr int fft_twoff(int F, int i) {
  int off = 0;
  for (int k = 0; k < i; ++k) off += fft_ns(F, k) * (fft_radix(F, k) - 1);
  return off;
}

bool fft_size_supported(int F) {
  return F == 128 || F == 256 || F == 512 || F == 768 || F == 1024 || F == 1536 || F == 2048;
}

FftPlan make_fft_plan(int F) {
  FftPlan p;
  p.F = F;
  p.npass = fft_npass(F);
  for (int i = 0; i < p.npass; ++i) {
    p.radix[i] = fft_radix(F, i);
    p.ns[i] = fft_ns(F, i);
    p.tw_off[i] = fft_twoff(F, i);
  }
  p.tw_count = fft_twoff(F, p.npass);
  return p;
}

// ---- complex helpers --------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// forward DFT of size R in registers (kernel e^{-2 pi i / R})
template <int R> __device__ __forceinline__ void dft(float2 *v);
template <> __device__ __forceinline__ void dft<2>(float2 *v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <> __device__ __forceinline__ void dft<3>(float2 *v) {
  const float h = 0.866025403784438646763723170752936183f;  // sqrt(3)/2
  float2 a = v[0], s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
  float2 m = make_float2(fmaf(-0.5f, s.x, a.x), fmaf(-0.5f, s.y, a.y));
  v[0] = cadd(a, s);
  // -i * h * d = (h d.y, -h d.x)
  v[1] = make_float2(fmaf(h, d.y, m.x), fmaf(-h, d.x, m.y));
  v[2] = make_float2(fmaf(-h, d.y, m.x), fmaf(h, d.x, m.y));
}
template <> __device__ __forceinline__ void dft<4>(float2 *v) {
  float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  float2 t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = make_float2(t1.x + t3.y, t1.y - t3.x);  // t1 - i t3
  v[3] = make_float2(t1.x - t3.y, t1.y + t3.x);  // t1 + i t3
}

// 16-point DFT as 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2; DFT-4 over n1, twiddle
// exp(-2 pi i n2 k1 / 16), DFT-4 over n2.
template <> __device__ __forceinline__ void dft<16>(float2 *v) {
  constexpr float C1 = 0.923879532511286756128f;  // cos(pi/8)
  constexpr float S1 = 0.382683432365089771728f;  // sin(pi/8)
  constexpr float H = 0.707106781186547524401f;   // sqrt(1/2)
  float2 y[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    float2 a[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
    dft<4>(a);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = a[k1];
  }
  // exp(-2 pi i m / 16) for m = n2 k1 in {1, 2, 3, 4, 6, 9}
  y[1][1] = cmul(y[1][1], make_float2(C1, -S1));
  y[1][2] = cmul(y[1][2], make_float2(H, -H));
  y[1][3] = cmul(y[1][3], make_float2(S1, -C1));
  y[2][1] = cmul(y[2][1], make_float2(H, -H));
  y[2][2] = make_float2(y[2][2].y, -y[2][2].x);  // times -i
  y[2][3] = cmul(y[2][3], make_float2(-H, -H));
  y[3][1] = cmul(y[3][1], make_float2(S1, -C1));
  y[3][2] = cmul(y[3][2], make_float2(-H, -H));
  y[3][3] = cmul(y[3][3], make_float2(-C1, S1));
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    float2 b[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
    dft<4>(b);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = b[k2];
  }
}

// One Stockham pass over NTR transforms of F points stored with row stride FS;
// tw is the twiddle table staged in shared memory.
template <int R, int NS, int F, int FS, int NTR, int NT>
__device__ __forceinline__ void stockham_pass(float2 *buf, const float2 *tw, int tid) {
  constexpr int NBF = NTR * (F / R);
  constexpr int NB = (NBF + NT - 1) / NT;
  float2 v[NB][R];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tid + b * NT;
    if (NBF % NT == 0 || j < NBF) {
      const int tr = j / (F / R);
      const int jj = j - tr * (F / R);
      const int k = jj % NS;
      const float2 *src = buf + tr * FS;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = src[fft_pad(jj + r * (F / R))];
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], tw[k * (R - 1) + (r - 1)]);
      }
      dft<R>(v[b]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tid + b * NT;
    if (NBF % NT == 0 || j < NBF) {
      const int tr = j / (F / R);
      const int jj = j - tr * (F / R);
      const int k = jj % NS;
      float2 *dst = buf + tr * FS;
      const int d0 = (jj - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[fft_pad(d0 + r * NS)] = v[b][r];
    }
  }
  __syncthreads();
}

// passes I .. END - 1 in place
template <int F, int FS, int NTR, int NT, int I, int END = fft_npass(F)>
__device__ __forceinline__ void run_passes(float2 *buf, const float2 *tw, int tid) {
  if constexpr (I < END) {
    constexpr int R = fft_radix(F, I);
    constexpr int NS = fft_ns(F, I);
    constexpr int OFF = fft_twoff(F, I);
    stockham_pass<R, NS, F, FS, NTR, NT>(buf, tw + OFF, tid);
    run_passes<F, FS, NTR, NT, I + 1, END>(buf, tw, tid);
  }
}

__device__ __forceinline__ float2 load_pair(const int16_t *p) {
  const short2 v = *reinterpret_cast<const short2 *>(p);
  return make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ float2 load_pair(const float *p) {
  return *reinterpret_cast<const float2 *>(p);
}

// ---- forward: analytic spectrum -------------------------------------------
// X[k][c] for channel c = iu * L + l (row tx_rows[iu] * L + l of rf).
__device__ __forceinline__ void store_x(float2 *X, size_t idx, float2 v) { X[idx] = v; }
__device__ __forceinline__ void store_x(__nv_bfloat162 *X, size_t idx, float2 v) {
  X[idx] = __floats2bfloat162_rn(v.x, v.y);
}
__device__ __forceinline__ void store_x(__half2 *X, size_t idx, float2 v) {
  X[idx] = __floats2half2_rn(v.x, v.y);
}

// 16-byte vector of a real record -> VE / 2 complex points
__device__ __forceinline__ void unpack16(const uint4 &u, const int16_t *, float2 *z) {
  const short2 *h = reinterpret_cast<const short2 *>(&u);
#pragma unroll
  for (int q = 0; q < 4; ++q) z[q] = make_float2((float)h[q].x, (float)h[q].y);
}
__device__ __forceinline__ void unpack16(const uint4 &u, const float *, float2 *z) {
  const float *f = reinterpret_cast<const float *>(&u);
  z[0] = make_float2(f[0], f[1]);
  z[1] = make_float2(f[2], f[3]);
}

// VEC: the records are 16-byte aligned (read with 16-byte vector loads)
template <int F, int C, int NT, typename TIn, typename TOut, bool VEC>
__global__ void __launch_bounds__(NT) k_spectrum(const TIn *__restrict__ rf,
                                                 const int32_t *__restrict__ tx_rows, int L,
                                                 int n_ch, const float2 *__restrict__ tw,
                                                 const float2 *__restrict__ rw,
                                                 TOut *__restrict__ X, float xscale) {
  constexpr int FS = fft_row(F);
  constexpr int T = 2 * F;
  extern __shared__ float2 sm[];
  __shared__ long long s_row[C];  // first sample of each record, -1 past the last channel
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * C;
  float2 *s_tw = sm + C * FS;  // twiddles of every pass
  for (int i = tid; i < fft_twoff(F, fft_npass(F)); i += NT) s_tw[i] = __ldg(tw + i);
  if (tid < C) {
    const int c = c0 + tid;
    long long r = -1;
    if (c < n_ch) {
      const int iu = c / L, l = c - iu * L;
      r = ((long long)__ldg(tx_rows + iu) * L + l) * T;
    }
    s_row[tid] = r;
  }
  __syncthreads();
  if constexpr (VEC) {
    constexpr int VE = 16 / (int)sizeof(TIn);  // samples per vector
    constexpr int NV = T / VE;                 // vectors per record
#pragma unroll 4
    for (int idx = tid; idx < C * NV; idx += NT) {
      const int cc = idx / NV, v = idx - cc * NV;
      const long long r = s_row[cc];
      float2 z[VE / 2];
      if (r >= 0) {
        const uint4 u = __ldg(reinterpret_cast<const uint4 *>(rf + r) + v);
        unpack16(u, rf, z);
      } else {
#pragma unroll
        for (int q = 0; q < VE / 2; ++q) z[q] = make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < VE / 2; ++q) sm[cc * FS + fft_pad(v * (VE / 2) + q)] = z[q];
    }
  } else {
#pragma unroll 4
    for (int idx = tid; idx < C * F; idx += NT) {
      const int cc = idx / F, n = idx - cc * F;
      const long long r = s_row[cc];
      sm[cc * FS + fft_pad(n)] = r >= 0 ? load_pair(rf + r + 2 * n) : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  run_passes<F, FS, C, NT, 0>(sm, s_tw, tid);
  for (int idx = tid; idx < C * F; idx += NT) {
    const int k = idx / C, cc = idx - k * C;
    const int c = c0 + cc;
    if (c >= n_ch) continue;
    const float2 zk = sm[cc * FS + fft_pad(k)];
    const float2 zm = sm[cc * FS + fft_pad(k == 0 ? 0 : F - k)];
    // E = (Z[k] + conj Z[F-k]) / 2,  O = (Z[k] - conj Z[F-k]) / (2i)
    const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    float2 x = cadd(e, cmul(__ldg(rw + k), o));
    const float h = (k == 0) ? xscale : 2.f * xscale;
    x.x *= h;
    x.y *= h;
    store_x(X, (size_t)k * n_ch + c, x);
  }
}

// ---- fused first and last passes of the persistent spectrum ----------------
// First pass (NS = 1) read straight from the staged real records: point n of
// record tr is the sample pair (2n, 2n + 1).  Writes the Stockham output of
// the pass into buf (a different buffer, so no barrier between read and
// write).  Records tr >= nc are not loaded and give zeros.
template <int F, int FS, int C, int NT, typename TIn>
__device__ __forceinline__ void first_pass_staged(const uint4 *stg, int nv, int nc, float2 *buf, int tid) {
  constexpr int R = fft_radix(F, 0);
  static_assert(fft_ns(F, 0) == 1, "first pass has NS = 1");
  constexpr int NBF = C * (F / R);
#pragma unroll 2
  for (int j = tid; j < NBF; j += NT) {
    const int tr = j / (F / R), jj = j - tr * (F / R);
    float2 v[R];
    const TIn *rec = reinterpret_cast<const TIn *>(stg + (size_t)tr * nv);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = tr < nc ? load_pair(rec + 2 * (jj + r * (F / R))) : make_float2(0.f, 0.f);
    dft<R>(v);
    float2 *dst = buf + tr * FS;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[fft_pad(jj * R + r)] = v[r];
  }
}

// Last pass (NS = F / R) fused with the split of the packed transform into the
// analytic spectrum, which pairs Z[k] with Z[F - k].  Output r of butterfly jj
// is point jj + r NS, and F - (jj + r NS) is output R - 1 - r of butterfly
// NS - jj; so one thread takes butterflies t and NS - t (t = 1 .. NS/2 - 1),
// or 0 and NS/2 (both paired with themselves), and forms the spectrum in
// registers.  Lanes run over transforms first, so a warp store writes runs of
// C adjacent channels.
template <int F, int FS, int C, int NT, typename TOut>
__device__ __forceinline__ void last_pass_spectrum(const float2 *buf, const float2 *tw, const float2 *rw, int nc,
                                                   int c0, int n_ch, float xscale, TOut *X, int tid) {
  constexpr int LAST = fft_npass(F) - 1;
  constexpr int R = fft_radix(F, LAST);
  constexpr int NS = fft_ns(F, LAST);
  static_assert(NS * R == F && NS % 2 == 0, "last pass");
  constexpr int H = NS / 2;
  const float2 *twl = tw + fft_twoff(F, LAST);
  for (int idx = tid; idx < C * H; idx += NT) {
    const int tr = idx % C, t = idx / C;
    if (tr >= nc) continue;
    const int A = t, B = t == 0 ? H : NS - t;
    const float2 *src = buf + tr * FS;
    float2 va[R], vb[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      va[r] = src[fft_pad(A + r * NS)];
      vb[r] = src[fft_pad(B + r * NS)];
    }
#pragma unroll
    for (int r = 1; r < R; ++r) {
      va[r] = cmul(va[r], twl[A * (R - 1) + (r - 1)]);
      vb[r] = cmul(vb[r], twl[B * (R - 1) + (r - 1)]);
    }
    dft<R>(va);
    dft<R>(vb);
    auto emit = [&](int k, float2 zk, float2 zm) {
      // E = (Z[k] + conj Z[F-k]) / 2,  O = (Z[k] - conj Z[F-k]) / (2i)
      const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      float2 x = cadd(e, cmul(__ldg(rw + k), o));
      const float h = (k == 0) ? xscale : 2.f * xscale;
      x.x *= h;
      x.y *= h;
      store_x(X, (size_t)k * n_ch + c0 + tr, x);
    };
#pragma unroll
    for (int r = 0; r < R; ++r) {
      emit(A + r * NS, va[r], t == 0 ? va[(R - r) % R] : vb[R - 1 - r]);
      emit(B + r * NS, vb[r], t == 0 ? vb[R - 1 - r] : va[R - 1 - r]);
    }
  }
}

// Persistent form of k_spectrum: each CTA loops over groups of C channels;
// the group's records (contiguous T samples each) arrive by 1D bulk copies in
// a staging buffer while the previous group is transformed and stored.
// Records must be 16-byte aligned (T * sizeof(TIn) is a multiple of 16 for
// every supported T).  Bounded waits as in k_inverse_tma.
template <int F, int C, int NT, typename TIn, typename TOut>
__global__ void __launch_bounds__(NT, (F == 1024 || F == 2048) ? 2 : 1) k_spectrum_tma(const TIn *__restrict__ rf,
                                                        const int32_t *__restrict__ tx_rows, int L, int n_ch,
                                                        const float2 *__restrict__ tw,
                                                        const float2 *__restrict__ rw,
                                                        TOut *__restrict__ X, float xscale, int *status) {
  constexpr int FS = fft_row(F);
  constexpr int T = 2 * F;
  constexpr int VE = 16 / (int)sizeof(TIn);  // samples per 16-byte vector
  constexpr int NV = T / VE;                 // vectors per record
  constexpr unsigned kRec = (unsigned)(T * sizeof(TIn));
  extern __shared__ __align__(128) float2 sm[];
  float2 *buf = sm;                                                       // [C][FS]
  float2 *s_tw = buf + C * FS;                                            // twiddles
  uint4 *stg = reinterpret_cast<uint4 *>(s_tw + ((fft_twoff(F, fft_npass(F)) + 1) & ~1));  // [C][NV]
  __shared__ __align__(8) uint64_t bar;
  __shared__ long long s_row[C];
  const int tid = threadIdx.x;
  const int n_groups = (n_ch + C - 1) / C;
  for (int i = tid; i < fft_twoff(F, fft_npass(F)); i += NT) s_tw[i] = __ldg(tw + i);
  if (tid == 0) tc::mbar_init(&bar, 1);
  tc::mbar_init_fence();
  __syncthreads();
  auto issue = [&](int g) {  // one thread
    const int c0 = g * C;
    const int nc = min(C, n_ch - c0);
    tma::mbar_expect_tx(&bar, kRec * (unsigned)nc);
    for (int cc = 0; cc < nc; ++cc) {
      const int c = c0 + cc;
      const int iu = c / L, l = c - iu * L;
      const long long r = ((long long)__ldg(tx_rows + iu) * L + l) * T;
      tma::bulk_1d(tc::smem_u32(stg + cc * NV), rf + r, kRec, &bar);
    }
  };
  int g = blockIdx.x;
  if (tid == 0 && g < n_groups) issue(g);
  uint32_t phase = 0;
  for (; g < n_groups; g += gridDim.x) {
    const bool ok = tc::mbar_wait(&bar, phase);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(status, (int)KK_ERR_TIMEOUT);
        tc::mbar_wait(&bar, phase);
      }
      return;
    }
    phase ^= 1u;
    const int c0 = g * C;
    const int nc = min(C, n_ch - c0);
    first_pass_staged<F, FS, C, NT, TIn>(stg, NV, nc, buf, tid);
    __syncthreads();  // staging consumed: prefetch the next group
    if (tid == 0 && g + (int)gridDim.x < n_groups) issue(g + gridDim.x);
    run_passes<F, FS, C, NT, 1, fft_npass(F) - 1>(buf, s_tw, tid);
    last_pass_spectrum<F, FS, C, NT, TOut>(buf, s_tw, rw, nc, c0, n_ch, xscale, X, tid);
    __syncthreads();  // buffers free for the next group
  }
  (void)s_row;
}

// ---- inverse of a half spectrum -------------------------------------------
// out[row][t], row < nrow, from Y[k][col(row)] (col = identity if null).
// rng (null: every sample): per output row, the samples [lo, hi) to store;
// a 16-byte store of samples (2m, 2m + 1) happens when it overlaps them.
template <int F, int C, int NT>
__global__ void __launch_bounds__(NT) k_inverse(const int2 *__restrict__ rng, const float2 *__restrict__ Y, int ncol,
                                                const int32_t *__restrict__ col_of_row, int nrow,
                                                const float2 *__restrict__ tw,
                                                const float2 *__restrict__ rw,
                                                float2 *__restrict__ out, float scale,
                                                const float *__restrict__ row_w,
                                                const int32_t *__restrict__ out_row) {
  constexpr int FS = fft_row(F);
  constexpr int T = 2 * F;
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * C;
  __shared__ int s_q[C];  // column of Y for each row, -1 past the last row
  float2 *s_tw = sm + 2 * C * FS;  // twiddles of every pass
  for (int i = tid; i < fft_twoff(F, fft_npass(F)); i += NT) s_tw[i] = __ldg(tw + i);
  if (tid < C) {
    const int row = r0 + tid;
    s_q[tid] = row < nrow ? (col_of_row ? __ldg(col_of_row + row) : row) : -1;
  }
  __syncthreads();
#pragma unroll 4
  for (int idx = tid; idx < C * F; idx += NT) {
    const int k = idx / C, rr = idx - k * C;
    const int q = s_q[rr];
    float2 y = make_float2(0.f, 0.f);
    if (q >= 0) y = __ldg(Y + (size_t)k * ncol + q);
    // inverse via conj(FFT(conj(.))): even samples from conj(Y),
    // odd samples from conj(Y e^{+2 pi i k/T}) = conj(Y) e^{-2 pi i k/T}
    const float2 a = make_float2(y.x, -y.y);
    sm[(2 * rr) * FS + fft_pad(k)] = a;
    sm[(2 * rr + 1) * FS + fft_pad(k)] = cmul(a, __ldg(rw + k));
  }
  __syncthreads();
  run_passes<F, FS, 2 * C, NT, 0>(sm, s_tw, tid);
  for (int idx = tid; idx < C * F; idx += NT) {
    const int rr = idx / F, m = idx - rr * F;
    const int row = r0 + rr;
    if (row >= nrow) continue;
    const float2 ev = sm[(2 * rr) * FS + fft_pad(m)];
    const float2 od = sm[(2 * rr + 1) * FS + fft_pad(m)];
    const float sc = row_w ? scale * __ldg(row_w + row) : scale;
    const float4 o = make_float4(ev.x * sc, -ev.y * sc, od.x * sc, -od.y * sc);
    const size_t orow = out_row ? (size_t)__ldg(out_row + row) : (size_t)row;
    const int2 rg = rng ? __ldg(rng + orow) : make_int2(0, T);
    if (2 * m + 1 >= rg.x && 2 * m < rg.y) *reinterpret_cast<float4 *>(out + orow * T + 2 * m) = o;
  }
}

// ---- fused first and last passes of the persistent inverse -----------------
// First pass (NS = 1) of the 2C transforms read straight from the staged Y
// tile [F][C]: transform 2 rr takes conj Y[k][rr], transform 2 rr + 1 takes
// conj Y[k][rr] e^{-2 pi i k / T}.  Lanes run over records first, so a warp
// reads contiguous runs of the tile.
template <int F, int FS, int C, int NT>
__device__ __forceinline__ void first_pass_inverse(const float2 *stg, const float2 *rw, float2 *buf, int tid) {
  constexpr int R = fft_radix(F, 0);
  static_assert(fft_ns(F, 0) == 1, "first pass has NS = 1");
  constexpr int NB = F / R;
  for (int j = tid; j < 2 * C * NB; j += NT) {
    const int rr = j % C, rest = j / C;
    const int jj = rest % NB, odd = rest / NB;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = jj + r * NB;
      const float2 y = stg[k * C + rr];
      const float2 a = make_float2(y.x, -y.y);
      v[r] = odd ? cmul(a, __ldg(rw + k)) : a;
    }
    dft<R>(v);
    float2 *dst = buf + (2 * rr + odd) * FS;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[fft_pad(jj * R + r)] = v[r];
  }
}

// Last pass (NS = F / R) of both transforms of a record, fused with the
// store: output r of butterfly jj is point m = jj + r NS of the even and the
// odd transform, i.e. samples 2m and 2m + 1 of the record, written as one
// 16-byte store (conjugated and scaled).  Lanes run over jj, so a warp
// store covers 512 contiguous bytes.
template <int F, int FS, int C, int NT>
__device__ __forceinline__ void last_pass_inverse(const float2 *buf, const float2 *tw, int r0, int nrow,
                                                  float2 *out, float scale, const float *row_w,
                                                  const int32_t *out_row, int tid, const int2 *rng) {
  constexpr int LAST = fft_npass(F) - 1;
  constexpr int R = fft_radix(F, LAST);
  constexpr int NS = fft_ns(F, LAST);
  constexpr int T = 2 * F;
  const float2 *twl = tw + fft_twoff(F, LAST);
  for (int idx = tid; idx < C * NS; idx += NT) {
    const int rr = idx / NS, jj = idx - rr * NS;
    const int row = r0 + rr;
    if (row >= nrow) continue;
    const float2 *se = buf + (2 * rr) * FS, *so = se + FS;
    float2 ve[R], vo[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ve[r] = se[fft_pad(jj + r * NS)];
      vo[r] = so[fft_pad(jj + r * NS)];
    }
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const float2 w = twl[jj * (R - 1) + (r - 1)];
      ve[r] = cmul(ve[r], w);
      vo[r] = cmul(vo[r], w);
    }
    dft<R>(ve);
    dft<R>(vo);
    const float sc = row_w ? scale * __ldg(row_w + row) : scale;
    const size_t orr = out_row ? (size_t)__ldg(out_row + row) : (size_t)row;
    float2 *orow = out + orr * T;
    const int2 rg = rng ? __ldg(rng + orr) : make_int2(0, T);  // samples to store
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = jj + r * NS;
      if (2 * m + 1 >= rg.x && 2 * m < rg.y)
        *reinterpret_cast<float4 *>(orow + 2 * m) =
            make_float4(ve[r].x * sc, -ve[r].y * sc, vo[r].x * sc, -vo[r].y * sc);
    }
  }
}

// ---- inverse with TMA prefetch (persistent) ---------------------------------
// The same transform as k_inverse for the common case where row r reads
// column r of Y (col_of_row is the identity) and ncol is even: each CTA loops
// over groups of C consecutive rows; the group's Y tile [F][C] arrives by 2D
// bulk copies (boxes of up to 256 bins x C columns) in a staging buffer while
// the previous group is transformed and stored, so the strided 8C-byte runs
// of the bin-major Y never stall the transform.  Every wait is bounded; a CTA
// that gives up sets *status to KK_ERR_TIMEOUT, waits (bounded) for the copy
// it issued and returns.
template <int F, int C, int NT>
__global__ void __launch_bounds__(NT, (F == 1024 || F == 2048) ? 2 : 1) k_inverse_tma(const __grid_constant__ CUtensorMap ymap, int nrow,
                                                    const float2 *__restrict__ tw,
                                                    const float2 *__restrict__ rw,
                                                    float2 *__restrict__ out, float scale,
                                                    const float *__restrict__ row_w,
                                                    const int32_t *__restrict__ out_row, int *status,
                                                    const int2 *__restrict__ rng) {
  constexpr int FS = fft_row(F);
  constexpr int BK = F < 256 ? F : 256;  // bins per box
  constexpr unsigned kTx = (unsigned)(C * F * sizeof(float2));
  extern __shared__ __align__(128) float2 sm[];
  float2 *stg = sm;                     // [F][C] tile of Y (bin-major, as in global memory)
  float2 *buf = sm + C * F;             // [2C][FS] transforms
  float2 *s_tw = buf + 2 * C * FS;      // twiddles of every pass
  __shared__ __align__(8) uint64_t bar;
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  const int n_groups = (nrow + C - 1) / C;
  for (int i = tid; i < fft_twoff(F, fft_npass(F)); i += NT) s_tw[i] = __ldg(tw + i);
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    s_bad = 0;
  }
  tc::mbar_init_fence();
  __syncthreads();
  auto issue = [&](int g) {
    tma::mbar_expect_tx(&bar, kTx);
#pragma unroll
    for (int b = 0; b < F / BK; ++b)
      tma::tma_2d(tc::smem_u32(stg + b * BK * C), &ymap, g * C, b * BK, &bar);
  };
  int g = blockIdx.x;
  if (tid == 0 && g < n_groups) issue(g);
  uint32_t phase = 0;
  for (; g < n_groups; g += gridDim.x) {
    const bool ok = tc::mbar_wait(&bar, phase);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicExch(status, (int)KK_ERR_TIMEOUT);
        tc::mbar_wait(&bar, phase);  // bounded: let the copy in flight land before exiting
      }
      return;
    }
    phase ^= 1u;
    const int r0 = g * C;
    // first pass from the staged tile: conj(Y) to the even transform,
    // conj(Y) e^{-2 pi i k / T} to the odd one
    first_pass_inverse<F, FS, C, NT>(stg, rw, buf, tid);
    __syncthreads();  // staging consumed: prefetch the next group while transforming this one
    if (tid == 0 && g + (int)gridDim.x < n_groups) issue(g + gridDim.x);
    run_passes<F, FS, 2 * C, NT, 1, fft_npass(F) - 1>(buf, s_tw, tid);
    last_pass_inverse<F, FS, C, NT>(buf, s_tw, r0, nrow, out, scale, row_w, out_row, tid, rng);
    __syncthreads();  // transforms stored: the buffers are free for the next group
  }
}

// ---- dispatch ----------------------------------------------------------------
template <int F>
struct FftCfg {
  static constexpr int CS = (F >= 1536) ? 4 : 8;   // records per CTA, forward
  static constexpr int CI = (F >= 1536) ? 2 : 4;   // records per CTA, inverse (2 transforms each)
  static constexpr int NT = (F <= 256) ? 256 : 512;
};

template <int F, typename TIn, typename TOut>
static cudaError_t spectrum_ft(const kk_plan &p, const void *rf, void *X, int n_ch,
                               const int32_t *rows, cudaStream_t s) {
  using Cfg = FftCfg<F>;
  if (((uintptr_t)rf % 16) == 0 && p.t.status && n_ch > 0) {
    constexpr int NV = 2 * F * (int)sizeof(TIn) / 16;
    const size_t tw_n = (size_t)((fft_twoff(F, fft_npass(F)) + 1) & ~1);
    const size_t smem = sizeof(float2) * ((size_t)Cfg::CS * fft_row(F) + tw_n) + sizeof(uint4) * Cfg::CS * NV;
    auto k = k_spectrum_tma<F, Cfg::CS, Cfg::NT, TIn, TOut>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int sms = 148, per_sm = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, Cfg::NT, smem);
    const int groups = (n_ch + Cfg::CS - 1) / Cfg::CS;
    const int grid = std::max(1, std::min(groups, sms * std::max(per_sm, 1)));
    k<<<grid, Cfg::NT, smem, s>>>((const TIn *)rf, rows, p.L, n_ch, p.t.fft_tw, p.t.rfft_w, (TOut *)X, p.x_scale,
                                  p.t.status);
    return cudaGetLastError();
  }
  const size_t smem = sizeof(float2) * (Cfg::CS * fft_row(F) + fft_twoff(F, fft_npass(F)));
  const dim3 grid((n_ch + Cfg::CS - 1) / Cfg::CS);
  const bool vec = ((uintptr_t)rf % 16) == 0;
  auto k = vec ? k_spectrum<F, Cfg::CS, Cfg::NT, TIn, TOut, true> : k_spectrum<F, Cfg::CS, Cfg::NT, TIn, TOut, false>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<grid, Cfg::NT, smem, s>>>((const TIn *)rf, rows, p.L, n_ch, p.t.fft_tw, p.t.rfft_w, (TOut *)X,
                                p.x_scale);
  return cudaGetLastError();
}

template <int F, typename TIn>
static cudaError_t spectrum_fi(const kk_plan &p, const void *rf, void *X, int n_ch,
                               const int32_t *rows, cudaStream_t s) {
  switch (p.precision) {
    case KK_PREC_BF16: return spectrum_ft<F, TIn, __nv_bfloat162>(p, rf, X, n_ch, rows, s);
    case KK_PREC_F16:
    case KK_PREC_F8E4M3: return spectrum_ft<F, TIn, __half2>(p, rf, X, n_ch, rows, s);
    default: return spectrum_ft<F, TIn, float2>(p, rf, X, n_ch, rows, s);
  }
}

template <int F>
static cudaError_t spectrum_f(const kk_plan &p, const void *rf, void *X, int n_rows,
                              const int32_t *rows, cudaStream_t s) {
  const int n_ch = n_rows * p.L;
  if (p.rf_dtype == KK_RF_I16) return spectrum_fi<F, int16_t>(p, rf, X, n_ch, rows, s);
  return spectrum_fi<F, float>(p, rf, X, n_ch, rows, s);
}

// Y [F][ncol] complex as (ncol, F) 8-byte elements, box {C, min(F, 256)}
static bool map_y(CUtensorMap *m, const float2 *Y, int ncol, int F, int C) {
  tma::EncodeFn enc = tma::encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)ncol, (cuuint64_t)F};
  const cuuint64_t strides[1] = {(cuuint64_t)ncol * sizeof(float2)};
  const cuuint32_t box[2] = {(cuuint32_t)C, (cuuint32_t)(F < 256 ? F : 256)};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<float2 *>(Y), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int F>
static cudaError_t inverse_f(const kk_plan &p, const float2 *Y, int ncol, const int32_t *col,
                             int nrow, float2 *out, cudaStream_t s, const float *row_w,
                             const int32_t *out_row) {
  using Cfg = FftCfg<F>;
  // KK plans with record trimming store only each record's reachable samples
  const int2 *rng = (!p.is_das && p.trim) ? p.t.rec_range : nullptr;
  // TMA path: identity column map (col null, or rows reading columns 0..nrow-1
  // in order, flagged by the plan), even ncol, 16-byte aligned Y
  if (col == nullptr && ncol % 2 == 0 && nrow <= ncol && ((uintptr_t)Y % 16) == 0 && p.t.status) {
    CUtensorMap m;
    if (map_y(&m, Y, ncol, F, Cfg::CI)) {
      const size_t smem = sizeof(float2) * ((size_t)Cfg::CI * F + 2 * Cfg::CI * fft_row(F) +
                                            fft_twoff(F, fft_npass(F)));
      auto k = k_inverse_tma<F, Cfg::CI, Cfg::NT>;
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int sms = 148, per_sm = 1;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, Cfg::NT, smem);
      const int groups = (nrow + Cfg::CI - 1) / Cfg::CI;
      const int grid = std::max(1, std::min(groups, sms * std::max(per_sm, 1)));
      k<<<grid, Cfg::NT, smem, s>>>(m, nrow, p.t.fft_tw, p.t.rfft_w, out, (float)(1.0 / (double)(2 * F)),
                                    row_w, out_row, p.t.status, rng);
      return cudaGetLastError();
    }
  }
  const size_t smem = sizeof(float2) * (2 * Cfg::CI * fft_row(F) + fft_twoff(F, fft_npass(F)));
  auto k = k_inverse<F, Cfg::CI, Cfg::NT>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const dim3 grid((nrow + Cfg::CI - 1) / Cfg::CI);
  k<<<grid, Cfg::NT, smem, s>>>(rng, Y, ncol, col, nrow, p.t.fft_tw, p.t.rfft_w, out,
                                (float)(1.0 / (double)(2 * F)), row_w, out_row);
  return cudaGetLastError();
}

cudaError_t launch_spectrum(const kk_plan &p, const void *rf, void *X, int n_rows,
                            const int32_t *rows, cudaStream_t s) {
  switch (p.F) {
    case 128: return spectrum_f<128>(p, rf, X, n_rows, rows, s);
    case 256: return spectrum_f<256>(p, rf, X, n_rows, rows, s);
    case 512: return spectrum_f<512>(p, rf, X, n_rows, rows, s);
    case 768: return spectrum_f<768>(p, rf, X, n_rows, rows, s);
    case 1024: return spectrum_f<1024>(p, rf, X, n_rows, rows, s);
    case 1536: return spectrum_f<1536>(p, rf, X, n_rows, rows, s);
    case 2048: return spectrum_f<2048>(p, rf, X, n_rows, rows, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_inverse(const kk_plan &p, const float2 *Y, int ncol, const int32_t *col,
                           int nrow, float2 *out, cudaStream_t s, const float *row_w,
                           const int32_t *out_row) {
  switch (p.F) {
    case 128: return inverse_f<128>(p, Y, ncol, col, nrow, out, s, row_w, out_row);
    case 256: return inverse_f<256>(p, Y, ncol, col, nrow, out, s, row_w, out_row);
    case 512: return inverse_f<512>(p, Y, ncol, col, nrow, out, s, row_w, out_row);
    case 768: return inverse_f<768>(p, Y, ncol, col, nrow, out, s, row_w, out_row);
    case 1024: return inverse_f<1024>(p, Y, ncol, col, nrow, out, s, row_w, out_row);
    case 1536: return inverse_f<1536>(p, Y, ncol, col, nrow, out, s, row_w, out_row);
    case 2048: return inverse_f<2048>(p, Y, ncol, col, nrow, out, s, row_w, out_row);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace kk
