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
#include "kk_internal.h"

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

template <int RI>
cudaError_t launch_ri(const kk_plan &p, const float2 *X, float2 *Y, cudaStream_t s) {
  const dim3 grid(p.F, (p.Mu + kTO - 1) / kTO, (p.Nu + 16 * RI - 1) / (16 * RI));
  k_shear_f32<RI><<<grid, 256, 0, s>>>(X, p.t.phase, p.L, p.Nu, p.Mu, Y);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_shear_f32(const kk_plan &p, const float2 *X, float2 *Y, cudaStream_t s) {
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
