// kk_sim.cu -- synthetic channel data on the GPU (input generation).
//
// Not part of the beamforming method: this produces the seeded synthetic
// RF that large benchmarks and the training of the learned refiner need in
// quantities a CPU cannot simulate.  Same forward model as the CPU input
// generator (linear superposition of two-way far-field delays, plane-wave
// transmit, spherical receive, Gaussian-modulated pulse), evaluated in FP32
// with fast intrinsics; the parity tests use CPU-generated inputs instead.
//
// One CTA per channel (transmit i, element l) accumulates every scatterer's
// pulse into a shared-memory record, then writes it out.  Optional white
// Gaussian noise comes from a counter-based generator (SplitMix64 hash of
// (seed, channel, sample) and a Box-Muller transform).
#include "kk_internal.h"

namespace kk {
namespace {

constexpr int kSimThreads = 256;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void __launch_bounds__(kSimThreads)
    k_simulate(const float2 *__restrict__ tx_sc, const float *__restrict__ elem_x, int L, int T,
               float fs_over_c, float fs, float f0, float alpha, float hw_samples,
               const float4 *__restrict__ scat, int n_scat, float noise_sigma,
               unsigned long long seed, float *__restrict__ rf) {
  extern __shared__ float acc[];  // [T]
  const int ch = blockIdx.x;
  const int i = ch / L, l = ch - i * L;
  const float2 sc = tx_sc[i];  // (sin, cos)
  const float u = elem_x[l];
  for (int t = threadIdx.x; t < T; t += kSimThreads) acc[t] = 0.f;
  __syncthreads();
  const float two_pi_f0_over_fs = 6.283185307f * f0 / fs;
  const float a_n = alpha / (fs * fs);  // Gaussian rate per sample^2
  for (int s = threadIdx.x; s < n_scat; s += kSimThreads) {
    const float4 p = scat[s];  // x, z, amplitude, unused
    const float dx = p.x - u;
    const float tau = fs_over_c * (p.x * sc.x + p.y * sc.y + sqrtf(dx * dx + p.y * p.y));  // samples
    int n0 = (int)ceilf(tau - hw_samples), n1 = (int)floorf(tau + hw_samples);
    n0 = max(n0, 0);
    n1 = min(n1, T - 1);
    for (int n = n0; n <= n1; ++n) {
      const float d = (float)n - tau;
      atomicAdd(&acc[n], p.z * __expf(-a_n * d * d) * __cosf(two_pi_f0_over_fs * d));
    }
  }
  __syncthreads();
  float *out = rf + (size_t)ch * T;
  for (int t = threadIdx.x; t < T; t += kSimThreads) {
    float v = acc[t];
    if (noise_sigma > 0.f) {
      const unsigned long long h = splitmix64(seed ^ splitmix64(((unsigned long long)ch << 32) | (unsigned)t));
      const float u1 = ((float)(h >> 40) + 1.f) * 0x1p-24f;  // (0, 1]
      const float u2 = (float)((h >> 16) & 0xFFFFFFull) * 0x1p-24f;
      v += noise_sigma * sqrtf(-2.f * __logf(u1)) * __cosf(6.283185307f * u2);
    }
    out[t] = v;
  }
}

}  // namespace
}  // namespace kk

using namespace kk;

extern "C" kk_status kk_simulate_rf(int32_t n_tx, const float *d_tx_sincos, int32_t n_elem,
                                    const float *d_elem_x, int32_t T, double fs, double c, double f0,
                                    double bw, int32_t n_scat, const float *d_scat, double noise_sigma,
                                    uint64_t seed, float *d_rf, void *stream) {
  if (n_tx < 1 || n_elem < 1 || T < 2 || n_scat < 0 || !d_tx_sincos || !d_elem_x || !d_rf ||
      (n_scat > 0 && !d_scat) || !(fs > 0) || !(c > 0) || !(f0 > 0) || !(bw > 0)) {
    set_error("bad simulation arguments");
    return KK_ERR_INVALID_ARG;
  }
  if ((size_t)T * sizeof(float) > 200 * 1024) { set_error("record too long for the simulator"); return KK_ERR_UNSUPPORTED; }
  // Gaussian envelope rate: spectrum at -6 dB at f0 (1 +- bw/2)
  const double alpha = 9.869604401089358 * f0 * f0 * bw * bw / (4.0 * std::log(std::pow(10.0, 6.0 / 20.0)));
  const double hw = 4.0 / std::sqrt(2.0 * alpha) * fs;  // +-4 sigma in samples
  const size_t smem = sizeof(float) * (size_t)T;
  cudaError_t e = cudaFuncSetAttribute(k_simulate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "simulator attribute");
  k_simulate<<<n_tx * n_elem, kSimThreads, smem, (cudaStream_t)stream>>>(
      (const float2 *)d_tx_sincos, d_elem_x, n_elem, T, (float)(fs / c), (float)fs, (float)f0,
      (float)alpha, (float)hw, (const float4 *)d_scat, n_scat, (float)noise_sigma, seed, d_rf);
  e = cudaGetLastError();
  return e == cudaSuccess ? KK_OK : cuda_fail(e, "simulator launch");
}
