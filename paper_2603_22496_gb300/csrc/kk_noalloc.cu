// kk_noalloc.cu -- KK image formation for callers that cannot allocate.
//
// kk_beamform keeps the partial images of its pair slices in the caller's
// workspace.  Some callers cannot provide one: code that runs where
// cudaMalloc is unavailable or forbidden (inside a host framework that owns
// all device memory through its own pool, a plugin loaded into such a
// process, a real-time loop that must not allocate).  For them this file
// holds the scratch in a fixed file-scope device array compiled into the
// library, and kk_beamform_noalloc launches the same gather and reduction
// kernels with it.  Nothing here calls cudaMalloc, cudaFree or any
// allocating routine.
#include "kk_internal.h"

namespace kk {
namespace {

// 8 MiB: one million complex partial pixels (pair slices x groups x pixels
// x y slices).  Every GPU that loads the library holds this array until the
// process exits.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;

static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocScratchBytes / sizeof(float2)];

// Device address of the scratch array on the current device.  Host code
// cannot use the symbol itself: it names a host-side stand-in.  Looked up on
// every call (cheap once the module is loaded), so a context that was torn
// down and re-created never receives a stale address.
kk_status scratch_address(void **out) {
  void *ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || ptr == nullptr) {
    if (e == cudaSuccess) e = cudaErrorInvalidSymbol;
    return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
  }
  *out = ptr;
  return KK_OK;
}

}  // namespace
}  // namespace kk

using namespace kk;

extern "C" kk_status kk_beamform_noalloc(const kk_plan *p, const void *d_rf_theta, void *d_B,
                                         float *d_I, void *stream) {
  NvtxRange range("kk_beamform_noalloc");
  kk_status st = check_beamform_args(p, d_rf_theta, d_B, d_I);
  if (st != KK_OK) return st;
  const size_t need = (p->bf_split > 1)
                          ? sizeof(float2) * (size_t)p->bf_split * p->J * p->grid.nx * p->grid.nz * p->ny
                          : 0;
  if (need > kNoAllocScratchBytes) {
    set_error("plan needs " + std::to_string(need) + " bytes of partial images; the no-allocation "
              "scratch holds " + std::to_string(kNoAllocScratchBytes) + " (use kk_beamform with a workspace)");
    return KK_ERR_INVALID_ARG;
  }
  DeviceGuard guard(p->device);
  if (!guard.ok) { set_error("cudaSetDevice failed"); return KK_ERR_CUDA; }
  void *scratch = nullptr;
  if (need > 0) st = scratch_address(&scratch);
  if (st != KK_OK) return st;
  // every slice writes each of its partial pixels, so nothing needs clearing
  cudaError_t e = launch_kk_gather(*p, (const float2 *)d_rf_theta, (float2 *)d_B, d_I,
                                   (float2 *)scratch, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "kk gather launch (no-allocation)");
  return KK_OK;
}
