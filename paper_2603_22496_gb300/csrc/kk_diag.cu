// kk_diag.cu -- checks of the library's failure detection: the bounded
// device-side waits, and the counters of the bounds-checked build.
//
// Every pipelined kernel of the library (bulk-copy-fed FFTs and contractions,
// tensor-core contractions and convolutions) waits on mbarriers through
// kk::tc::mbar_wait, which gives up after a time limit; the kernel then
// records KK_ERR_TIMEOUT in a status word and returns.  kk_plan_check_wait_
// timeout makes that path run: a CTA waits, through the same bounded wait,
// on an mbarrier that nothing signals, and records the timeout in the plan's
// status word.  No copy or MMA is in flight, so nothing outlives the kernel.
#include <algorithm>

#include "kk_internal.h"
#include "kk_tc.h"

namespace kk {
namespace {

__global__ void __launch_bounds__(128) k_wait_unsignalled(unsigned long long limit_ns, int *status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);  // one arrival completes phase 0; none ever comes
    tc::mbar_init_fence();
  }
  __syncthreads();
  const bool ok = tc::mbar_wait_for(&bar, 0u, limit_ns);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(status, (int)KK_ERR_TIMEOUT);
}

}  // namespace
}  // namespace kk

using namespace kk;

extern "C" kk_status kk_plan_check_wait_timeout(const kk_plan *p, int64_t limit_ns, void *stream) {
  if (!p) { set_error("null plan"); return KK_ERR_INVALID_ARG; }
  const unsigned long long lim =
      (unsigned long long)std::min<int64_t>(std::max<int64_t>(limit_ns, 1000), 1000000000);
  DeviceGuard guard(p->device);
  if (!guard.ok) { set_error("cudaSetDevice failed"); return KK_ERR_CUDA; }
  k_wait_unsignalled<<<1, 128, 0, (cudaStream_t)stream>>>(lim, p->t.status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "wait-timeout check launch");
  return KK_OK;
}

extern "C" kk_status kk_debug_bounds(int64_t *violations) {
  if (!violations) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
#ifdef KK_DEBUG_BOUNDS
  unsigned long long a = 0, b = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = take_bounds_kk(&a);
  if (e == cudaSuccess) e = take_bounds_das(&b);
  if (e != cudaSuccess) return cuda_fail(e, "bounds counters");
  *violations = (int64_t)(a + b);
  return KK_OK;
#else
  *violations = 0;
  set_error("not a bounds-checked build (compile with KK_DEBUG_BOUNDS)");
  return KK_ERR_UNSUPPORTED;
#endif
}
