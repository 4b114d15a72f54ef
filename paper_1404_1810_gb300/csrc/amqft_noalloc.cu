// Allocation-free execution of the multi-pass path (include/amqft.h,
// amqft_exec_static).  The paper has no counterpart: the AM-QFT arithmetic is
// the multi-pass kernels' own; only the place of their workspace changes.
//
// Who needs it: callers that must not allocate device memory when they run a
// transform.  cudaMalloc/cudaFree may synchronise the whole device (stalling
// every other stream of the process), fail once another allocator (a caching
// allocator, an arena of a serving process) owns the free memory, and are not
// allowed at all in some contexts; a plan for 2^17..2^24 allocates its
// workspace (up to 2 GiB) when it is created and holds it for its lifetime,
// too much for callers that keep many plans of different lengths.  Here the
// workspace is a fixed device array compiled into the library, shared by all
// plans on a device; a plan created with batch 0 holds only its constant
// table.
//
// The scratch holds two ping-pong buffers of 4 regions per transform for up to
// AMQFT_STATIC_SCRATCH_FLOATS floats: two transforms of 2^20 per chunk, 15 of
// 2^17.  Nothing in it needs to start at zero: every word that feeds a result
// is written by the load pass of the same call before any other pass reads
// it; the pad words after each region are copied between the buffers but
// never used.  Calls on one device
// that overlap in time (on different streams, or from several host threads
// without ordering) race on the scratch; calls on one stream are ordered.
#include <stdint.h>

#include "amqft.h"
#include "amqft_internal.h"
#include "amqft_multipass_impl.cuh"

namespace amqft {
namespace {

static_assert(AMQFT_STATIC_SCRATCH_FLOATS == 2LL * 2 * 4 * ((1LL << (AMQFT_STATIC_LOG2N_MAX - 1)) + 32),
              "the static scratch holds two transforms of the largest length");

// The workspace: a file-scope device array, one per device (the module is
// loaded into each device's context), zero-filled at load and never freed.
static __device__ __align__(256) float g_scratch[AMQFT_STATIC_SCRATCH_FLOATS];

// Device address of g_scratch in the current context.  Looked up on every
// call (a host-side lookup) rather than cached, so that a context destroyed
// and recreated (cudaDeviceReset, a framework resetting the device) never
// leaves a stale address behind.
cudaError_t scratch_address(float** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<float*>(p);
  return cudaSuccess;
}

}  // namespace
}  // namespace amqft

using namespace amqft;

extern "C" int amqft_exec_static(amqft_plan_t plan, int64_t batch, const void* in, void* out, int inverse,
                                 void* stream) {
  clear_error();
  PlanView pv;
  int rc = plan_view(plan, &pv);
  if (rc != AMQFT_OK) return set_error(rc, "amqft_exec_static: plan is NULL");
  if (pv.log2n < AMQFT_STATIC_LOG2N_MIN || pv.log2n > AMQFT_STATIC_LOG2N_MAX)
    return set_error(AMQFT_ERR_N,
                     "amqft_exec_static: log2n=%d outside [%d, %d]: the static scratch (%lld floats) holds the "
                     "multi-pass workspace up to 2^%d; lengths up to 2^%d use no workspace (amqft_exec_fwd/inv)",
                     pv.log2n, AMQFT_STATIC_LOG2N_MIN, AMQFT_STATIC_LOG2N_MAX, (long long)AMQFT_STATIC_SCRATCH_FLOATS,
                     AMQFT_STATIC_LOG2N_MAX, AMQFT_LOG2N_FUSED_MAX);
  if (pv.dtype != AMQFT_C64) return set_error(AMQFT_ERR_DTYPE, "amqft_exec_static: AMQFT_C64 plans only");
  if (batch < 0) return set_error(AMQFT_ERR_ARG, "amqft_exec_static: batch=%lld < 0", (long long)batch);
  if (batch == 0) return AMQFT_OK;
  if (!in || !out) return set_error(AMQFT_ERR_ALIGN, "amqft_exec_static: in or out is NULL");
  if (((uintptr_t)in | (uintptr_t)out) & 7u)
    return set_error(AMQFT_ERR_ALIGN, "amqft_exec_static: in/out must be 8-byte aligned");
  const long long N = 1LL << pv.log2n;
  const uintptr_t bytes = (uintptr_t)(N * batch * 8);
  const uintptr_t a0 = (uintptr_t)in, b0 = (uintptr_t)out;
  if (a0 != b0 && a0 < b0 + bytes && b0 < a0 + bytes)
    return set_error(AMQFT_ERR_INPLACE, "amqft_exec_static: in and out overlap without being equal");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(AMQFT_ERR_CUDA, "amqft_exec_static: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev != pv.device)
    return set_error(AMQFT_ERR_DEVICE, "amqft_exec_static: current device %d, plan was made on device %d", dev,
                     pv.device);
  float* scratch = nullptr;
  e = scratch_address(&scratch);
  if (e != cudaSuccess)
    return set_error(AMQFT_ERR_CUDA, "amqft_exec_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  // same region geometry as a plan's own workspace
  const long long RSg = ((N / 2 + 2 + 31) / 32) * 32;
  const long long per_t = 2LL * 4 * RSg;
  const long long chunk = AMQFT_STATIC_SCRATCH_FLOATS / per_t;  // >= 2 for log2n <= AMQFT_STATIC_LOG2N_MAX
  cudaStream_t st = (cudaStream_t)stream;
  for (long long t0 = 0; t0 < batch; t0 += chunk) {
    MpArgs a = {};
    a.in = in;
    a.out = out;
    a.exp_in = nullptr;
    a.exp_out = nullptr;
    a.dtype = AMQFT_C64;
    a.ctab = pv.ctab;
    a.nt = (batch - t0) < chunk ? (batch - t0) : chunk;
    a.t0 = t0;
    a.logN = pv.log2n;
    a.inverse = inverse ? 1 : 0;
    a.RSg = RSg;
    a.tlist = nullptr;
    a.toff = nullptr;
    a.ntdev = nullptr;
    long long nl = 0;
    e = multipass_dispatch(pv.variant, a, scratch, scratch + chunk * 4 * RSg, *pv.small, st, &nl);
    add_launches(plan, nl);
    if (e != cudaSuccess)
      return set_error(AMQFT_ERR_CUDA, "amqft_exec_static: multi-pass launch: %s", cudaGetErrorString(e));
  }
  return AMQFT_OK;
}
