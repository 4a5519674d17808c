// De-dispersion for callers that cannot allocate device memory.
//
// sps_dedisperse needs a caller-provided workspace (the three shifted copies
// of the batch, and in subband mode the step-one series).  Some callers cannot
// provide one: a real-time beam loop that must keep a fixed device-memory
// footprint once the observation has started (an allocation there can stall
// the loop or fail under memory pressure), or code behind an interface that
// hands it only the input and output buffers.  sps_dedisperse_noalloc serves
// them: it runs the same kernels with a workspace carved from a file-scope
// device array of fixed size, and it allocates nothing.
//
// Costs and rules of the shared array:
//   * every device that loads this part of the library keeps the array
//     (kStaticScratchBytes) until the process exits;
//   * all calls on a device share it and it keeps the last call's contents;
//     nothing in it needs to start at zero (the kernels overwrite all they
//     read), but two calls whose work overlaps on the GPU (different streams,
//     or different host threads) race on it and corrupt each other's results;
//   * host code cannot use the array's name as a device address; every call
//     looks the address up (cudaGetSymbolAddress) with the plan's device
//     current.  The first call on a device loads the array there, so that first
//     call should come before any stream capture.  Later lookups are cheap, and
//     because none is cached, a device reset (which reloads the module,
//     possibly at another address) never leaves a stale address behind.
#include "sps_internal.h"

namespace sps {
namespace {

// 96 MiB: enough for the brute-force search of one 1536-channel, 1.024 s beam
// with the single-channel kernel (three shifted copies of 1536 x 17136 bytes,
// 79 MB), not for the pre-summed pair or quad series (236 or 614 MB) nor for
// the subband path.
constexpr size_t kStaticScratchBytes = size_t(96) << 20;

__device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device.
sps_status static_scratch(void** out) {
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
  *out = ptr;
  return SPS_OK;
}

}  // namespace
}  // namespace sps

using namespace sps;

extern "C" sps_status sps_dedisperse_noalloc(const sps_plan* plan, const uint8_t* x, int64_t x_pitch, int32_t* D,
                                              void* stream) {
  clear_error();
  if (!plan) return fail(SPS_ERR_INVALID_ARG, "null plan");
  const size_t need = plan_workspace_bytes(plan);
  if (need > kStaticScratchBytes)
    return fail(SPS_ERR_UNSUPPORTED, "this plan needs " + std::to_string(need) +
                                         " bytes of workspace; the static scratch of sps_dedisperse_noalloc holds " +
                                         std::to_string(kStaticScratchBytes) + " (use sps_dedisperse with a workspace)");
  int device = -1;
  SPS_CUDA(cudaGetDevice(&device));
  if (device != plan->device) return fail(SPS_ERR_INVALID_ARG, "the plan's device must be the current device");
  void* scratch = nullptr;
  if (sps_status s = static_scratch(&scratch)) return s;
  return dedisperse_into(plan, x, x_pitch, D, scratch, kStaticScratchBytes, (cudaStream_t)stream);
}
