// Failure-detection self-check: the bounded wait every kernel uses, made to
// run out on purpose.  One block initialises an mbarrier that nothing ever
// arrives at and waits on it for a given number of polls; the wait gives up,
// records kStatusWaitTimeout in the plan's status word and the block returns
// normally, so the context stays usable.  No copy is issued and no address is
// touched but the block's own shared memory and the status word.
#include "sps_internal.h"
#include "tma.cuh"

namespace sps {
namespace {

__global__ void __launch_bounds__(32) wait_runs_out_kernel(uint32_t* status, uint32_t polls) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  mbar_wait_polls(&bar, 0, status, polls);  // phase 0 never completes
}

}  // namespace
}  // namespace sps

using namespace sps;

extern "C" sps_status sps_plan_check_wait_timeout(const sps_plan* plan, int32_t polls, void* stream) {
  clear_error();
  if (!plan) return fail(SPS_ERR_INVALID_ARG, "null plan");
  if (polls < 1 || polls > (1 << 20)) return fail(SPS_ERR_INVALID_ARG, "polls must lie in [1, 2^20]");
  wait_runs_out_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(plan->d_status, (uint32_t)polls);
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}
