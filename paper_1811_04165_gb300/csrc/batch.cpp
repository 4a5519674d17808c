// Batched beams: one CUDA graph holding every beam's search.
//
// Beams are independent (Sec. 1: the ALERT survey spreads its beams over a GPU
// cluster), so the graph forks into `branches` concurrent chains; each chain
// owns a region of the caller's workspace and searches its beams one after the
// other (pre-pass, de-dispersion, S/N, detection per beam).  Beams are assigned
// largest first to the chain with the least work so far (work = DM trials x
// samples x channels).  Capture happens once, at creation; a launch is one
// cudaGraphLaunch.  The graph holds raw pointers to the plans' device tables,
// so every launch first checks that no plan has been reconfigured since.
#include <algorithm>
#include <numeric>
#include <vector>

#include "sps_internal.h"

struct sps_batch {
  int device = 0;
  std::vector<const sps_plan*> plans;
  std::vector<uint64_t> gens;  // each plan's configuration generation at capture
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace sps {
namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

double beam_work(const sps_plan* p) { return (double)p->dms.size() * p->n_t * p->channels; }

// Branch of each beam and the workspace each branch needs.
sps_status assign(const sps_plan* const* plans, int32_t n, int32_t branches, std::vector<int32_t>* branch_of,
                  std::vector<size_t>* ws) {
  if (!plans || n < 1) return fail(SPS_ERR_INVALID_ARG, "need at least one beam");
  if (branches < 1) return fail(SPS_ERR_INVALID_ARG, "branches must be >= 1");
  const int32_t B = std::min(branches, n);
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  for (int32_t b = 0; b < n; b++)
    if (!plans[b]) return fail(SPS_ERR_INVALID_ARG, "null plan");
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return beam_work(plans[a]) > beam_work(plans[b]); });
  std::vector<double> load(B, 0.0);
  branch_of->assign(n, 0);
  ws->assign(B, 0);
  for (int32_t b : order) {
    const int32_t k = (int32_t)(std::min_element(load.begin(), load.end()) - load.begin());
    (*branch_of)[b] = k;
    load[k] += beam_work(plans[b]);
    (*ws)[k] = std::max((*ws)[k], plan_workspace_bytes(plans[b]));
  }
  return SPS_OK;
}

}  // namespace
}  // namespace sps

using namespace sps;

extern "C" {

sps_status sps_batch_workspace_bytes(const sps_plan* const* plans, int32_t n_beams, int32_t branches,
                                     size_t* bytes) {
  clear_error();
  if (!bytes) return fail(SPS_ERR_INVALID_ARG, "null argument");
  std::vector<int32_t> branch_of;
  std::vector<size_t> ws;
  if (sps_status s = assign(plans, n_beams, branches, &branch_of, &ws)) return s;
  size_t total = 0;
  for (size_t w : ws) total += round_up(w);
  *bytes = total;
  return SPS_OK;
}

sps_status sps_batch_create(const sps_plan* const* plans, const sps_beam_buffers* buffers, int32_t n_beams,
                            int32_t branches, void* workspace, size_t workspace_bytes, sps_batch** out) {
  clear_error();
  if (!out || !buffers) return fail(SPS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  std::vector<int32_t> branch_of;
  std::vector<size_t> ws;
  if (sps_status s = assign(plans, n_beams, branches, &branch_of, &ws)) return s;
  const int device = plans[0]->device;
  for (int32_t b = 0; b < n_beams; b++)
    if (plans[b]->device != device) return fail(SPS_ERR_INVALID_ARG, "all plans must be on one device");
  std::vector<size_t> offset(ws.size(), 0);
  size_t total = 0;
  for (size_t k = 0; k < ws.size(); k++) {
    offset[k] = total;
    total += round_up(ws[k]);
  }
  if (!workspace || workspace_bytes < total || ((uintptr_t)workspace % kAlign))
    return fail(SPS_ERR_INVALID_ARG, "workspace missing, smaller than sps_batch_workspace_bytes or not 256-byte aligned");

  int cur = 0;
  SPS_CUDA(cudaGetDevice(&cur));
  if (cur != device) SPS_CUDA(cudaSetDevice(device));
  const int32_t B = (int32_t)ws.size();
  std::vector<cudaStream_t> streams(B, nullptr);
  std::vector<cudaEvent_t> joins(B, nullptr);
  cudaStream_t cap = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  sps_status st = SPS_OK;
  auto cuda_ok = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == SPS_OK) st = cuda_fail(e, what);
    return st == SPS_OK;
  };
  if (cuda_ok(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreateWithFlags") &&
      cuda_ok(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "cudaEventCreateWithFlags")) {
    for (int32_t k = 0; k < B && st == SPS_OK; k++) {
      cuda_ok(cudaStreamCreateWithFlags(&streams[k], cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
      if (st == SPS_OK) cuda_ok(cudaEventCreateWithFlags(&joins[k], cudaEventDisableTiming), "cudaEventCreateWithFlags");
    }
  }
  if (st == SPS_OK && cuda_ok(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture")) {
    cuda_ok(cudaEventRecord(fork, cap), "cudaEventRecord");
    for (int32_t k = 0; k < B && st == SPS_OK; k++) cuda_ok(cudaStreamWaitEvent(streams[k], fork, 0), "cudaStreamWaitEvent");
    for (int32_t b = 0; b < n_beams && st == SPS_OK; b++) {
      const sps_beam_buffers& u = buffers[b];
      const int32_t k = branch_of[b];
      uint8_t* w = static_cast<uint8_t*>(workspace) + offset[k];
      st = run_search(plans[b], u.x, u.x_pitch, u.D, w, ws[k], u.snr, u.peak_t, u.peak_val, u.best, streams[k]);
    }
    // join every branch, also after a failure, so that the capture ends cleanly
    for (int32_t k = 0; k < B; k++) {
      cuda_ok(cudaEventRecord(joins[k], streams[k]), "cudaEventRecord");
      cuda_ok(cudaStreamWaitEvent(cap, joins[k], 0), "cudaStreamWaitEvent");
    }
    cuda_ok(cudaStreamEndCapture(cap, &graph), "cudaStreamEndCapture");
  }
  sps_batch* batch = nullptr;
  if (st == SPS_OK) {
    batch = new sps_batch();
    batch->device = device;
    batch->graph = graph;
    graph = nullptr;
    if (!cuda_ok(cudaGraphInstantiate(&batch->exec, batch->graph, 0), "cudaGraphInstantiate")) {
      cudaGraphDestroy(batch->graph);
      delete batch;
      batch = nullptr;
    } else {
      for (int32_t b = 0; b < n_beams; b++) {
        batch->plans.push_back(plans[b]);
        batch->gens.push_back(plans[b]->config_gen);
      }
    }
  }
  if (graph) cudaGraphDestroy(graph);
  for (int32_t k = 0; k < B; k++) {
    if (joins[k]) cudaEventDestroy(joins[k]);
    if (streams[k]) cudaStreamDestroy(streams[k]);
  }
  if (fork) cudaEventDestroy(fork);
  if (cap) cudaStreamDestroy(cap);
  if (cur != device) cudaSetDevice(cur);
  if (st != SPS_OK) return st;
  *out = batch;
  return SPS_OK;
}

sps_status sps_batch_launch(sps_batch* batch, void* stream) {
  clear_error();
  NvtxRange nvtx("sps_batch_launch");
  if (!batch) return fail(SPS_ERR_INVALID_ARG, "null batch");
  for (size_t b = 0; b < batch->plans.size(); b++)
    if (batch->plans[b]->config_gen != batch->gens[b])
      return fail(SPS_ERR_INVALID_ARG, "a plan was reconfigured after the batch was captured");
  SPS_CUDA(cudaGraphLaunch(batch->exec, (cudaStream_t)stream));
  return SPS_OK;
}

sps_status sps_batch_destroy(sps_batch* batch) {
  if (!batch) return SPS_OK;
  if (batch->exec) cudaGraphExecDestroy(batch->exec);
  if (batch->graph) cudaGraphDestroy(batch->graph);
  delete batch;
  return SPS_OK;
}

}  // extern "C"
