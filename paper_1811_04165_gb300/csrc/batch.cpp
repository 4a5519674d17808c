// Batched beams: one CUDA graph holding every beam's search.
//
// Beams are independent (Sec. 1: the ALERT survey spreads its beams over a GPU
// cluster), so the graph forks into `branches` concurrent chains.  Beams whose
// brute-force kernel is the pre-summed one are searched in three phases: their
// pre-passes (series into each beam's own workspace region) on the branches;
// then, per kernel configuration, ONE launch of the pass over a device work
// list of (beam, DM tile, time tile) descriptors covering all those beams, so
// the beams' tiles fill the GPU together with no per-beam tail wave; then their
// S/N kernels on the branches again.  Other beams (single-channel kernel,
// subband mode) run their whole search on a branch, each branch owning a
// region of the caller's workspace.  Beams are assigned largest first to the
// branch with the least work so far (work = DM trials x samples x channels).
// Capture happens once, at creation; a launch is one cudaGraphLaunch.  The
// graph holds raw pointers to the plans' device tables, so every launch first
// checks that no plan has been reconfigured since.
#include <algorithm>
#include <map>
#include <numeric>
#include <tuple>
#include <vector>

#include "sps_internal.h"

struct sps_batch {
  int device = 0;
  std::vector<const sps_plan*> plans;
  std::vector<uint64_t> gens;  // each plan's configuration generation at capture
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  sps::PresumPassArgs* d_passes = nullptr;  // batched passes' arguments (device)
  int4* d_work = nullptr;                   // their work list (device)
  int32_t list_launches = 0;                // batched pass launches per graph launch
};

namespace sps {
namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

double beam_work(const sps_plan* p) { return (double)p->dms.size() * p->n_t * p->channels; }

// Beams share a pass launch when they have the same kernel configuration and
// the same number of resident blocks per SM: the launch gives every block the
// largest stage of its beams, which must not cost the others occupancy.
using ConfigKey = std::tuple<int32_t, int32_t, int32_t, int32_t, int32_t, int32_t, int32_t>;

ConfigKey key_of(const sps_plan* p, int32_t smem_per_sm) {
  const sps_dedisp_config& c = p->cfg.brute;
  const size_t per_block = presum_smem_bytes(c, p->presum_data_bytes) + 1024;  // + the block's reserved share
  const int32_t resident = (int32_t)std::max<size_t>(1, (size_t)smem_per_sm / per_block);
  return ConfigKey{c.dms_per_thread, c.samples_per_thread, c.warps_dm, c.warps_time, c.chunk, c.presum, resident};
}

// The batch's layout: each beam's branch, whether its pass is batched, and
// its workspace region.  Branch k owns one region sized for its largest
// unbatched beam; every batched beam has a region of its own, since all their
// series must exist when the batched pass runs.
struct Layout {
  std::vector<int32_t> branch_of;
  std::vector<char> batched;
  std::vector<size_t> ws_offset, ws_bytes;  // per beam
  size_t total = 0;
};

sps_status plan_layout(const sps_plan* const* plans, int32_t n, int32_t branches, Layout* L) {
  if (!plans || n < 1) return fail(SPS_ERR_INVALID_ARG, "need at least one beam");
  if (branches < 1) return fail(SPS_ERR_INVALID_ARG, "branches must be >= 1");
  for (int32_t b = 0; b < n; b++)
    if (!plans[b]) return fail(SPS_ERR_INVALID_ARG, "null plan");
  const int32_t B = std::min(branches, n);
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return beam_work(plans[a]) > beam_work(plans[b]); });
  std::vector<double> load(B, 0.0);
  std::vector<size_t> branch_ws(B, 0);
  L->branch_of.assign(n, 0);
  L->batched.assign(n, 0);
  L->ws_offset.assign(n, 0);
  L->ws_bytes.assign(n, 0);
  for (int32_t b : order) {
    const int32_t k = (int32_t)(std::min_element(load.begin(), load.end()) - load.begin());
    L->branch_of[b] = k;
    load[k] += beam_work(plans[b]);
    L->batched[b] = batched_pass_form(plans[b]) ? 1 : 0;
    if (!L->batched[b]) branch_ws[k] = std::max(branch_ws[k], plan_workspace_bytes(plans[b]));
  }
  std::vector<size_t> branch_off(B, 0);
  size_t total = 0;
  for (int32_t k = 0; k < B; k++) {
    branch_off[k] = total;
    total += round_up(branch_ws[k]);
  }
  for (int32_t b = 0; b < n; b++) {
    if (L->batched[b]) {
      L->ws_offset[b] = total;
      L->ws_bytes[b] = plan_workspace_bytes(plans[b]);
      total += round_up(L->ws_bytes[b]);
    } else {
      L->ws_offset[b] = branch_off[L->branch_of[b]];
      L->ws_bytes[b] = branch_ws[L->branch_of[b]];
    }
  }
  L->total = total;
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
  Layout L;
  if (sps_status s = plan_layout(plans, n_beams, branches, &L)) return s;
  *bytes = L.total;
  return SPS_OK;
}

sps_status sps_batch_create(const sps_plan* const* plans, const sps_beam_buffers* buffers, int32_t n_beams,
                            int32_t branches, void* workspace, size_t workspace_bytes, sps_batch** out) {
  clear_error();
  if (!out || !buffers) return fail(SPS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  Layout L;
  if (sps_status s = plan_layout(plans, n_beams, branches, &L)) return s;
  const int device = plans[0]->device;
  for (int32_t b = 0; b < n_beams; b++)
    if (plans[b]->device != device) return fail(SPS_ERR_INVALID_ARG, "all plans must be on one device");
  if (!workspace || workspace_bytes < L.total || ((uintptr_t)workspace % kAlign))
    return fail(SPS_ERR_INVALID_ARG, "workspace missing, smaller than sps_batch_workspace_bytes or not 256-byte aligned");

  // batched passes grouped by kernel configuration and occupancy, beams in order
  int32_t smem_per_sm = 0;
  SPS_CUDA(cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
  std::map<ConfigKey, std::vector<int32_t>> groups;
  for (int32_t b = 0; b < n_beams; b++)
    if (L.batched[b]) groups[key_of(plans[b], smem_per_sm)].push_back(b);
  std::vector<int32_t> pass_of(n_beams, -1);  // index into the passes array
  int32_t n_passes = 0;
  for (auto& g : groups)
    for (int32_t b : g.second) pass_of[b] = n_passes++;

  int cur = 0;
  SPS_CUDA(cudaGetDevice(&cur));
  if (cur != device) SPS_CUDA(cudaSetDevice(device));
  const int32_t B = std::min(branches, n_beams);
  std::vector<cudaStream_t> streams(B, nullptr);
  std::vector<cudaEvent_t> joins(B, nullptr);
  std::vector<cudaEvent_t> pre_done(n_beams, nullptr);
  std::vector<cudaEvent_t> group_done(groups.size(), nullptr);
  cudaStream_t cap = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  sps_batch* batch = new sps_batch();
  batch->device = device;
  std::vector<PresumPassArgs> passes(n_passes);
  std::vector<int4> work;
  sps_status st = SPS_OK;
  auto cuda_ok = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == SPS_OK) st = cuda_fail(e, what);
    return st == SPS_OK;
  };
  if (n_passes) {
    int64_t n_work = 0;
    for (int32_t b = 0; b < n_beams; b++) {
      if (!L.batched[b]) continue;
      const sps_dedisp_config& c = plans[b]->cfg.brute;
      PresumPassArgs shape{};
      shape.n_dm = (int32_t)plans[b]->dms.size();
      shape.n_out = plans[b]->n_t;
      shape.n_groups = 1;
      n_work += presum_pass_blocks(shape, c);
    }
    if (cuda_ok(cudaMalloc(&batch->d_passes, sizeof(PresumPassArgs) * n_passes), "cudaMalloc"))
      cuda_ok(cudaMalloc(&batch->d_work, sizeof(int4) * n_work), "cudaMalloc");
  }
  if (st == SPS_OK && cuda_ok(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreateWithFlags") &&
      cuda_ok(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "cudaEventCreateWithFlags")) {
    for (int32_t k = 0; k < B && st == SPS_OK; k++) {
      cuda_ok(cudaStreamCreateWithFlags(&streams[k], cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
      if (st == SPS_OK) cuda_ok(cudaEventCreateWithFlags(&joins[k], cudaEventDisableTiming), "cudaEventCreateWithFlags");
    }
    for (int32_t b = 0; b < n_beams && st == SPS_OK; b++)
      if (L.batched[b]) cuda_ok(cudaEventCreateWithFlags(&pre_done[b], cudaEventDisableTiming), "cudaEventCreateWithFlags");
    for (size_t g = 0; g < group_done.size() && st == SPS_OK; g++)
      cuda_ok(cudaEventCreateWithFlags(&group_done[g], cudaEventDisableTiming), "cudaEventCreateWithFlags");
  }
  if (st == SPS_OK && cuda_ok(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture")) {
    cuda_ok(cudaEventRecord(fork, cap), "cudaEventRecord");
    for (int32_t k = 0; k < B && st == SPS_OK; k++) cuda_ok(cudaStreamWaitEvent(streams[k], fork, 0), "cudaStreamWaitEvent");
    // phase 1: whole searches of unbatched beams, pre-passes of batched ones
    for (int32_t b = 0; b < n_beams && st == SPS_OK; b++) {
      const sps_beam_buffers& u = buffers[b];
      cudaStream_t sk = streams[L.branch_of[b]];
      uint8_t* w = static_cast<uint8_t*>(workspace) + L.ws_offset[b];
      if (!L.batched[b]) {
        st = run_search(plans[b], u.x, u.x_pitch, u.D, w, L.ws_bytes[b], u.snr, u.peak_t, u.peak_val, u.best, sk);
      } else {
        st = brute_prepass(plans[b], u.x, u.x_pitch, u.D, w, L.ws_bytes[b], sk, &passes[pass_of[b]]);
        if (st == SPS_OK) cuda_ok(cudaEventRecord(pre_done[b], sk), "cudaEventRecord");
      }
    }
    // phase 2: one batched pass per group, after its beams' pre-passes; groups
    // go to different branches so that one group's tail overlaps the next
    size_t gi = 0;
    for (auto it = groups.begin(); it != groups.end() && st == SPS_OK; ++it, ++gi) {
      const std::vector<int32_t>& beams = it->second;
      cudaStream_t sg = streams[gi % B];
      const int32_t first = pass_of[beams[0]];
      const size_t w0 = work.size();
      int32_t max_data = 0;
      for (int32_t b : beams) {
        cuda_ok(cudaStreamWaitEvent(sg, pre_done[b], 0), "cudaStreamWaitEvent");
        presum_pass_work(passes[pass_of[b]], plans[b]->cfg.brute, pass_of[b] - first, &work);
        max_data = std::max(max_data, passes[pass_of[b]].data_bytes);
      }
      if (st == SPS_OK)
        st = launch_presum_pass_list(batch->d_passes + first, batch->d_work + w0, (int64_t)(work.size() - w0),
                                     plans[beams[0]]->cfg.brute, max_data, sg);
      batch->list_launches++;
      if (st == SPS_OK) cuda_ok(cudaEventRecord(group_done[gi], sg), "cudaEventRecord");
    }
    // phase 3: S/N of batched beams on their branches
    gi = 0;
    for (auto it = groups.begin(); it != groups.end() && st == SPS_OK; ++it, ++gi) {
      for (int32_t b : it->second) {
        const sps_beam_buffers& u = buffers[b];
        cudaStream_t sk = streams[L.branch_of[b]];
        if (!cuda_ok(cudaStreamWaitEvent(sk, group_done[gi], 0), "cudaStreamWaitEvent")) break;
        st = snr_into(plans[b], u.D, u.snr, u.peak_t, u.peak_val, u.best, sk);
        if (st) break;
      }
    }
    // join every branch, also after a failure, so that the capture ends cleanly
    for (int32_t k = 0; k < B; k++) {
      cuda_ok(cudaEventRecord(joins[k], streams[k]), "cudaEventRecord");
      cuda_ok(cudaStreamWaitEvent(cap, joins[k], 0), "cudaStreamWaitEvent");
    }
    cuda_ok(cudaStreamEndCapture(cap, &graph), "cudaStreamEndCapture");
  }
  // the batched passes' arguments and work list, before the first launch
  if (st == SPS_OK && n_passes) {
    int64_t n_work = 0;
    for (int32_t b = 0; b < n_beams; b++)
      if (L.batched[b]) n_work += presum_pass_blocks(passes[pass_of[b]], plans[b]->cfg.brute);
    if ((int64_t)work.size() != n_work) st = fail(SPS_ERR_INVALID_ARG, "batched work list size changed");
  }
  if (st == SPS_OK && n_passes) {
    if (cuda_ok(cudaMemcpy(batch->d_passes, passes.data(), sizeof(PresumPassArgs) * passes.size(),
                           cudaMemcpyHostToDevice), "cudaMemcpy"))
      cuda_ok(cudaMemcpy(batch->d_work, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice), "cudaMemcpy");
  }
  if (st == SPS_OK) {
    batch->graph = graph;
    graph = nullptr;
    if (cuda_ok(cudaGraphInstantiate(&batch->exec, batch->graph, 0), "cudaGraphInstantiate")) {
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
  for (cudaEvent_t e : pre_done)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : group_done)
    if (e) cudaEventDestroy(e);
  if (fork) cudaEventDestroy(fork);
  if (cap) cudaStreamDestroy(cap);
  if (cur != device) cudaSetDevice(cur);
  if (st != SPS_OK) {
    sps_batch_destroy(batch);
    return st;
  }
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
  cudaFree(batch->d_passes);
  cudaFree(batch->d_work);
  delete batch;
  return SPS_OK;
}

sps_status sps_batch_list_launches(const sps_batch* batch, int32_t* n) {
  if (!batch || !n) return fail(SPS_ERR_INVALID_ARG, "null argument");
  *n = batch->list_launches;
  return SPS_OK;
}

}  // extern "C"
