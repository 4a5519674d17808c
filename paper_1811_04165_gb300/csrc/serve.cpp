// Real-time serving of streaming beams: admission against an HBM budget,
// device-resident overlap tails, in-order per-beam dispatch onto concurrent
// stream slots, completion times on the GPU timeline mapped to the host clock.
#include <algorithm>
#include <chrono>
#include <deque>
#include <vector>

#include "sps_internal.h"

namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Beam {
  const sps_plan* plan = nullptr;
  int64_t pitch = 0;          // device input row pitch (>= N_in, multiple of 16)
  int64_t tail = 0;           // N_in - N_t samples carried into the next batch
  uint8_t* x[2] = {nullptr, nullptr};
  int32_t* D = nullptr;
  double* snr = nullptr;
  int32_t* peak_t = nullptr;
  int32_t* peak_val = nullptr;
  int32_t* best = nullptr;
  int64_t batches = 0;        // batches dispatched so far (selects the input buffer)
  bool busy = false;
  size_t footprint = 0;
};

struct Job {
  int32_t beam;
  const uint8_t* host_x;
  int64_t host_pitch;
  double* snr_host;
  int32_t* best_host;
  uint64_t tag;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  int32_t beam = -1;
  uint64_t tag = 0;
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct sps_server {
  int device = 0;
  size_t budget = 0;
  size_t used = 0;
  std::vector<Beam> beams;
  std::vector<Slot> slots;
  std::deque<Job> queue;
  uint8_t* ws = nullptr;      // slots x ws_slot bytes
  size_t ws_slot = 0;
  cudaEvent_t ref = nullptr;  // GPU-timeline origin
  double ref_host = 0.0;      // host clock at `ref`
};

namespace sps {
namespace {

sps_status grow_workspace(sps_server* s, size_t need) {
  if (need <= s->ws_slot) return SPS_OK;
  // every slot must be idle while the pool is replaced
  for (const Slot& sl : s->slots)
    if (sl.busy) SPS_CUDA(cudaStreamSynchronize(sl.stream));
  uint8_t* fresh = nullptr;
  if (cudaMalloc(&fresh, need * s->slots.size()) != cudaSuccess) {
    cudaGetLastError();
    return fail(SPS_ERR_OOM, "workspace slots");
  }
  cudaFree(s->ws);
  s->ws = fresh;
  s->ws_slot = need;
  return SPS_OK;
}

sps_status dispatch_one(sps_server* s, Slot& sl, const Job& j) {
  Beam& b = s->beams[j.beam];
  const sps_plan* p = b.plan;
  const int cur = (int)(b.batches & 1);
  uint8_t* x = b.x[cur];
  const uint8_t* prev = b.x[cur ^ 1];
  const size_t C = (size_t)p->channels;
  cudaStream_t st = sl.stream;
  // the previous batch's last N_in - N_t samples lead this batch (zeros before the first)
  if (b.tail > 0) {
    if (b.batches == 0)
      SPS_CUDA(cudaMemset2DAsync(x, b.pitch, 0, (size_t)b.tail, C, st));
    else
      SPS_CUDA(cudaMemcpy2DAsync(x, b.pitch, prev + p->n_t, b.pitch, (size_t)b.tail, C, cudaMemcpyDeviceToDevice,
                                 st));
  }
  SPS_CUDA(cudaMemcpy2DAsync(x + b.tail, b.pitch, j.host_x, j.host_pitch, (size_t)p->n_t, C,
                             cudaMemcpyHostToDevice, st));
  const size_t slot_index = (size_t)(&sl - s->slots.data());
  if (sps_status r = run_search(p, x, b.pitch, b.D, s->ws + slot_index * s->ws_slot, s->ws_slot, b.snr, b.peak_t,
                                b.peak_val, b.best, st))
    return r;
  const size_t n_snr = p->widths.size() * p->dms.size();
  if (j.snr_host)
    SPS_CUDA(cudaMemcpyAsync(j.snr_host, b.snr, n_snr * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (j.best_host) SPS_CUDA(cudaMemcpyAsync(j.best_host, b.best, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SPS_CUDA(cudaEventRecord(sl.done, st));
  b.batches++;
  b.busy = true;
  sl.busy = true;
  sl.beam = j.beam;
  sl.tag = j.tag;
  return SPS_OK;
}

// Starts queued batches, in arrival order, whose beam is idle, while slots are free.
sps_status dispatch(sps_server* s) {
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    auto free_slot = std::find_if(s->slots.begin(), s->slots.end(), [](const Slot& sl) { return !sl.busy; });
    if (free_slot == s->slots.end()) break;
    if (s->beams[it->beam].busy) {
      ++it;
      continue;
    }
    const Job j = *it;
    it = s->queue.erase(it);
    if (sps_status r = dispatch_one(s, *free_slot, j)) return r;
  }
  return SPS_OK;
}

}  // namespace
}  // namespace sps

using namespace sps;

extern "C" {

double sps_server_clock(void) { return now_s(); }

sps_status sps_server_create(const sps_server_desc* desc, sps_server** out) {
  clear_error();
  if (!desc || !out) return fail(SPS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (desc->max_inflight < 1) return fail(SPS_ERR_INVALID_ARG, "max_inflight must be >= 1");
  sps_server* s = new sps_server();
  cudaGetDevice(&s->device);
  s->budget = desc->hbm_budget_bytes;
  s->slots.resize(desc->max_inflight);
  sps_status st = SPS_OK;
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sl.done) != cudaSuccess) {
      st = fail(SPS_ERR_CUDA, "stream or event creation");
      break;
    }
  }
  if (st == SPS_OK && (cudaEventCreate(&s->ref) != cudaSuccess || cudaEventRecord(s->ref, s->slots[0].stream) != cudaSuccess ||
                       cudaEventSynchronize(s->ref) != cudaSuccess))
    st = fail(SPS_ERR_CUDA, "reference event");
  s->ref_host = now_s();
  if (st != SPS_OK) {
    sps_server_destroy(s);
    return st;
  }
  *out = s;
  return SPS_OK;
}

sps_status sps_server_add_beam(sps_server* s, const sps_plan* p, int32_t* beam_id) {
  clear_error();
  if (!s || !p || !beam_id) return fail(SPS_ERR_INVALID_ARG, "null argument");
  if (p->device != s->device) return fail(SPS_ERR_INVALID_ARG, "plan on another device");
  Beam b;
  b.plan = p;
  b.pitch = (p->n_in + 15) / 16 * 16;
  b.tail = p->n_in - p->n_t;
  const size_t C = (size_t)p->channels, n_snr = p->widths.size() * p->dms.size();
  const size_t x_bytes = round_up((size_t)b.pitch * C);
  const size_t d_bytes = round_up(p->dms.size() * (size_t)p->n_t * sizeof(int32_t));
  const size_t t_bytes = round_up(n_snr * sizeof(double)) + 2 * round_up(n_snr * sizeof(int32_t)) + kAlign;
  const size_t ws_need = round_up(plan_workspace_bytes(p));
  const size_t ws_extra = ws_need > s->ws_slot ? (ws_need - s->ws_slot) * s->slots.size() : 0;
  b.footprint = 2 * x_bytes + d_bytes + t_bytes;
  if (s->used + b.footprint + ws_extra > s->budget)
    return fail(SPS_ERR_UNSUPPORTED, "beam does not fit the server's HBM budget");
  if (sps_status r = grow_workspace(s, ws_need)) return r;
  s->used += ws_extra;
  uint8_t* mem = nullptr;
  if (cudaMalloc(&mem, b.footprint) != cudaSuccess) {
    cudaGetLastError();
    return fail(SPS_ERR_OOM, "beam buffers");
  }
  b.x[0] = mem;
  b.x[1] = mem + x_bytes;
  b.D = reinterpret_cast<int32_t*>(mem + 2 * x_bytes);
  uint8_t* t = mem + 2 * x_bytes + d_bytes;
  b.snr = reinterpret_cast<double*>(t);
  b.peak_t = reinterpret_cast<int32_t*>(t + round_up(n_snr * sizeof(double)));
  b.peak_val = reinterpret_cast<int32_t*>(t + round_up(n_snr * sizeof(double)) + round_up(n_snr * sizeof(int32_t)));
  b.best = reinterpret_cast<int32_t*>(t + round_up(n_snr * sizeof(double)) + 2 * round_up(n_snr * sizeof(int32_t)));
  s->used += b.footprint;
  s->beams.push_back(b);
  *beam_id = (int32_t)s->beams.size() - 1;
  return SPS_OK;
}

sps_status sps_server_submit(sps_server* s, int32_t beam, const uint8_t* host_x, int64_t host_pitch,
                             double* snr_host, int32_t* best_host, uint64_t tag) {
  clear_error();
  NvtxRange nvtx("sps_server_submit");
  if (!s || !host_x) return fail(SPS_ERR_INVALID_ARG, "null argument");
  if (beam < 0 || beam >= (int32_t)s->beams.size()) return fail(SPS_ERR_INVALID_ARG, "unknown beam");
  if (host_pitch < s->beams[beam].plan->n_t) return fail(SPS_ERR_INVALID_ARG, "host_pitch smaller than N_t");
  s->queue.push_back(Job{beam, host_x, host_pitch, snr_host, best_host, tag});
  return dispatch(s);
}

sps_status sps_server_poll(sps_server* s, uint64_t* tags, double* done_s, int32_t max, int32_t* n) {
  clear_error();
  if (!s || !n || (max > 0 && (!tags || !done_s))) return fail(SPS_ERR_INVALID_ARG, "null argument");
  *n = 0;
  for (Slot& sl : s->slots) {
    if (!sl.busy || *n >= max) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return cuda_fail(q, "cudaEventQuery");
    float ms = 0.f;
    SPS_CUDA(cudaEventElapsedTime(&ms, s->ref, sl.done));
    tags[*n] = sl.tag;
    done_s[*n] = s->ref_host + 1e-3 * ms;
    (*n)++;
    sl.busy = false;
    s->beams[sl.beam].busy = false;
  }
  return dispatch(s);
}

sps_status sps_server_pending(const sps_server* s, int32_t* n) {
  if (!s || !n) return fail(SPS_ERR_INVALID_ARG, "null argument");
  int32_t k = (int32_t)s->queue.size();
  for (const Slot& sl : s->slots) k += sl.busy ? 1 : 0;
  *n = k;
  return SPS_OK;
}

sps_status sps_server_destroy(sps_server* s) {
  if (!s) return SPS_OK;
  for (Slot& sl : s->slots)
    if (sl.stream) cudaStreamSynchronize(sl.stream);
  for (Beam& b : s->beams) cudaFree(b.x[0]);
  cudaFree(s->ws);
  for (Slot& sl : s->slots) {
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  if (s->ref) cudaEventDestroy(s->ref);
  delete s;
  return SPS_OK;
}

}  // extern "C"
