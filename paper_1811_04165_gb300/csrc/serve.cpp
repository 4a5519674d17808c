// Real-time serving of streaming beams (Sec. 1: every beam's 1.024 s batch must
// be searched within 1.024 s).  The server owns one device arena of the HBM
// budget.  Each beam keeps only its overlap tail there between batches; a
// batch gets its input buffer, D, S/N tables and workspace from the arena
// when it is dispatched and gives them back when it completes, so queued
// batches are admitted as slots and memory free up (continuous batching).
// Completion times are read on the GPU timeline and mapped to the host clock.
#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <vector>

#include "sps_internal.h"

namespace {

constexpr size_t kAlign = 256;

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over [0, size) with coalescing frees; offsets and sizes
// are multiples of kAlign.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    size_ = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round_up(std::max<size_t>(bytes, 1));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round_up(std::max<size_t>(bytes, 1));
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + bytes == next->first) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t used() const { return used_; }
  size_t size() const { return size_; }

 private:
  std::map<size_t, size_t> free_;  // offset -> bytes
  size_t size_ = 0, used_ = 0;
};

struct Beam {
  const sps_plan* plan = nullptr;
  int64_t pitch = 0;        // device input row pitch (>= N_in, multiple of 16)
  int64_t tail = 0;         // N_in - N_t samples carried into the next batch
  int64_t tail_pitch = 0;   // bytes per row of the resident tail
  size_t tail_off = 0;      // arena offset of the tail [channels][tail_pitch]
  size_t tail_bytes = 0;
  size_t batch_bytes = 0;   // arena bytes one batch of this beam takes while in flight
  int64_t batches = 0;      // batches dispatched so far
  int32_t queued = 0;       // batches waiting in the queue
  bool busy = false;        // a batch is in flight
  bool removed = false;     // no further submissions; the tail goes once idle
  bool tail_held = false;
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
  size_t off = 0, bytes = 0;  // the batch's arena block
};

struct Report {
  uint64_t tag;
  double done_s;
  sps_status status;
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct sps_server {
  int device = 0;
  uint8_t* base = nullptr;  // the arena's device memory (hbm_budget_bytes)
  Arena arena;
  std::vector<Beam> beams;
  std::vector<Slot> slots;
  std::deque<Job> queue;
  std::deque<Report> reports;  // completed or failed batches not yet returned by poll
  int64_t admitted = 0, waits_for_memory = 0, failed = 0;
  cudaEvent_t ref = nullptr;   // GPU-timeline origin
  double ref_host = 0.0;       // host clock at `ref`
};

namespace sps {
namespace {

// Arena bytes of one batch: input (with its tail), D, the S/N tables, best and
// the plan's workspace, each 256-byte aligned.
struct BatchLayout {
  size_t x, d, snr, pt, pv, best, ws, total;
};

BatchLayout batch_layout(const sps_plan* p, int64_t pitch) {
  BatchLayout l{};
  const size_t n_snr = p->widths.size() * p->dms.size();
  l.x = 0;
  l.d = l.x + round_up((size_t)pitch * p->channels);
  l.snr = l.d + round_up(p->dms.size() * (size_t)p->n_t * sizeof(int32_t));
  l.pt = l.snr + round_up(n_snr * sizeof(double));
  l.pv = l.pt + round_up(n_snr * sizeof(int32_t));
  l.best = l.pv + round_up(n_snr * sizeof(int32_t));
  l.ws = l.best + kAlign;
  l.total = l.ws + round_up(plan_workspace_bytes(p));
  return l;
}

void release_tail_if_done(sps_server* s, Beam& b) {
  if (b.removed && b.tail_held && !b.busy && b.queued == 0) {
    s->arena.release(b.tail_off, b.tail_bytes);
    b.tail_held = false;
  }
}

// Enqueues one batch on a free slot whose arena block has been allocated.
sps_status dispatch_one(sps_server* s, Slot& sl, const Job& j) {
  Beam& b = s->beams[j.beam];
  const sps_plan* p = b.plan;
  const BatchLayout l = batch_layout(p, b.pitch);
  if (l.total > sl.bytes)
    return fail(SPS_ERR_INVALID_ARG, "the beam's plan needs more memory than when the beam was added "
                                     "(its configuration changed)");
  uint8_t* blk = s->base + sl.off;
  uint8_t* x = blk + l.x;
  int32_t* D = reinterpret_cast<int32_t*>(blk + l.d);
  double* snr = reinterpret_cast<double*>(blk + l.snr);
  int32_t* best = reinterpret_cast<int32_t*>(blk + l.best);
  uint8_t* tail = s->base + b.tail_off;
  const size_t C = (size_t)p->channels;
  cudaStream_t st = sl.stream;
  // the beam's resident tail (zeros before its first batch) leads the N_t new samples
  if (b.tail > 0) {
    if (b.batches == 0)
      SPS_CUDA(cudaMemset2DAsync(x, b.pitch, 0, (size_t)b.tail, C, st));
    else
      SPS_CUDA(cudaMemcpy2DAsync(x, b.pitch, tail, b.tail_pitch, (size_t)b.tail, C, cudaMemcpyDeviceToDevice, st));
  }
  SPS_CUDA(cudaMemcpy2DAsync(x + b.tail, b.pitch, j.host_x, j.host_pitch, (size_t)p->n_t, C,
                             cudaMemcpyHostToDevice, st));
  // the last N_in - N_t samples of this window lead the next batch
  if (b.tail > 0)
    SPS_CUDA(cudaMemcpy2DAsync(tail, b.tail_pitch, x + p->n_t, b.pitch, (size_t)b.tail, C, cudaMemcpyDeviceToDevice,
                               st));
  // the stream has advanced by this batch whatever happens to its search
  b.batches++;
  if (sps_status r = run_search(p, x, b.pitch, D, blk + l.ws, l.total - l.ws, snr,
                                reinterpret_cast<int32_t*>(blk + l.pt), reinterpret_cast<int32_t*>(blk + l.pv), best,
                                st))
    return r;
  const size_t n_snr = p->widths.size() * p->dms.size();
  if (j.snr_host) SPS_CUDA(cudaMemcpyAsync(j.snr_host, snr, n_snr * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (j.best_host) SPS_CUDA(cudaMemcpyAsync(j.best_host, best, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SPS_CUDA(cudaEventRecord(sl.done, st));
  return SPS_OK;
}

// Starts queued batches in arrival order, each beam's in order, while slots
// are free: a batch whose beam is busy waits; so does a batch whose arena
// block does not fit now (later batches of other beams that fit may pass it).
// A batch that fails to start is reported through poll with its status.
void dispatch(sps_server* s) {
  std::vector<char> blocked(s->beams.size(), 0);
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    auto free_slot = std::find_if(s->slots.begin(), s->slots.end(), [](const Slot& sl) { return !sl.busy; });
    if (free_slot == s->slots.end()) break;
    Beam& b = s->beams[it->beam];
    if (blocked[it->beam] || b.busy) {
      blocked[it->beam] = 1;
      ++it;
      continue;
    }
    size_t off = 0;
    if (!s->arena.alloc(b.batch_bytes, &off)) {
      s->waits_for_memory++;
      blocked[it->beam] = 1;
      ++it;
      continue;
    }
    const Job j = *it;
    it = s->queue.erase(it);
    b.queued--;
    Slot& sl = *free_slot;
    sl.off = off;
    sl.bytes = b.batch_bytes;
    const sps_status r = dispatch_one(s, sl, j);
    if (r != SPS_OK) {
      // what was enqueued before the failure must finish before the block is reused
      cudaStreamSynchronize(sl.stream);
      cudaGetLastError();
      s->arena.release(off, b.batch_bytes);
      s->reports.push_back(Report{j.tag, now_s(), r});
      s->failed++;
      release_tail_if_done(s, b);
      continue;
    }
    b.busy = true;
    sl.busy = true;
    sl.beam = j.beam;
    sl.tag = j.tag;
    s->admitted++;
  }
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
  if (desc->hbm_budget_bytes < kAlign) return fail(SPS_ERR_INVALID_ARG, "hbm_budget_bytes below 256");
  sps_server* s = new sps_server();
  cudaGetDevice(&s->device);
  const size_t budget = desc->hbm_budget_bytes / kAlign * kAlign;
  if (cudaMalloc(&s->base, budget) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return fail(SPS_ERR_OOM, "the server's arena (hbm_budget_bytes)");
  }
  s->arena.reset(budget);
  s->slots.resize(desc->max_inflight);
  sps_status st = SPS_OK;
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sl.done) != cudaSuccess) {
      st = fail(SPS_ERR_CUDA, "stream or event creation");
      break;
    }
  }
  if (st == SPS_OK && (cudaEventCreate(&s->ref) != cudaSuccess ||
                       cudaEventRecord(s->ref, s->slots[0].stream) != cudaSuccess ||
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
  b.tail_pitch = (b.tail + 15) / 16 * 16;
  b.tail_bytes = round_up((size_t)b.tail_pitch * p->channels);
  b.batch_bytes = batch_layout(p, b.pitch).total;
  // resident tails of every beam plus one batch of this one must fit the arena,
  // or this beam's batches could never run
  size_t resident = 0;
  for (const Beam& o : s->beams) resident += o.tail_held ? o.tail_bytes : 0;
  if (resident + b.tail_bytes + b.batch_bytes > s->arena.size())
    return fail(SPS_ERR_UNSUPPORTED, "beam does not fit the server's HBM budget (its overlap tail and one batch: " +
                                         std::to_string(b.tail_bytes + b.batch_bytes) + " bytes)");
  if (!s->arena.alloc(b.tail_bytes, &b.tail_off))
    return fail(SPS_ERR_UNSUPPORTED, "beam does not fit the server's HBM budget (no room for its overlap tail now)");
  b.tail_held = true;
  s->beams.push_back(b);
  *beam_id = (int32_t)s->beams.size() - 1;
  return SPS_OK;
}

sps_status sps_server_remove_beam(sps_server* s, int32_t beam) {
  clear_error();
  if (!s) return fail(SPS_ERR_INVALID_ARG, "null argument");
  if (beam < 0 || beam >= (int32_t)s->beams.size() || s->beams[beam].removed)
    return fail(SPS_ERR_INVALID_ARG, "unknown or removed beam");
  Beam& b = s->beams[beam];
  b.removed = true;
  release_tail_if_done(s, b);
  return SPS_OK;
}

sps_status sps_server_submit(sps_server* s, int32_t beam, const uint8_t* host_x, int64_t host_pitch,
                             double* snr_host, int32_t* best_host, uint64_t tag) {
  clear_error();
  NvtxRange nvtx("sps_server_submit");
  if (!s || !host_x) return fail(SPS_ERR_INVALID_ARG, "null argument");
  if (beam < 0 || beam >= (int32_t)s->beams.size()) return fail(SPS_ERR_INVALID_ARG, "unknown beam");
  Beam& b = s->beams[beam];
  if (b.removed) return fail(SPS_ERR_INVALID_ARG, "beam removed");
  if (host_pitch < b.plan->n_t) return fail(SPS_ERR_INVALID_ARG, "host_pitch smaller than N_t");
  // every check is done: from here the batch is queued and its outcome is
  // reported by sps_server_poll, whatever happens when it is dispatched
  s->queue.push_back(Job{beam, host_x, host_pitch, snr_host, best_host, tag});
  b.queued++;
  dispatch(s);
  return SPS_OK;
}

sps_status sps_server_poll(sps_server* s, uint64_t* tags, double* done_s, sps_status* status, int32_t max,
                           int32_t* n) {
  clear_error();
  if (!s || !n || (max > 0 && (!tags || !done_s))) return fail(SPS_ERR_INVALID_ARG, "null argument");
  *n = 0;
  for (Slot& sl : s->slots) {
    if (!sl.busy) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    Report r{sl.tag, now_s(), SPS_OK};
    if (q == cudaSuccess) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, s->ref, sl.done) == cudaSuccess) r.done_s = s->ref_host + 1e-3 * ms;
    } else {
      cudaGetLastError();
      r.status = SPS_ERR_CUDA;
      s->failed++;
    }
    s->reports.push_back(r);
    s->arena.release(sl.off, sl.bytes);
    sl.busy = false;
    Beam& b = s->beams[sl.beam];
    b.busy = false;
    release_tail_if_done(s, b);
  }
  dispatch(s);
  while (*n < max && !s->reports.empty()) {
    const Report& r = s->reports.front();
    tags[*n] = r.tag;
    done_s[*n] = r.done_s;
    if (status) status[*n] = r.status;
    (*n)++;
    s->reports.pop_front();
  }
  return SPS_OK;
}

sps_status sps_server_pending(const sps_server* s, int32_t* n) {
  if (!s || !n) return fail(SPS_ERR_INVALID_ARG, "null argument");
  int32_t k = (int32_t)s->queue.size() + (int32_t)s->reports.size();
  for (const Slot& sl : s->slots) k += sl.busy ? 1 : 0;
  *n = k;
  return SPS_OK;
}

sps_status sps_server_get_stats(const sps_server* s, sps_server_stats* out) {
  if (!s || !out) return fail(SPS_ERR_INVALID_ARG, "null argument");
  sps_server_stats st{};
  st.budget_bytes = s->arena.size();
  st.used_bytes = s->arena.used();
  for (const Beam& b : s->beams) st.resident_bytes += b.tail_held ? b.tail_bytes : 0;
  for (const Slot& sl : s->slots) {
    st.inflight += sl.busy ? 1 : 0;
    st.batch_bytes += sl.busy ? sl.bytes : 0;
  }
  st.queued = (int32_t)s->queue.size();
  st.admitted = s->admitted;
  st.waits_for_memory = s->waits_for_memory;
  st.failed = s->failed;
  *out = st;
  return SPS_OK;
}

sps_status sps_server_destroy(sps_server* s) {
  if (!s) return SPS_OK;
  for (Slot& sl : s->slots)
    if (sl.stream) cudaStreamSynchronize(sl.stream);
  cudaFree(s->base);
  for (Slot& sl : s->slots) {
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  if (s->ref) cudaEventDestroy(s->ref);
  delete s;
  return SPS_OK;
}

}  // extern "C"
