// extern "C" entry points of libsps.so: argument checks, then kernel launches.
#include <algorithm>
#include <cstring>
#include <string>

#include "sps_internal.h"

namespace sps {

namespace {
thread_local std::string g_last_error;
}

sps_status fail(sps_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

sps_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return SPS_ERR_CUDA;
}

void clear_error() { g_last_error.clear(); }

sps_status plan_create(const sps_plan_desc* d, sps_plan** out);

namespace {

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

sps_status check_plan(const sps_plan* p) {
  if (!p) return fail(SPS_ERR_INVALID_ARG, "null plan");
  return SPS_OK;
}

sps_status check_x(const sps_plan* p, const uint8_t* x, int64_t pitch) {
  if (!x) return fail(SPS_ERR_INVALID_ARG, "null input");
  if (!aligned16(x)) return fail(SPS_ERR_INVALID_ARG, "input must be 16-byte aligned");
  if (pitch < p->n_in || pitch % 16) return fail(SPS_ERR_INVALID_ARG, "x_pitch must be >= N_in and a multiple of 16");
  return SPS_OK;
}

// Workspace layout: the staged form of the batch -- three shifted copies of x
// (single-channel kernel) or the pre-summed series (pairs or quads) -- then, in
// SUBBAND mode, the step-one output Y.  workspace_needed is what the current
// configuration uses; sps_plan_workspace_bytes reports the largest of the
// forms so that a buffer of that size fits any configuration.
size_t x4_bytes(const sps_plan* p) { return (size_t)3 * p->channels * p->pitch4; }

size_t q_bytes(const sps_plan* p, int64_t n_series) { return (size_t)n_series * 2 * p->q_pitch * sizeof(uint16_t); }

size_t y_bytes(const sps_plan* p) {
  return p->mode == SPS_MODE_SUBBAND ? (size_t)p->coarse_dms.size() * p->n_subbands * p->y_pitch * sizeof(uint16_t)
                                     : 0;
}

bool uses_presum(const sps_plan* p) { return p->mode == SPS_MODE_BRUTE ? p->cfg.brute.presum : p->cfg.step1.presum; }

size_t y_offset(const sps_plan* p) {
  return ((uses_presum(p) ? q_bytes(p, p->n_presum_series) : x4_bytes(p)) + 255) / 256 * 256;
}

// With zapped channels the workspace starts with the masked copy of x.
size_t zap_bytes(const sps_plan* p) {
  return p->zap.empty() ? 0 : ((size_t)p->channels * p->pitch4 + 255) / 256 * 256;
}

size_t workspace_needed(const sps_plan* p) { return zap_bytes(p) + y_offset(p) + y_bytes(p); }

size_t workspace_any_config(const sps_plan* p) {
  return zap_bytes(p) + (std::max(x4_bytes(p), q_bytes(p, p->max_presum_series)) + 255) / 256 * 256 + y_bytes(p);
}

// Points the search at the masked copy of x when channels are zapped; moves
// the workspace past it.
sps_status prepare_input(const sps_plan* p, const uint8_t** x, int64_t* pitch, uint8_t** ws, cudaStream_t st) {
  if (p->zap.empty()) return SPS_OK;
  if (sps_status s = launch_zap_copy(*x, *pitch, (int32_t)p->n_in, p->d_zap, p->channels, *ws, p->pitch4, st))
    return s;
  *x = *ws;
  *pitch = p->pitch4;
  *ws += zap_bytes(p);
  return SPS_OK;
}

U8PassArgs u8_args(const sps_plan* p, const uint8_t* x, int64_t pitch, const uint8_t* x4) {
  U8PassArgs a{};
  a.x = x;
  a.pitch = pitch;
  a.x4 = x4;
  a.pitch4 = p->pitch4;
  a.win_limit = (int32_t)p->pitch4;
  a.b0 = p->d_b0;
  a.offs = p->d_offs;
  a.channels = p->channels;
  a.status = p->d_status;
  a.one = 1u;
  return a;
}

// The pre-summed series of one uint8 pass (the pre-pass), and the arguments of
// the pass that reads them.
sps_status presum_prepass(const sps_plan* p, const sps_dedisp_config& cfg, const uint8_t* x, int64_t pitch,
                          uint8_t* ws, int32_t rows, int32_t per, int32_t n_out, int64_t out_pitch, int32_t dmax,
                          void* out, int32_t out_u16, cudaStream_t st, PresumPassArgs* args) {
  uint16_t* q = reinterpret_cast<uint16_t*>(ws);
  const int32_t K = 1 << cfg.presum;
  sps_status s = launch_presum_series(x, pitch, (int32_t)p->n_in, p->d_presum_units, p->n_presum_units, K,
                                      p->presum_max_rel, p->d_presum_series, p->n_presum_series, q, p->q_pitch, st);
  if (s) return s;
  PresumPassArgs& a = *args;
  a = PresumPassArgs{};
  a.q = q;
  a.q_pitch = p->q_pitch;
  a.copies = p->d_presum_copies;
  a.copies_max = p->presum_copies_max;
  a.data_bytes = p->presum_data_bytes;
  a.offs = p->d_presum_offs;
  a.di_pad = presum_di_pad(cfg);
  a.n_dm = rows;
  a.n_groups = p->channels / per;
  a.group_units = (per + K - 1) / K;
  a.fold_units = 65535 / (255 * K);
  a.max_start = (int32_t)(p->n_in - p->n_t);
  a.n_out = n_out;
  a.out_pitch = out_pitch;
  a.dmax_tile = dmax;
  a.out = out;
  a.out_u16 = out_u16;
  a.status = p->d_status;
  a.window_bytes = presum_window_bytes(cfg, dmax);
  return SPS_OK;
}

// One uint8 pass (brute force or step one) with the configured kernel.
sps_status run_u8_pass(const sps_plan* p, const sps_dedisp_config& cfg, const uint8_t* x, int64_t pitch,
                       uint8_t* ws, int32_t rows, int32_t per, int32_t n_out, int64_t out_pitch, int32_t dmax,
                       void* out, int32_t out_u16, cudaStream_t st) {
  if (cfg.presum) {
    PresumPassArgs a{};
    sps_status s = presum_prepass(p, cfg, x, pitch, ws, rows, per, n_out, out_pitch, dmax, out, out_u16, st, &a);
    if (s) return s;
    return launch_presum_pass(a, cfg, st);
  }
  sps_status s = launch_expand(x, pitch, (int32_t)p->n_in, p->channels, ws, p->pitch4, st);
  if (s) return s;
  U8PassArgs a = u8_args(p, x, pitch, ws);
  a.di_pad = u8_di_pad(cfg);
  a.n_dm = rows;
  a.group_channels = per;
  a.n_groups = p->channels / per;
  a.n_out = n_out;
  a.out_pitch = out_pitch;
  a.dmax_tile = dmax;
  a.out = out;
  a.out_u16 = out_u16;
  return launch_u8_pass(a, cfg, st);
}

sps_status run_step1(const sps_plan* p, const uint8_t* x, int64_t pitch, uint8_t* ws, uint16_t* Y,
                     cudaStream_t st) {
  return run_u8_pass(p, p->cfg.step1, x, pitch, ws, (int32_t)p->coarse_dms.size(), p->channels / p->n_subbands,
                     (int32_t)p->n_1, p->y_pitch, p->dmax_step1, Y, 1, st);
}

sps_status run_step2(const sps_plan* p, const uint16_t* Y, int32_t* D, cudaStream_t st) {
  Step2Args a{};
  a.y = Y;
  a.y_pitch = p->y_pitch;
  a.y_len = (int32_t)p->n_1;
  a.d2 = p->d_d2;
  a.tiles = p->d_step2_tiles;
  a.n_tiles = p->n_step2_tiles;
  a.n_subbands = p->n_subbands;
  a.n_t = p->n_t;
  a.dmax_tile = p->dmax_step2;
  a.flush_every = p->step2_flush;
  a.D = D;
  a.status = p->d_status;
  return launch_step2(a, p->cfg.step2, st);
}

sps_status check_workspace(const sps_plan* p, void* ws, size_t ws_bytes) {
  if (!ws || ws_bytes < workspace_needed(p) || !aligned16(ws))
    return fail(SPS_ERR_INVALID_ARG, "workspace missing, smaller than sps_plan_workspace_bytes or not 16-byte aligned");
  return SPS_OK;
}

sps_status run_dedisperse(const sps_plan* p, const uint8_t* x, int64_t pitch, int32_t* D, void* ws,
                          size_t ws_bytes, cudaStream_t st) {
  sps_status s = check_x(p, x, pitch);
  if (s) return s;
  if (!D || !aligned16(D)) return fail(SPS_ERR_INVALID_ARG, "D must be non-null and 16-byte aligned");
  if ((s = check_workspace(p, ws, ws_bytes))) return s;
  uint8_t* x4 = static_cast<uint8_t*>(ws);
  if ((s = prepare_input(p, &x, &pitch, &x4, st))) return s;
  if (p->mode == SPS_MODE_BRUTE)
    return run_u8_pass(p, p->cfg.brute, x, pitch, x4, (int32_t)p->dms.size(), p->channels, p->n_t, p->n_t,
                       p->dmax_brute, D, 0, st);
  uint16_t* Y = reinterpret_cast<uint16_t*>(x4 + y_offset(p));
  if ((s = run_step1(p, x, pitch, x4, Y, st))) return s;
  return run_step2(p, Y, D, st);
}

sps_status run_snr(const sps_plan* p, const int32_t* D, double* snr, int32_t* peak_t, int32_t* peak_val,
                   int32_t* best, cudaStream_t st) {
  if (!D || !snr || !peak_t || !peak_val) return fail(SPS_ERR_INVALID_ARG, "null pointer");
  SnrArgs a{};
  a.D = D;
  a.max_boxcar = (int64_t)255 * p->channels * p->widths.back();
  a.status = p->d_status;
  a.n_dms = (int32_t)p->dms.size();
  a.n_t = p->n_t;
  a.widths = p->d_widths;
  a.n_widths = (int32_t)p->widths.size();
  a.snr = snr;
  a.peak_t = peak_t;
  a.peak_val = peak_val;
  a.decimate = p->smoothing == SPS_SMOOTH_DECIMATE ? 1 : 0;
  a.pow2_widths = 0;
  bool pow2 = p->widths.size() <= 30;
  for (size_t k = 0; k < p->widths.size() && pow2; k++) pow2 = p->widths[k] == (1 << k);
  if (pow2) a.pow2_widths = (int32_t)p->widths.size();
  a.best = best;
  return launch_snr(a, p->cfg.snr, st);
}

}  // namespace

size_t plan_workspace_bytes(const sps_plan* p) { return workspace_needed(p); }

sps_status run_search(const sps_plan* p, const uint8_t* x, int64_t pitch, int32_t* D, void* ws, size_t ws_bytes,
                      double* snr, int32_t* peak_t, int32_t* peak_val, int32_t* best, cudaStream_t st) {
  sps_status s = run_dedisperse(p, x, pitch, D, ws, ws_bytes, st);
  if (s) return s;
  return run_snr(p, D, snr, peak_t, peak_val, best, st);
}

sps_status dedisperse_into(const sps_plan* p, const uint8_t* x, int64_t pitch, int32_t* D, void* ws,
                           size_t ws_bytes, cudaStream_t st) {
  return run_dedisperse(p, x, pitch, D, ws, ws_bytes, st);
}

bool batched_pass_form(const sps_plan* p) { return p->mode == SPS_MODE_BRUTE && p->cfg.brute.presum > 0; }

sps_status brute_prepass(const sps_plan* p, const uint8_t* x, int64_t pitch, int32_t* D, void* ws,
                         size_t ws_bytes, cudaStream_t st, PresumPassArgs* args) {
  if (!batched_pass_form(p)) return fail(SPS_ERR_INVALID_ARG, "not a pre-summed brute-force plan");
  sps_status s = check_x(p, x, pitch);
  if (s) return s;
  if (!D || !aligned16(D)) return fail(SPS_ERR_INVALID_ARG, "D must be non-null and 16-byte aligned");
  if ((s = check_workspace(p, ws, ws_bytes))) return s;
  uint8_t* w = static_cast<uint8_t*>(ws);
  if ((s = prepare_input(p, &x, &pitch, &w, st))) return s;
  return presum_prepass(p, p->cfg.brute, x, pitch, w, (int32_t)p->dms.size(), p->channels, p->n_t, p->n_t,
                        p->dmax_brute, D, 0, st, args);
}

sps_status snr_into(const sps_plan* p, const int32_t* D, double* snr, int32_t* peak_t, int32_t* peak_val,
                    int32_t* best, cudaStream_t st) {
  return run_snr(p, D, snr, peak_t, peak_val, best, st);
}

}  // namespace sps

using namespace sps;

extern "C" {

sps_status sps_plan_create(const sps_plan_desc* desc, sps_plan** out) {
  clear_error();
  return plan_create(desc, out);
}

sps_status sps_plan_destroy(sps_plan* p) {
  if (!p) return SPS_OK;
  int cur = 0;
  bool swap = cudaGetDevice(&cur) == cudaSuccess && cur != p->device;
  if (swap) cudaSetDevice(p->device);
  cudaFree(p->d_delays);
  cudaFree(p->d_d1);
  cudaFree(p->d_d2);
  cudaFree(p->d_widths);
  cudaFree(p->d_step2_tiles);
  cudaFree(p->d_status);
  cudaFree(p->d_b0);
  cudaFree(p->d_offs);
  cudaFree(p->d_presum_series);
  cudaFree(p->d_presum_units);
  cudaFree(p->d_zap);
  cudaFree(p->d_presum_copies);
  cudaFree(p->d_presum_offs);
  if (swap) cudaSetDevice(cur);
  delete p;
  return SPS_OK;
}

int64_t sps_plan_input_samples(const sps_plan* p) { return p ? p->n_in : -1; }

int64_t sps_plan_step1_samples(const sps_plan* p) { return p ? p->n_1 : -1; }

sps_status sps_plan_delay_table(const sps_plan* p, int32_t* out) {
  clear_error();
  if (sps_status s = check_plan(p)) return s;
  if (!out) return fail(SPS_ERR_INVALID_ARG, "null output");
  const int32_t C = p->channels, n = (int32_t)p->dms.size();
  if (p->mode == SPS_MODE_BRUTE) {
    std::memcpy(out, p->delays.data(), p->delays.size() * sizeof(int32_t));
  } else {
    const int32_t S = p->n_subbands, per = C / S;
    for (int32_t i = 0; i < n; i++)
      for (int32_t c = 0; c < C; c++)
        out[(size_t)i * C + c] = p->d1[(size_t)p->coarse_of[i] * C + c] + p->d2[(size_t)i * S + c / per];
  }
  return SPS_OK;
}

sps_status sps_plan_subband_tables(const sps_plan* p, int32_t* d1, int32_t* d2) {
  clear_error();
  if (sps_status s = check_plan(p)) return s;
  if (p->mode != SPS_MODE_SUBBAND) return fail(SPS_ERR_INVALID_ARG, "plan is not in SUBBAND mode");
  if (!d1 || !d2) return fail(SPS_ERR_INVALID_ARG, "null output");
  std::memcpy(d1, p->d1.data(), p->d1.size() * sizeof(int32_t));
  std::memcpy(d2, p->d2.data(), p->d2.size() * sizeof(int32_t));
  return SPS_OK;
}

sps_status sps_plan_workspace_bytes(const sps_plan* p, size_t* bytes) {
  clear_error();
  if (sps_status s = check_plan(p)) return s;
  if (!bytes) return fail(SPS_ERR_INVALID_ARG, "null output");
  *bytes = workspace_any_config(p);
  return SPS_OK;
}

sps_status sps_plan_get_config(const sps_plan* p, sps_kernel_config* out) {
  clear_error();
  if (sps_status s = check_plan(p)) return s;
  if (!out) return fail(SPS_ERR_INVALID_ARG, "null output");
  *out = p->cfg;
  return SPS_OK;
}

sps_status sps_plan_set_config(sps_plan* p, const sps_kernel_config* cfg) {
  clear_error();
  if (sps_status s = check_plan(p)) return s;
  if (!cfg) return fail(SPS_ERR_INVALID_ARG, "null config");
  return apply_config(p, *cfg);
}

sps_status sps_dedisperse(const sps_plan* p, const uint8_t* x, int64_t pitch, int32_t* D, void* ws,
                          size_t ws_bytes, void* stream) {
  clear_error();
  NvtxRange nvtx("sps_dedisperse");
  if (sps_status s = check_plan(p)) return s;
  return run_dedisperse(p, x, pitch, D, ws, ws_bytes, (cudaStream_t)stream);
}

sps_status sps_subband_step1(const sps_plan* p, const uint8_t* x, int64_t pitch, uint16_t* Y, void* ws,
                             size_t ws_bytes, void* stream) {
  clear_error();
  NvtxRange nvtx("sps_subband_step1");
  if (sps_status s = check_plan(p)) return s;
  if (p->mode != SPS_MODE_SUBBAND) return fail(SPS_ERR_INVALID_ARG, "plan is not in SUBBAND mode");
  if (sps_status s = check_x(p, x, pitch)) return s;
  if (!Y || !aligned16(Y)) return fail(SPS_ERR_INVALID_ARG, "Y must be non-null and 16-byte aligned");
  if (sps_status s = check_workspace(p, ws, ws_bytes)) return s;
  uint8_t* w = static_cast<uint8_t*>(ws);
  if (sps_status s = prepare_input(p, &x, &pitch, &w, (cudaStream_t)stream)) return s;
  return run_step1(p, x, pitch, w, Y, (cudaStream_t)stream);
}

sps_status sps_subband_step2(const sps_plan* p, const uint16_t* Y, int32_t* D, void* stream) {
  clear_error();
  NvtxRange nvtx("sps_subband_step2");
  if (sps_status s = check_plan(p)) return s;
  if (p->mode != SPS_MODE_SUBBAND) return fail(SPS_ERR_INVALID_ARG, "plan is not in SUBBAND mode");
  if (!Y || !aligned16(Y) || !D || !aligned16(D)) return fail(SPS_ERR_INVALID_ARG, "Y and D must be 16-byte aligned");
  return run_step2(p, Y, D, (cudaStream_t)stream);
}

sps_status sps_integrate(const sps_plan* p, const int32_t* D, int32_t* B, void* stream) {
  clear_error();
  NvtxRange nvtx("sps_integrate");
  if (sps_status s = check_plan(p)) return s;
  if (!D || !B) return fail(SPS_ERR_INVALID_ARG, "null pointer");
  return launch_integrate(D, (int32_t)p->dms.size(), p->n_t, p->d_widths, (int32_t)p->widths.size(),
                          p->smoothing == SPS_SMOOTH_DECIMATE ? 1 : 0, B, p->d_status, (cudaStream_t)stream);
}

sps_status sps_snr(const sps_plan* p, const int32_t* D, double* snr, int32_t* peak_t, int32_t* peak_val,
                   int32_t* best, void* stream) {
  clear_error();
  NvtxRange nvtx("sps_snr");
  if (sps_status s = check_plan(p)) return s;
  return run_snr(p, D, snr, peak_t, peak_val, best, (cudaStream_t)stream);
}

sps_status sps_search(const sps_plan* p, const uint8_t* x, int64_t pitch, int32_t* D, void* ws,
                      size_t ws_bytes, double* snr, int32_t* peak_t, int32_t* peak_val, int32_t* best,
                      void* stream) {
  clear_error();
  NvtxRange nvtx("sps_search");
  if (sps_status s = check_plan(p)) return s;
  sps_status s = run_dedisperse(p, x, pitch, D, ws, ws_bytes, (cudaStream_t)stream);
  if (s) return s;
  return run_snr(p, D, snr, peak_t, peak_val, best, (cudaStream_t)stream);
}

sps_status sps_search_host(const sps_plan* p, const uint8_t* x_host, int64_t pitch, uint8_t* x_dev, int32_t* D,
                           void* ws, size_t ws_bytes, double* snr_dev, int32_t* peak_t_dev,
                           int32_t* peak_val_dev, int32_t* best_dev, double* snr_host, int32_t* peak_t_host,
                           int32_t* peak_val_host, int32_t* best_host, void* stream) {
  clear_error();
  NvtxRange nvtx("sps_search_host");
  if (sps_status s = check_plan(p)) return s;
  if (!x_host) return fail(SPS_ERR_INVALID_ARG, "null host input");
  if (sps_status s = check_x(p, x_dev, pitch)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n_out = (size_t)p->dms.size() * p->widths.size();
  SPS_CUDA(cudaMemcpyAsync(x_dev, x_host, (size_t)p->channels * pitch, cudaMemcpyHostToDevice, st));
  sps_status s = run_dedisperse(p, x_dev, pitch, D, ws, ws_bytes, st);
  if (s) return s;
  s = run_snr(p, D, snr_dev, peak_t_dev, peak_val_dev, best_dev, st);
  if (s) return s;
  if (snr_host) SPS_CUDA(cudaMemcpyAsync(snr_host, snr_dev, n_out * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (peak_t_host)
    SPS_CUDA(cudaMemcpyAsync(peak_t_host, peak_t_dev, n_out * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (peak_val_host)
    SPS_CUDA(cudaMemcpyAsync(peak_val_host, peak_val_dev, n_out * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (best_host && best_dev) SPS_CUDA(cudaMemcpyAsync(best_host, best_dev, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SPS_CUDA(cudaStreamSynchronize(st));
  return SPS_OK;
}

sps_status sps_presum_tables_verify(const int32_t* delays, int32_t rows, int32_t channels, int32_t per,
                                    int32_t build_n_out, int32_t read_n_out, const sps_dedisp_config* cfg) {
  clear_error();
  if (!delays || !cfg) return fail(SPS_ERR_INVALID_ARG, "null argument");
  if (rows < 1 || channels < 1 || per < 1 || channels % per || build_n_out < 1 || read_n_out < 1)
    return fail(SPS_ERR_INVALID_ARG, "rows, channels, per (dividing channels) and n_out must be positive");
  std::string why;
  if (!presum_config_supported(*cfg, &why)) return fail(SPS_ERR_INVALID_ARG, why);
  const std::vector<int32_t> d(delays, delays + (size_t)rows * channels);
  PresumTables t;
  if (sps_status s = build_presum_tables(d, rows, channels, per, build_n_out, *cfg, &t)) return s;
  if (!verify_presum_tables(d, rows, channels, per, read_n_out, *cfg, t, &why)) return fail(SPS_ERR_INVALID_ARG, why);
  return SPS_OK;
}

sps_status sps_plan_status(const sps_plan* p, uint32_t* host_status, int32_t clear) {
  clear_error();
  if (sps_status s = check_plan(p)) return s;
  if (!host_status) return fail(SPS_ERR_INVALID_ARG, "null output");
  SPS_CUDA(cudaMemcpy(host_status, p->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (clear) SPS_CUDA(cudaMemset(p->d_status, 0, sizeof(uint32_t)));
  return *host_status ? fail(SPS_ERR_TIMEOUT, "a kernel's bounded wait ran out") : SPS_OK;
}

const char* sps_status_string(sps_status s) {
  switch (s) {
    case SPS_OK: return "ok";
    case SPS_ERR_INVALID_ARG: return "invalid argument";
    case SPS_ERR_UNSUPPORTED: return "unsupported";
    case SPS_ERR_CUDA: return "CUDA error";
    case SPS_ERR_OOM: return "out of memory";
    case SPS_ERR_TIMEOUT: return "timeout";
    case SPS_ERR_NO_DEVICE: return "no device";
  }
  return "unknown status";
}

const char* sps_last_error(void) { return g_last_error.c_str(); }

int32_t sps_abi_version(void) { return 104; }

}  // extern "C"
