// Plan construction: channel frequencies, integer delay tables and sizes.
//
// The paper (Sec. 1) describes de-dispersion only as the shift and
// integration of frequency channels; the delay law and its rounding are the
// cold-plasma dispersion law evaluated in FP64 and rounded half away from zero:
//   d(DM, c) = round(DM * k_DM * (f_c^-2 - f_top^-2) / t_samp),
// channel centres f_c ascending, the top channel as reference.  For the
// two-step path (Sec. 2, first footnote; Table 2 SUBBANDS, SUBBANDING_DMS,
// DMS) the intra-subband delay uses the coarse DM and the subband's top
// channel, the inter-subband delay the full trial DM.
// This file must be compiled without floating-point contraction so that the
// tables do not depend on the host architecture.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "sps_internal.h"

namespace {

constexpr double kDispersion = 4.148808e3;  // s MHz^2 pc^-1 cm^3

double centre_mhz(double f_lo, double f_hi, int32_t channels, int32_t c) {
  double width = (f_hi - f_lo) / (double)channels;
  return f_lo + ((double)c + 0.5) * width;
}

// samples of delay per unit DM between frequency f and reference f_ref
double samples_per_dm(double f, double f_ref, double t_samp) {
  double a = 1.0 / (f * f);
  double b = 1.0 / (f_ref * f_ref);
  return kDispersion * (a - b) / t_samp;
}

int32_t round_delay(double dm, double k) { return (int32_t)std::llround(dm * k); }

template <class T>
sps_status upload(const std::vector<T>& h, T** d) {
  if (h.empty()) { *d = nullptr; return SPS_OK; }
  cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(T));
  if (e == cudaErrorMemoryAllocation) return sps::fail(SPS_ERR_OOM, "device allocation of a plan table failed");
  if (e != cudaSuccess) return sps::cuda_fail(e, "cudaMalloc(plan table)");
  SPS_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SPS_OK;
}

// Largest delay spread inside any block of `tile` consecutive rows of a
// row-major table [rows][cols] whose columns are non-decreasing down the rows.
int32_t tile_spread(const std::vector<int32_t>& t, int32_t rows, int32_t cols, int32_t tile) {
  int32_t best = 0;
  for (int32_t r0 = 0; r0 < rows; r0 += tile) {
    int32_t r1 = std::min(r0 + tile, rows) - 1;
    for (int32_t c = 0; c < cols; c++)
      best = std::max(best, t[(size_t)r1 * cols + c] - t[(size_t)r0 * cols + c]);
  }
  return best;
}

// Staged-window tables of the uint8 pass for one configuration (see
// dedisperse_u8.cu): per DM tile and channel the first trial's delay rounded
// down to 16 (where the window starts), and per (tile, channel, trial) the
// byte offset of that trial's first sample inside the staged stage: copy
// (e & 3), channel row (c mod chunk), byte (e & ~3), e = d(i, c) - start.
// Tiles start at multiples of 128 samples, so none of this depends on time.
void build_u8_tables(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per,
                     const sps_dedisp_config& cfg, int32_t dmax, std::vector<int32_t>* b0,
                     std::vector<uint32_t>* offs) {
  const int32_t Di = cfg.warps_dm * cfg.dms_per_thread;
  const int32_t di_pad = sps::u8_di_pad(cfg);
  const int32_t wb = sps::u8_window_bytes(cfg, dmax);
  const int32_t copy_stride = cfg.chunk * wb;
  const int32_t n_tiles = (rows + Di - 1) / Di;
  const int32_t G = C / per, pairs = (per + 1) / 2;
  b0->assign((size_t)n_tiles * C, 0);
  offs->assign((size_t)n_tiles * G * pairs * di_pad * 2, 0u);
  for (int32_t tile = 0; tile < n_tiles; tile++) {
    const int32_t i0 = tile * Di;
    for (int32_t c = 0; c < C; c++) {
      const int32_t d0 = d[(size_t)i0 * C + c];
      (*b0)[(size_t)tile * C + c] = d0 & ~15;
      const int32_t g = c / per, cw = c % per, cl = cw % cfg.chunk;
      for (int32_t r = 0; r < di_pad; r++) {
        const int32_t i = std::min(i0 + std::min(r, Di - 1), rows - 1);
        const int32_t e = (d0 & 15) + d[(size_t)i * C + c] - d0;
        const uint32_t off = (uint32_t)((e & 3) * copy_stride + cl * wb + (e & ~3));
        (*offs)[((((size_t)tile * G + g) * pairs + cw / 2) * di_pad + r) * 2 + (cw & 1)] = off;
      }
    }
  }
}

}  // namespace

int64_t sps_plan::max_delay_brute() const {
  int64_t m = 0;
  for (int32_t v : delays) m = std::max<int64_t>(m, v);
  return m;
}

namespace sps {

// Default configurations, tried in order at plan creation: the pre-summed
// (quad) kernel for brute force (fastest on finely channelised bands), then the single-channel
// kernel, then smaller chunks for plans whose DM tiles span long delays.
std::vector<sps_kernel_config> default_configs() {
  std::vector<sps_kernel_config> out;
  const sps_dedisp_config u8[3] = {{4, 16, 8, 1, 16, 0}, {4, 16, 8, 1, 4, 0}, {1, 4, 1, 1, 2, 0}};
  const sps_dedisp_config s2[3] = {{4, 16, 8, 1, 8, 0}, {4, 16, 8, 1, 2, 0}, {1, 4, 1, 1, 1, 0}};
  sps_kernel_config c{};
  c.brute = {4, 16, 8, 1, 16, 2};
  c.step1 = u8[0];
  c.step2 = s2[0];
  c.snr = {256};
  out.push_back(c);
  for (int k = 0; k < 3; k++) {
    c.brute = u8[k];
    c.step1 = u8[k];
    c.step2 = s2[k];
    out.push_back(c);
  }
  return out;
}

// Largest packed window data of any (tile, group, chunk) of the pre-summed
// kernel for a configuration (cached).
int32_t cached_presum_stage(const sps_plan* p, int which, const sps_dedisp_config& c) {
  const int32_t Di = c.warps_dm * c.dms_per_thread, cu = presum_chunk(c);
  const int32_t Tt = c.warps_time * 32 * c.samples_per_thread;
  const int64_t key = ((int64_t)which << 62) | ((int64_t)c.presum << 58) | ((int64_t)Di << 42) |
                      ((int64_t)cu << 26) | Tt;
  auto it = p->presum_stage_cache.find(key);
  if (it != p->presum_stage_cache.end()) return it->second;
  const int32_t K = 1 << c.presum;
  const int32_t v = which == 0
                        ? presum_stage_data(p->delays, (int32_t)p->dms.size(), p->channels, p->channels, K, Di, cu, Tt)
                        : presum_stage_data(p->d1, (int32_t)p->coarse_dms.size(), p->channels,
                                            p->channels / p->n_subbands, K, Di, cu, Tt);
  p->presum_stage_cache[key] = v;
  return v;
}

// Largest delay spread of the plan's table for tiles of `tile` rows (cached).
int32_t cached_spread(const sps_plan* p, int which, int32_t tile) {
  const int64_t key = (int64_t)which << 32 | (uint32_t)tile;
  auto it = p->spread_cache.find(key);
  if (it != p->spread_cache.end()) return it->second;
  int32_t v = which == 0 ? tile_spread(p->delays, (int32_t)p->dms.size(), p->channels, tile)
                         : tile_spread(p->d1, (int32_t)p->coarse_dms.size(), p->channels, tile);
  p->spread_cache[key] = v;
  return v;
}

// Validate a configuration against the compiled variants and the device's
// shared memory, without changing the plan; fills the per-config sizes.
sps_status check_config(const sps_plan* p, const sps_kernel_config& cfg, ConfigCheck* out) {
  std::string why;
  auto pass_ok = [&](const sps_dedisp_config& c) {
    return c.presum ? presum_config_supported(c, &why) : u8_config_supported(c, &why);
  };
  for (int32_t v : {cfg.brute.presum, cfg.step1.presum})
    if (v < 0 || v > 2) return fail(SPS_ERR_INVALID_ARG, "presum must be 0, 1 or 2");
  if (p->mode == SPS_MODE_BRUTE && !pass_ok(cfg.brute))
    return fail(SPS_ERR_INVALID_ARG, "brute config: " + why);
  if (p->mode == SPS_MODE_SUBBAND) {
    if (!pass_ok(cfg.step1)) return fail(SPS_ERR_INVALID_ARG, "step1 config: " + why);
    if (!step2_config_supported(cfg.step2, &why)) return fail(SPS_ERR_INVALID_ARG, "step2 config: " + why);
  }
  if (!snr_config_supported(cfg.snr, &why)) return fail(SPS_ERR_INVALID_ARG, "snr config: " + why);

  const int32_t n_dms = (int32_t)p->dms.size();
  ConfigCheck c;
  if (p->mode == SPS_MODE_BRUTE) {
    const int32_t di = cfg.brute.warps_dm * cfg.brute.dms_per_thread;
    c.dmax_b = cached_spread(p, 0, di);
    const size_t need =
        cfg.brute.presum
            ? presum_smem_bytes(cfg.brute, cached_presum_stage(p, 0, cfg.brute))
            : u8_smem_bytes(cfg.brute, c.dmax_b, p->channels, 1);
    if (need > (size_t)p->max_smem)
      return fail(SPS_ERR_INVALID_ARG, "brute config needs more shared memory than a block may use");
  } else {
    c.dmax_1 = cached_spread(p, 1, cfg.step1.warps_dm * cfg.step1.dms_per_thread);
    // step-two tiles: runs of trials sharing one coarse DM, at most Di long
    const int32_t di = cfg.step2.warps_dm * cfg.step2.dms_per_thread;
    const int32_t S = p->n_subbands;
    for (int32_t i = 0; i < n_dms;) {
      const int32_t k = p->coarse_of[i];
      int32_t j = i;
      while (j < n_dms && p->coarse_of[j] == k && j - i < di) j++;
      c.tiles.push_back(k);
      c.tiles.push_back(i);
      c.tiles.push_back(j - i);
      for (int32_t s = 0; s < S; s++)
        c.dmax_2 = std::max(c.dmax_2, p->d2[(size_t)(j - 1) * S + s] - p->d2[(size_t)i * S + s]);
      i = j;
    }
    const int32_t di1 = cfg.step1.warps_dm * cfg.step1.dms_per_thread;
    const size_t need1 =
        cfg.step1.presum
            ? presum_smem_bytes(cfg.step1, cached_presum_stage(p, 1, cfg.step1))
            : u8_smem_bytes(cfg.step1, c.dmax_1, p->channels / S, S);
    if (need1 > (size_t)p->max_smem)
      return fail(SPS_ERR_INVALID_ARG, "step1 config needs more shared memory than a block may use");
    if (step2_smem_bytes(cfg.step2, c.dmax_2, p->n_subbands) > (size_t)p->max_smem)
      return fail(SPS_ERR_INVALID_ARG, "step2 config needs more shared memory than a block may use");
  }
  if (out) *out = std::move(c);
  return SPS_OK;
}

// Recompute everything that depends on the kernel configuration.
sps_status apply_config(sps_plan* p, const sps_kernel_config& cfg) {
  ConfigCheck chk;
  if (sps_status s = check_config(p, cfg, &chk)) return s;
  const int32_t n_dms = (int32_t)p->dms.size();
  const int32_t dmax_b = chk.dmax_b, dmax_1 = chk.dmax_1, dmax_2 = chk.dmax_2;
  const std::vector<int32_t>& tiles = chk.tiles;
  const sps_dedisp_config& pass = p->mode == SPS_MODE_BRUTE ? cfg.brute : cfg.step1;
  if (pass.presum) {
    PresumTables pt;
    sps_status s = p->mode == SPS_MODE_BRUTE
                       ? build_presum_tables(p->delays, n_dms, p->channels, p->channels, (int32_t)p->n_t, pass, &pt)
                       : build_presum_tables(p->d1, (int32_t)p->coarse_dms.size(), p->channels,
                                             p->channels / p->n_subbands, (int32_t)p->n_1, pass, &pt);
    if (s) return s;
    PresumSeries* dser = nullptr;
    PresumUnit* dunit = nullptr;
    int4* dslot = nullptr;
    uint16_t* doffs = nullptr;
    s = upload(pt.series, &dser);
    if (s == SPS_OK) s = upload(pt.units, &dunit);
    if (s == SPS_OK) s = upload(pt.copies, &dslot);
    if (s == SPS_OK) s = upload(pt.offs, &doffs);
    if (s != SPS_OK) {
      cudaFree(dser);
      cudaFree(dunit);
      cudaFree(dslot);
      return s;
    }
    cudaFree(p->d_presum_series);
    cudaFree(p->d_presum_units);
    cudaFree(p->d_presum_copies);
    cudaFree(p->d_presum_offs);
    p->d_presum_series = dser;
    p->d_presum_units = dunit;
    p->n_presum_units = (int32_t)pt.units.size();
    p->presum_max_rel = pt.max_rel;
    p->d_presum_copies = dslot;
    p->d_presum_offs = doffs;
    p->n_presum_series = (int32_t)pt.series.size();
    p->presum_copies_max = pt.copies_max;
    p->presum_data_bytes = pt.data_bytes;
  } else {
    std::vector<int32_t> b0;
    std::vector<uint32_t> offs;
    if (p->mode == SPS_MODE_BRUTE)
      build_u8_tables(p->delays, n_dms, p->channels, p->channels, cfg.brute, dmax_b, &b0, &offs);
    else
      build_u8_tables(p->d1, (int32_t)p->coarse_dms.size(), p->channels, p->channels / p->n_subbands, cfg.step1,
                      dmax_1, &b0, &offs);
    int32_t* db0 = nullptr;
    uint32_t* doffs = nullptr;
    sps_status st = upload(b0, &db0);
    if (st == SPS_OK) st = upload(offs, &doffs);
    if (st != SPS_OK) {
      cudaFree(db0);
      return st;
    }
    cudaFree(p->d_b0);
    cudaFree(p->d_offs);
    p->d_b0 = db0;
    p->d_offs = doffs;
  }
  if (p->mode == SPS_MODE_SUBBAND) {
    int32_t* dt = nullptr;
    sps_status st = upload(tiles, &dt);
    if (st != SPS_OK) return st;
    if (p->d_step2_tiles) cudaFree(p->d_step2_tiles);
    p->d_step2_tiles = dt;
    p->n_step2_tiles = (int32_t)(tiles.size() / 3);
    p->step2_tiles_host = tiles;
  }
  p->cfg = cfg;
  p->config_gen++;
  p->dmax_brute = dmax_b;
  p->dmax_step1 = dmax_1;
  p->dmax_step2 = dmax_2;
  return SPS_OK;
}

sps_status plan_create(const sps_plan_desc* d, sps_plan** out) {
  if (!d || !out) return fail(SPS_ERR_INVALID_ARG, "null descriptor or output pointer");
  *out = nullptr;
  if (d->channels < 1) return fail(SPS_ERR_INVALID_ARG, "channels must be >= 1");
  if (!(d->f_lo_mhz > 0.0) || !(d->f_hi_mhz > d->f_lo_mhz))
    return fail(SPS_ERR_INVALID_ARG, "need 0 < f_lo < f_hi");
  if (!(d->t_samp_s > 0.0)) return fail(SPS_ERR_INVALID_ARG, "t_samp must be > 0");
  if (d->n_samples < 1) return fail(SPS_ERR_INVALID_ARG, "n_samples must be >= 1");
  if (d->n_dms < 1 || !d->dms) return fail(SPS_ERR_INVALID_ARG, "need at least one DM");
  if (d->n_widths < 1 || !d->widths) return fail(SPS_ERR_INVALID_ARG, "need at least one width");
  for (int32_t i = 0; i < d->n_dms; i++) {
    if (!(d->dms[i] >= 0.0) || !std::isfinite(d->dms[i])) return fail(SPS_ERR_INVALID_ARG, "DMs must be finite and >= 0");
    if (i && d->dms[i] < d->dms[i - 1]) return fail(SPS_ERR_INVALID_ARG, "DMs must be ascending");
  }
  for (int32_t w = 0; w < d->n_widths; w++) {
    if (d->widths[w] < 1 || d->widths[w] > d->n_samples)
      return fail(SPS_ERR_INVALID_ARG, "widths must lie in [1, n_samples]");
    if (w && d->widths[w] <= d->widths[w - 1]) return fail(SPS_ERR_INVALID_ARG, "widths must be strictly ascending");
  }
  if (d->mode != SPS_MODE_BRUTE && d->mode != SPS_MODE_SUBBAND)
    return fail(SPS_ERR_INVALID_ARG, "unknown mode");
  if (d->smoothing != SPS_SMOOTH_SLIDING && d->smoothing != SPS_SMOOTH_DECIMATE)
    return fail(SPS_ERR_INVALID_ARG, "unknown smoothing");

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(SPS_ERR_NO_DEVICE, "no CUDA device visible");
  }

  sps_plan* p = new (std::nothrow) sps_plan();
  if (!p) return fail(SPS_ERR_OOM, "host allocation failed");
  SPS_CUDA(cudaGetDevice(&p->device));
  p->mode = d->mode;
  p->channels = d->channels;
  p->f_lo = d->f_lo_mhz;
  p->f_hi = d->f_hi_mhz;
  p->t_samp = d->t_samp_s;
  p->n_t = d->n_samples;
  p->dms.assign(d->dms, d->dms + d->n_dms);
  p->widths.assign(d->widths, d->widths + d->n_widths);
  p->smoothing = d->smoothing;
  if (d->zap && std::any_of(d->zap, d->zap + d->channels, [](uint8_t z) { return z != 0; }))
    for (int32_t c = 0; c < d->channels; c++) p->zap.push_back(d->zap[c] ? 1 : 0);
  const int32_t C = d->channels, n_dms = d->n_dms;
  const double f_ref = centre_mhz(p->f_lo, p->f_hi, C, C - 1);
  int64_t max_total = 0;

  if (d->mode == SPS_MODE_BRUTE) {
    p->delays.resize((size_t)n_dms * C);
    for (int32_t c = 0; c < C; c++) {
      double k = samples_per_dm(centre_mhz(p->f_lo, p->f_hi, C, c), f_ref, p->t_samp);
      for (int32_t i = 0; i < n_dms; i++) p->delays[(size_t)i * C + c] = round_delay(p->dms[i], k);
    }
    max_total = p->max_delay_brute();
  } else {
    const int32_t S = d->n_subbands;
    if (S < 1 || C % S) { delete p; return fail(SPS_ERR_INVALID_ARG, "n_subbands must divide channels"); }
    if (C / S > 257) {
      delete p;
      return fail(SPS_ERR_UNSUPPORTED, "a subband may hold at most 257 channels (16-bit step-one sums)");
    }
    if (d->n_coarse < 1 || !d->coarse_dms) { delete p; return fail(SPS_ERR_INVALID_ARG, "need coarse DMs"); }
    for (int32_t k = 0; k < d->n_coarse; k++) {
      if (!(d->coarse_dms[k] >= 0.0) || (k && d->coarse_dms[k] < d->coarse_dms[k - 1])) {
        delete p;
        return fail(SPS_ERR_INVALID_ARG, "coarse DMs must be >= 0 and ascending");
      }
    }
    p->n_subbands = S;
    p->coarse_dms.assign(d->coarse_dms, d->coarse_dms + d->n_coarse);
    p->coarse_of.resize(n_dms);
    if (d->coarse_of) {
      for (int32_t i = 0; i < n_dms; i++) {
        int32_t k = d->coarse_of[i];
        if (k < 0 || k >= d->n_coarse || (i && k < d->coarse_of[i - 1])) {
          delete p;
          return fail(SPS_ERR_INVALID_ARG, "coarse_of must be non-decreasing and < n_coarse");
        }
        p->coarse_of[i] = k;
      }
    } else {
      if (n_dms % d->n_coarse) { delete p; return fail(SPS_ERR_INVALID_ARG, "n_coarse must divide n_dms when coarse_of is NULL"); }
      for (int32_t i = 0; i < n_dms; i++) p->coarse_of[i] = i / (n_dms / d->n_coarse);
    }
    const int32_t per = C / S;
    p->d1.resize((size_t)d->n_coarse * C);
    p->d2.resize((size_t)n_dms * S);
    for (int32_t c = 0; c < C; c++) {
      int32_t s = c / per;
      double ftop = centre_mhz(p->f_lo, p->f_hi, C, (s + 1) * per - 1);
      double k1 = samples_per_dm(centre_mhz(p->f_lo, p->f_hi, C, c), ftop, p->t_samp);
      for (int32_t k = 0; k < d->n_coarse; k++) p->d1[(size_t)k * C + c] = round_delay(p->coarse_dms[k], k1);
    }
    for (int32_t s = 0; s < S; s++) {
      double ftop = centre_mhz(p->f_lo, p->f_hi, C, (s + 1) * per - 1);
      double k2 = samples_per_dm(ftop, f_ref, p->t_samp);
      for (int32_t i = 0; i < n_dms; i++) p->d2[(size_t)i * S + s] = round_delay(p->dms[i], k2);
    }
    int64_t m1 = 0, m2 = 0;
    for (int32_t v : p->d1) m1 = std::max<int64_t>(m1, v);
    for (int32_t v : p->d2) m2 = std::max<int64_t>(m2, v);
    p->n_1 = p->n_t + m2;
    p->y_pitch = (p->n_1 + 7) / 8 * 8;
    max_total = m1 + m2;
    // 16-bit step-two accumulation: subbands per flush so that the lane sum
    // of step-one values (each <= 255 * per) stays below 65536
    p->step2_flush = std::max<int32_t>(1, 65535 / (255 * per));
  }
  p->n_in = p->n_t + max_total;
  p->pitch4 = (p->n_in + 15) / 16 * 16;
  p->q_pitch = (int32_t)((p->n_in + 15) / 16 * 16);
  for (int32_t K : {2, 4})
    p->max_presum_series = std::max(p->max_presum_series,
                                    d->mode == SPS_MODE_BRUTE
                                        ? count_presum_series(p->delays, n_dms, C, C, K)
                                        : count_presum_series(p->d1, d->n_coarse, C, C / d->n_subbands, K));
  if (cudaDeviceGetAttribute(&p->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device) != cudaSuccess) {
    delete p;
    return fail(SPS_ERR_CUDA, "cudaDeviceGetAttribute(max shared memory)");
  }
  if (p->n_in > INT32_MAX / 2) { delete p; return fail(SPS_ERR_UNSUPPORTED, "input rows too long"); }
  int64_t max_sum = (int64_t)255 * C * p->widths.back();
  if (max_sum > INT32_MAX) { delete p; return fail(SPS_ERR_UNSUPPORTED, "boxcar sums could exceed int32"); }

  sps_status st = upload(p->widths, &p->d_widths);
  if (st == SPS_OK) st = upload(p->zap, &p->d_zap);
  if (st == SPS_OK) {
    std::vector<uint32_t> zero(1, 0u);
    st = upload(zero, &p->d_status);
  }
  if (st == SPS_OK) st = upload(p->delays, &p->d_delays);
  if (st == SPS_OK) st = upload(p->d1, &p->d_d1);
  if (st == SPS_OK) st = upload(p->d2, &p->d_d2);
  if (st == SPS_OK) {
    for (const sps_kernel_config& c : default_configs()) {
      st = apply_config(p, c);
      if (st != SPS_ERR_INVALID_ARG) break;
    }
  }
  if (st != SPS_OK) {
    sps_plan_destroy(p);
    return st;
  }
  *out = p;
  return SPS_OK;
}

}  // namespace sps
