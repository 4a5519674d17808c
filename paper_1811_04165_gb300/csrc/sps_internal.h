// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sps.h"

#include <nvtx3/nvToolsExt.h>

namespace sps {

// An NVTX range around a host entry point: profilers that record NVTX (ncu
// --nvtx, Nsight Systems) see each call and the kernels it launched; without
// one attached a push and a pop cost a few nanoseconds.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};


// Records a message for sps_last_error() and returns the status.
sps_status fail(sps_status s, const std::string& msg);
sps_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define SPS_CUDA(call)                                        \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return ::sps::cuda_fail(e_, #call); \
  } while (0)

// Kernel-side description of one de-dispersion pass over uint8 channels
// (brute force, or subband step one with one output row per (coarse, subband)).
struct U8PassArgs {
  const uint8_t* x;        // [channels][pitch]: copy 0 of every window
  int64_t pitch;           // bytes per channel row
  const uint8_t* x4;       // [3][channels][pitch4]: rows shifted by 1, 2, 3 bytes
  int64_t pitch4;          // bytes per shifted row (N_in rounded up to 16)
  int32_t win_limit;       // no staged window reads at or beyond this byte of a row
  const int32_t* b0;       // [n_tiles][channels]: first-trial delay rounded down to 16
  const uint32_t* offs;    // [n_tiles][n_groups][channel pairs][di_pad][2]: staged offsets
  int32_t di_pad;          // trials per tile rounded up to even
  int32_t n_dm;            // delay-table rows
  int32_t channels;        // total channels
  int32_t group_channels;  // channels summed into one output row
  int32_t n_groups;        // output rows per DM (1 for brute force)
  int32_t n_out;           // output samples per row
  int64_t out_pitch;       // output row pitch in elements
  int32_t dmax_tile;       // largest delay spread inside one DM tile of this config
  void* out;               // int32 rows (brute) or uint16 rows (step one)
  int32_t out_u16;         // 1: write uint16 sums (step one)
  uint32_t* status;        // device status word (bounded-wait timeouts)
  uint32_t one;            // 1, passed at run time (see madd in dedisperse_u8.cu)
};

// De-dispersion over pre-summed units of K = 2^presum adjacent channels
// (dedisperse_presum.cu, presum_tables.cpp).
struct PresumPassArgs {
  const uint16_t* q;       // [n_series][2][q_pitch]: unit-sum series, second copy shifted by one
  int32_t q_pitch;         // samples per series row (N_in rounded up to 16)
  const int4* copies;      // [tiles][groups][chunks][copies_max + 1]: {row, start,
                           // (stage byte / 16) | (bytes / 16) << 16, 0}; last {count, total bytes}
  int32_t copies_max;
  int32_t data_bytes;      // bytes of series windows per stage (the table follows)
  const uint16_t* offs;    // [tiles][groups][units][di_pad]: staged offsets in 4-byte words
  int32_t di_pad;
  int32_t n_dm;            // delay-table rows
  int32_t n_groups;
  int32_t group_units;     // units per group
  int32_t fold_units;      // units a 16-bit lane sums exactly: 65535 / (255 K)
  int32_t max_start;       // bound on any staged window's start (the pass's largest delay)
  int32_t n_out;
  int64_t out_pitch;
  int32_t dmax_tile;
  void* out;
  int32_t out_u16;
  uint32_t* status;
  int32_t window_bytes;    // staged bytes of one series window (the batched form reads it here)
};

// One pre-summed series: channels c0 .. c0 + n - 1, channel c0 + j (j < n - 1)
// taken rel[j] samples later than the last one.
// [lo, hi): the samples of the series (both copies) that any valid output
// reads, multiples of 8; the pre-pass writes only those.
struct PresumSeries {
  int32_t c0, n, rel[3], lo, hi, pad;
};

// One unit of K adjacent channels and the range of its series in the table;
// max_rel = the largest relative delay of any of its series (of its first
// channel); [lo, hi) = the union of its series' sample ranges.
struct PresumUnit {
  int32_t c0, n, s_begin, s_end, max_rel, lo, hi, pad;
};
static_assert(sizeof(PresumSeries) == 32 && sizeof(PresumUnit) == 32, "read as two int4 by the pre-pass");

struct PresumTables {
  std::vector<PresumSeries> series;
  std::vector<PresumUnit> units;
  int32_t max_rel = 0;
  std::vector<int4> copies;
  std::vector<uint16_t> offs;
  int32_t copies_max = 0;
  int32_t data_bytes = 0;
};

// Step two over uint16 subband series.
struct Step2Args {
  const uint16_t* y;       // [n_coarse][S][y_pitch]
  int64_t y_pitch;         // elements
  int32_t y_len;           // valid samples per Y row (N_1)
  const int32_t* d2;       // [n_dms][S]
  const int32_t* tiles;    // [n_tiles][3] = {coarse k, first DM, DM count}
  int32_t n_tiles;
  int32_t n_subbands;
  int32_t n_t;             // output samples per row
  int32_t dmax_tile;       // largest step-two delay spread inside a tile
  int32_t flush_every;     // subbands per 16-bit accumulation
  int32_t* D;              // [n_dms][n_t]
  uint32_t* status;        // device status word (bounded-wait timeouts)
};

struct SnrArgs {
  const int32_t* D;        // [n_dms][n_t]
  int64_t max_boxcar;      // 255 * channels * widest width
  int32_t n_dms;
  int32_t n_t;
  const int32_t* widths;   // device [n_widths]
  int32_t n_widths;
  double* snr;             // [n_widths][n_dms]
  int32_t* peak_t;
  int32_t* peak_val;
  uint32_t* status;
  int32_t decimate;        // 1: widths are downsampling factors
  int32_t pow2_widths;     // NW when the widths are exactly 1, 2, ..., 2^(NW-1); else 0
  int32_t* best;           // device int32[4] for the detection, or null
};

// Kernel launchers (dedisperse_u8.cu, dedisperse_presum.cu, dedisperse_step2.cu,
// snr.cu, zap.cu).  launch_snr also writes the detection when SnrArgs::best is
// set.  They validate the configuration
// against the kernel's compiled variants and return UNSUPPORTED otherwise.
sps_status launch_u8_pass(const U8PassArgs& a, const sps_dedisp_config& cfg, cudaStream_t st);
sps_status launch_step2(const Step2Args& a, const sps_dedisp_config& cfg, cudaStream_t st);
sps_status launch_snr(const SnrArgs& a, const sps_snr_config& cfg, cudaStream_t st);
sps_status launch_integrate(const int32_t* D, int32_t n_dms, int32_t n_t, const int32_t* widths,
                            int32_t n_widths, int32_t decimate, int32_t* B, uint32_t* status, cudaStream_t st);
sps_status launch_expand(const uint8_t* x, int64_t pitch, int32_t in_len, int32_t channels, uint8_t* x4,
                         int64_t pitch4, cudaStream_t st);
sps_status launch_presum_series(const uint8_t* x, int64_t pitch, int32_t in_len, const PresumUnit* units,
                                int32_t n_units, int32_t unit_channels, int32_t max_rel, const PresumSeries* series,
                                int32_t n_series, uint16_t* q, int32_t q_pitch, cudaStream_t st);
sps_status launch_presum_pass(const PresumPassArgs& a, const sps_dedisp_config& cfg, cudaStream_t st);
// Batched pre-summed pass: one launch over the work list of several passes of
// configuration `cfg` (d_passes / d_work in device memory; max_data_bytes =
// the largest data_bytes of the passes).  presum_pass_work appends the work
// items of pass index `pass`; presum_pass_blocks counts them.
sps_status launch_presum_pass_list(const PresumPassArgs* d_passes, const int4* d_work, int64_t n_work,
                                   const sps_dedisp_config& cfg, int32_t max_data_bytes, cudaStream_t st);
void presum_pass_work(const PresumPassArgs& a, const sps_dedisp_config& cfg, int32_t pass, std::vector<int4>* work);
int64_t presum_pass_blocks(const PresumPassArgs& a, const sps_dedisp_config& cfg);
sps_status launch_zap_copy(const uint8_t* x, int64_t pitch, int32_t in_len, const uint8_t* zap, int32_t channels,
                           uint8_t* out, int64_t out_pitch, cudaStream_t st);
bool presum_config_supported(const sps_dedisp_config& cfg, std::string* why);
size_t presum_smem_bytes(const sps_dedisp_config& cfg, int32_t data_bytes);
int presum_window_bytes(const sps_dedisp_config& cfg, int32_t dmax_tile);
int presum_di_pad(const sps_dedisp_config& cfg);
int presum_chunk(const sps_dedisp_config& cfg);  // units staged per chunk
// Host tables (presum_tables.cpp): series count over all rows, the largest
// packed window data of any (tile, group, chunk), and the full tables of one
// configuration.
int64_t count_presum_series(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per, int32_t K);
int32_t presum_stage_data(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per, int32_t K, int32_t Di,
                          int32_t units_per_chunk, int32_t Tt);
sps_status build_presum_tables(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per, int32_t n_out,
                               const sps_dedisp_config& cfg, PresumTables* out);
bool verify_presum_tables(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per, int32_t read_n_out,
                          const sps_dedisp_config& cfg, const PresumTables& t, std::string* why);
bool u8_config_supported(const sps_dedisp_config& cfg, std::string* why);
bool step2_config_supported(const sps_dedisp_config& cfg, std::string* why);
bool snr_config_supported(const sps_snr_config& cfg, std::string* why);
size_t u8_smem_bytes(const sps_dedisp_config& cfg, int32_t dmax_tile, int32_t group_channels, int32_t n_groups);
int u8_window_bytes(const sps_dedisp_config& cfg, int32_t dmax_tile);
int u8_di_pad(const sps_dedisp_config& cfg);
size_t step2_smem_bytes(const sps_dedisp_config& cfg, int32_t dmax_tile, int32_t n_subbands);

// Workspace a plan's de-dispersion needs, and de-dispersion into a given
// workspace (abi.cpp); used by entry points that supply their own workspace.
size_t plan_workspace_bytes(const sps_plan* p);

// Per-configuration sizes of a plan (plan.cpp).
struct ConfigCheck {
  int32_t dmax_b = 0, dmax_1 = 0, dmax_2 = 0;
  std::vector<int32_t> tiles;  // step-two tiles
};
sps_status check_config(const sps_plan* p, const sps_kernel_config& cfg, ConfigCheck* out);
sps_status apply_config(sps_plan* p, const sps_kernel_config& cfg);
sps_status run_search(const sps_plan* p, const uint8_t* x, int64_t pitch, int32_t* D, void* ws, size_t ws_bytes,
                      double* snr, int32_t* peak_t, int32_t* peak_val, int32_t* best, cudaStream_t st);
sps_status dedisperse_into(const sps_plan* p, const uint8_t* x, int64_t pitch, int32_t* D, void* ws,
                           size_t ws_bytes, cudaStream_t st);
// The batched brute-force form (batch.cpp): plans whose brute-force kernel is
// the pre-summed one run their pre-pass here (checks, zapping, the series into
// the workspace) and return the arguments of their pass, which a batched list
// launch then runs; snr_into is the S/N step of sps_search on its own.
bool batched_pass_form(const sps_plan* p);
sps_status brute_prepass(const sps_plan* p, const uint8_t* x, int64_t pitch, int32_t* D, void* ws,
                         size_t ws_bytes, cudaStream_t st, PresumPassArgs* args);
sps_status snr_into(const sps_plan* p, const int32_t* D, double* snr, int32_t* peak_t, int32_t* peak_val,
                    int32_t* best, cudaStream_t st);

}  // namespace sps

struct sps_plan {
  int device = 0;
  int32_t mode = SPS_MODE_BRUTE;
  int32_t channels = 0;
  double f_lo = 0, f_hi = 0, t_samp = 0;
  int32_t n_t = 0;
  std::vector<double> dms;
  std::vector<int32_t> widths;
  int32_t n_subbands = 0;
  std::vector<double> coarse_dms;
  std::vector<int32_t> coarse_of;

  // host tables
  std::vector<int32_t> delays;  // BRUTE: [n_dms][C]
  std::vector<int32_t> d1;      // SUBBAND: [n_coarse][C]
  std::vector<int32_t> d2;      // SUBBAND: [n_dms][S]
  std::vector<int32_t> step2_tiles_host;
  int64_t n_in = 0;             // input samples per channel
  int64_t n_1 = 0;              // SUBBAND: step-one samples
  int64_t y_pitch = 0;          // SUBBAND: elements per Y row
  int32_t step2_flush = 1;

  // device copies (owned)
  int32_t* d_delays = nullptr;
  int32_t* d_d1 = nullptr;
  int32_t* d_d2 = nullptr;
  int32_t* d_widths = nullptr;
  int32_t smoothing = SPS_SMOOTH_SLIDING;
  std::vector<uint8_t> zap;      // per channel, 1 = zapped (empty: none zapped)
  uint8_t* d_zap = nullptr;
  int32_t* d_step2_tiles = nullptr;
  int32_t n_step2_tiles = 0;
  uint32_t* d_status = nullptr;  // kernels' status word (bounded-wait timeouts)

  // staged-window tables of the uint8 pass (brute force, or step one)
  int32_t* d_b0 = nullptr;
  uint32_t* d_offs = nullptr;
  int64_t pitch4 = 0;            // bytes per row of the shifted copies

  // pre-summed-series tables (when the uint8 pass has presum > 0)
  sps::PresumSeries* d_presum_series = nullptr;
  sps::PresumUnit* d_presum_units = nullptr;
  int32_t n_presum_units = 0;
  int32_t presum_max_rel = 0;
  int4* d_presum_copies = nullptr;
  uint16_t* d_presum_offs = nullptr;
  int32_t n_presum_series = 0;   // of the current configuration's table
  int32_t presum_copies_max = 0;
  int32_t presum_data_bytes = 0;
  int32_t q_pitch = 0;           // samples per series row
  int64_t max_presum_series = 0; // over presum 1 and 2 (sizes the workspace)

  int max_smem = 0;              // opt-in shared memory per block of the device
  mutable std::map<int64_t, int32_t> spread_cache;     // tile delay spread by (table, rows)
  mutable std::map<int64_t, int32_t> presum_stage_cache;  // stage data by (table, K, rows, units, samples)

  sps_kernel_config cfg{};
  uint64_t config_gen = 0;       // bumped whenever the device tables are rebuilt
  // delay spread of one DM tile for the current configuration
  int32_t dmax_brute = 0, dmax_step1 = 0, dmax_step2 = 0;

  int64_t max_delay_brute() const;
};
