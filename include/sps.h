/*
 * sps.h -- C ABI of the GB300 single-pulse-search library (libsps.so).
 *
 * The library implements the data-parallel hot path of the AMBER single-pulse
 * search (Mikhailov & Sclocco, "AMBER auto-tuning optimization with genetic
 * algorithms"):
 *   incoherent de-dispersion of a uint8 filterbank over many DM trials
 *   (brute force, the one-step path of Sec. 5, or the two-step subband path of
 *   Sec. 2 and its first footnote), boxcar integration over a set of widths
 *   (the "smoothing" of Sec. 2) and per-(DM, width) S/N with peak extraction
 *   (the S/N step of Sec. 2); beside it the paper's genetic-algorithm tuner of
 *   all kernels' launch parameters together (Sec. 3.2), exhaustive search and
 *   pure random search (Sec. 4).
 *
 * Conventions shared by every entry point:
 *   - Status codes only; nothing is thrown across the ABI.  A failed call
 *     leaves its outputs unspecified and records a message for
 *     sps_last_error() (per calling thread).
 *   - "device" pointers are CUDA global-memory addresses on the plan's device
 *     (the device current when the plan was created); "host" pointers are CPU
 *     memory.  The caller owns every buffer passed in; the library never frees
 *     or retains them beyond the call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device entry points enqueue asynchronously on it and do not
 *     synchronise; results are ready when the stream has drained.
 *   - All integer results are exact; they are bit-identical for any launch
 *     configuration.
 *   - A plan is immutable after sps_plan_create / sps_plan_set_config and may
 *     be used from several streams at once, given distinct output/workspace
 *     buffers.
 */
#ifndef SPS_H
#define SPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPS_OK = 0,
  SPS_ERR_INVALID_ARG = 1,  /* a size, pointer, alignment or ordering check failed */
  SPS_ERR_UNSUPPORTED = 2,  /* valid request outside what the kernels implement   */
  SPS_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed                 */
  SPS_ERR_OOM = 4,          /* device or host allocation failed                     */
  SPS_ERR_TIMEOUT = 5,      /* a kernel's bounded wait ran out (sps_plan_status)    */
  SPS_ERR_NO_DEVICE = 6     /* no CUDA device is visible                            */
} sps_status;

enum { SPS_MODE_BRUTE = 0, SPS_MODE_SUBBAND = 1 };
enum { SPS_SMOOTH_SLIDING = 0, SPS_SMOOTH_DECIMATE = 1 };

typedef struct sps_plan sps_plan; /* opaque */

/* Survey description (Table 2 analogue).
 * Channel c (0 = lowest frequency) is centred at f_lo + (c + 1/2)(f_hi - f_lo)/channels.
 * The dispersion delay of channel c at trial DM is
 *   d = round_half_away(DM * 4.148808e3 * (f_c^-2 - f_top^-2) / t_samp)  samples,
 * f_top = the top channel's centre; the DM list must be ascending and >= 0.
 * SUBBAND mode (Sec. 2, first footnote): n_subbands divides channels, subband s
 * holds channels [s*C/S, (s+1)*C/S) with its top channel as reference;
 *   step one shifts channels inside a subband with the coarse DM of the trial,
 *   step two shifts subbands with the full trial DM.
 * coarse_dms (ascending) lists the step-one DMs; coarse_of[i] (non-decreasing,
 * < n_coarse) maps trial i to its coarse DM, NULL = i / (n_dms / n_coarse).
 * smoothing (Sec. 2 "downsampling (smoothing)"; Table 2 DOWNSAMPLING, NRSAMPLES):
 *   SLIDING  - widths are boxcar widths: B_w[t] = sum_{u<w} D[t+u], t <= N_t - w;
 *   DECIMATE - widths are downsampling factors f: X_f[j] = sum_{u<f} D[j f + u],
 *              j < N_t / f (the trailing N_t mod f samples are dropped); S/N is
 *              taken over the N_t / f downsampled samples (factor 1 = the
 *              series itself, Sec. 5) and peak_t is in input samples, f * j.
 * zap (Sec. 2, footnote: channels zapped for terrestrial RFI): zapped channels
 * contribute nothing to any sum; the search then reads a masked copy of x in
 * the workspace (sps_plan_workspace_bytes includes it). */
typedef struct {
  int32_t channels;
  double f_lo_mhz;
  double f_hi_mhz;
  double t_samp_s;
  int32_t n_samples;        /* N_t: output samples per batch                       */
  const double* dms;        /* host, n_dms entries                                 */
  int32_t n_dms;
  const int32_t* widths;    /* host, ascending, 1 <= w <= n_samples                */
  int32_t n_widths;
  int32_t mode;             /* SPS_MODE_BRUTE or SPS_MODE_SUBBAND                  */
  int32_t n_subbands;       /* SUBBAND only                                        */
  const double* coarse_dms; /* SUBBAND only, host, n_coarse entries                */
  int32_t n_coarse;
  const int32_t* coarse_of; /* SUBBAND only, host, n_dms entries or NULL           */
  int32_t smoothing;        /* SPS_SMOOTH_SLIDING (0) or SPS_SMOOTH_DECIMATE (1)   */
  const uint8_t* zap;       /* host, `channels` flags, non-zero = zapped, or NULL  */
} sps_plan_desc;

/* Launch and tiling parameters of one de-dispersion kernel (the Table 3 genes,
 * re-cast for sm_103a).  Block tile = (warps_dm * dms_per_thread) DMs by
 * (warps_time * 32 * samples_per_thread) samples; channels (or subbands) are
 * staged through shared memory `chunk` at a time.  `presum` (brute force and
 * step one) selects the kernel: 0 sums single channels; 1 and 2 sum series of
 * 2^presum adjacent channels pre-added once per batch (pairs, quads), each
 * series taken at the delay of its highest-frequency channel.  All are exact. */
typedef struct {
  int32_t dms_per_thread;     /* register tile along DM                            */
  int32_t samples_per_thread; /* register tile along time (4*k for the uint8 path)  */
  int32_t warps_dm;           /* warps of a block along DM                          */
  int32_t warps_time;         /* warps of a block along time                        */
  int32_t chunk;              /* channels (subbands) staged per shared-memory pass  */
  int32_t presum;             /* 0 single channels, 1 pairs, 2 quads (pre-summed)   */
} sps_dedisp_config;

/* Launch parameters of the fused boxcar + S/N kernel. */
typedef struct {
  int32_t threads;            /* threads per block (one block per DM row)           */
} sps_snr_config;

typedef struct {
  sps_dedisp_config brute;    /* one-step de-dispersion                             */
  sps_dedisp_config step1;    /* subband step one                                   */
  sps_dedisp_config step2;    /* subband step two                                   */
  sps_snr_config snr;         /* boxcar + S/N                                       */
} sps_kernel_config;

/* ---------------------------------------------------------------- plan */

/* Build a plan on the current CUDA device: channel frequencies and integer
 * delay tables in FP64 (host), uploaded to device memory the plan owns, plus
 * the default kernel configuration.  Copies every array of `desc`.
 * Errors: INVALID_ARG for inconsistent sizes, unsorted DMs, widths outside
 * [1, n_samples] or subbands not dividing channels; UNSUPPORTED when a
 * subband holds more than 257 channels (its sums must fit 16 bits);
 * NO_DEVICE / OOM / CUDA from device set-up. */
sps_status sps_plan_create(const sps_plan_desc* desc, sps_plan** out);
sps_status sps_plan_destroy(sps_plan* plan);

/* N_in: input samples each channel row must hold (N_t + the largest total delay). */
int64_t sps_plan_input_samples(const sps_plan* plan);
/* N_1: samples per step-one row (N_t + largest step-two delay); 0 in BRUTE mode. */
int64_t sps_plan_step1_samples(const sps_plan* plan);

/* Host copy of the brute-force delay table [n_dms][channels] (BRUTE mode) or of
 * the composed two-step table d1[k(i)][c] + d2[i][s(c)] (SUBBAND mode). */
sps_status sps_plan_delay_table(const sps_plan* plan, int32_t* host_out);
/* SUBBAND mode: host copies of d1 [n_coarse][channels] and d2 [n_dms][n_subbands]. */
sps_status sps_plan_subband_tables(const sps_plan* plan, int32_t* host_d1, int32_t* host_d2);

/* Bytes of device workspace that sps_dedisperse / sps_search need under any
 * kernel configuration: with zapped channels, a masked copy of x; then the
 * staged form of the batch (three copies shifted by 1, 2 and 3 samples for the
 * single-channel kernel, or the pre-summed pair or quad series, whichever is
 * largest); plus, in SUBBAND mode, the step-one output Y.  The calls themselves
 * accept any workspace at least as large as the current configuration uses. */
sps_status sps_plan_workspace_bytes(const sps_plan* plan, size_t* bytes);

sps_status sps_plan_get_config(const sps_plan* plan, sps_kernel_config* out);
/* Validates every field against the device's limits before accepting it. */
sps_status sps_plan_set_config(sps_plan* plan, const sps_kernel_config* cfg);

/* ---------------------------------------------------------------- hot path */

/* De-dispersion (Sec. 1 "shift and integration of frequency channels"):
 *   D[i][t] = sum_c x[c][t + d(i, c)],  0 <= t < N_t,  i < n_dms,
 * with d the brute-force table, or, in SUBBAND mode, step one then step two.
 * x: device, uint8 [channels][x_pitch], x_pitch >= N_in, a multiple of 16, x
 *    16-byte aligned; samples at and beyond N_in are ignored.
 * D: device, int32 [n_dms][N_t], 16-byte aligned.
 * workspace: device, >= sps_plan_workspace_bytes, 16-byte aligned; its
 *    contents need not be initialised and are overwritten. */
sps_status sps_dedisperse(const sps_plan* plan, const uint8_t* x, int64_t x_pitch, int32_t* D,
                          void* workspace, size_t workspace_bytes, void* stream);

/* sps_dedisperse without a workspace argument, for callers that cannot
 * allocate device memory when they run: a real-time beam loop held to a fixed
 * device-memory footprint once the observation has started, or code behind an
 * interface that hands it only its input and output buffers.  The paper has no
 * counterpart; this is a library convenience.
 * Same inputs, outputs and results as sps_dedisperse.  The workspace comes
 * from a file-scope device array of 96 MiB (enough for the brute-force search
 * of one 1536-channel, 1.024 s beam with the single-channel kernel, presum = 0:
 * 79 MB; not for the pre-summed series of presum 1 or 2, 236 and 614 MB, nor
 * for the subband path);
 * plans whose current configuration needs more are rejected with UNSUPPORTED
 * and a message giving both sizes.
 * Allocates nothing.  Every device that loads this entry point keeps the
 * array until the process exits.  All calls on a device share the array:
 * calls whose work overlaps on the GPU (other streams or threads) race and
 * corrupt each other's results.  Every call looks up the array's device
 * address (with the plan's device current, which is required); the first call
 * on each device loads the array there and should come before any stream
 * capture.  Nothing is cached, so the entry point stays valid after a device
 * reset. */
sps_status sps_dedisperse_noalloc(const sps_plan* plan, const uint8_t* x, int64_t x_pitch, int32_t* D,
                                  void* stream);

/* Subband step one alone (Sec. 2, first footnote):
 *   Y[k][s][t] = sum_{c in s} x[c][t + d1(k, c)],  t < N_1,
 * Y: device, uint16 [n_coarse][n_subbands][y_pitch], y_pitch = N_1 rounded up
 * to a multiple of 8; workspace as for sps_dedisperse (its shifted copies are
 * used, its Y part is not). */
sps_status sps_subband_step1(const sps_plan* plan, const uint8_t* x, int64_t x_pitch, uint16_t* Y,
                             void* workspace, size_t workspace_bytes, void* stream);
/* Subband step two alone: D[i][t] = sum_s Y[k(i)][s][t + d2(i, s)], t < N_t. */
sps_status sps_subband_step2(const sps_plan* plan, const uint16_t* Y, int32_t* D, void* stream);

/* Boxcar integration, materialised (for checking):
 *   B[w][i][t] = sum_{u < width_w} D[i][t + u] for t <= N_t - width_w, else 0;
 * with DECIMATE smoothing, B[w][i][j] = X_f[j] (f = width_w) for j < N_t / f,
 * else 0.
 * D: device int32 [n_dms][N_t]; B: device int32 [n_widths][n_dms][N_t]. */
sps_status sps_integrate(const sps_plan* plan, const int32_t* D, int32_t* B, void* stream);

/* Fused boxcar + S/N + peak (nothing materialised).  For each width w and DM i,
 * over the N = N_t - width + 1 valid boxcar samples B:
 *   snr = (N*max(B) - sum B) / sqrt(N*sum B^2 - (sum B)^2),
 * i.e. (peak - mean) / population sigma, from exact integer moments; 0 when
 * the series is constant.  peak_t = first t with B[t] = max(B).  With
 * DECIMATE smoothing the same over the N = N_t / f samples X_f[j]; peak_t is
 * then f times the first j of the maximum.
 * D must hold what sps_dedisperse produces for this plan: values in
 * [0, 255 * channels]; the kernel sizes its partial sums from that bound.
 * snr: device double [n_widths][n_dms]; peak_t, peak_val: device int32, same
 * shape.  best (may be NULL): device int32[4] = {DM index, width index,
 * peak_t, peak_val} of the largest S/N (ties: smaller DM, then smaller width).
 * Rows are staged whole in shared memory when they fit (about 56000 samples);
 * longer rows are streamed in chunks for widths 1, 2, 4, ..., 64 and refused
 * with UNSUPPORTED for other width sets and for decimating smoothing. */
sps_status sps_snr(const sps_plan* plan, const int32_t* D, double* snr, int32_t* peak_t,
                   int32_t* peak_val, int32_t* best, void* stream);

/* The whole hot path on device buffers: sps_dedisperse then sps_snr. */
sps_status sps_search(const sps_plan* plan, const uint8_t* x, int64_t x_pitch, int32_t* D,
                      void* workspace, size_t workspace_bytes, double* snr, int32_t* peak_t,
                      int32_t* peak_val, int32_t* best, void* stream);

/* The whole hot path from host memory: copies x_host (pinned memory keeps the
 * copy asynchronous) into x_dev, searches, copies snr / peak_t / peak_val /
 * best back into host memory and waits for `stream`.  Device buffers are as
 * for sps_search; any host output may be NULL to skip its copy. */
sps_status sps_search_host(const sps_plan* plan, const uint8_t* x_host, int64_t x_pitch,
                           uint8_t* x_dev, int32_t* D, void* workspace, size_t workspace_bytes,
                           double* snr_dev, int32_t* peak_t_dev, int32_t* peak_val_dev,
                           int32_t* best_dev, double* snr_host, int32_t* peak_t_host,
                           int32_t* peak_val_host, int32_t* best_host, void* stream);

/* ---------------------------------------------------------------- tuning */

/* Auto-tuning (Sec. 3.2 and Sec. 4): the genetic algorithm that tunes every
 * kernel's genes together, pure random search and exhaustive search, over a
 * discrete space.  An individual is one value index per gene; genes are
 * grouped by kernel (kernel_of non-decreasing).  Fitness is lower-is-better;
 * +inf marks a failed configuration (the penalty of Sec. 4).
 * Random numbers come from SplitMix64 seeded with `seed`; a run is
 * reproducible draw for draw (the order of draws is fixed in tune.cpp).
 * GA: N_pop individuals (even), tournament pools of max(2, round(pool_fraction
 * * N_pop)) distinct individuals, N_pop tournaments, pairing without identical
 * partners, per-kernel crossover with p_cross (uniform coin-toss or one-point,
 * undone when it breaks validity), per-kernel mutation with p_mut to a
 * different valid value, next population = fitter half of parents + fitter
 * half of offspring (an offspring left unevaluated because the budget ran
 * out takes no place; further parents fill it).  The evaluation budget counts
 * distinct individuals; repeats are served from a cache.
 * Resume (checkpoint of the best per generation, Sec. 4): `known_points` /
 * `known_fitness` hold n_known earlier evaluations (a tuning log); a point
 * found there takes the logged fitness instead of being measured, and
 * otherwise counts and traces like a new evaluation.  Since a search is
 * reproducible draw for draw, re-running it with its own log replays the
 * logged evaluations exactly and continues from where the log ends. */
enum { SPS_TUNE_GA = 0, SPS_TUNE_RANDOM = 1, SPS_TUNE_EXHAUSTIVE = 2 };
enum { SPS_CROSS_UNIFORM = 0, SPS_CROSS_ONE_POINT = 1 };
enum { SPS_SPACE_FULL = 0, SPS_SPACE_REDUCED = 1 };
#define SPS_TUNE_MAX_VALUES 8

typedef struct {
  int32_t n_genes;
  const int32_t* n_values;   /* host, values per gene (>= 1)                       */
  const int32_t* kernel_of;  /* host, kernel index per gene, non-decreasing        */
} sps_space;

typedef struct {
  int32_t algorithm;         /* SPS_TUNE_*                                         */
  int32_t crossover;         /* SPS_CROSS_* (GA)                                   */
  int32_t population;        /* N_pop (GA)                                         */
  int32_t max_generations;   /* GA stop                                            */
  double p_cross;            /* per-kernel crossover probability (GA)              */
  double p_mut;              /* per-kernel mutation probability (GA)               */
  double pool_fraction;      /* tournament pool as a fraction of N_pop (GA)        */
  int64_t max_evaluations;   /* budget of distinct evaluations (GA, random)        */
  uint64_t seed;
  const int32_t* known_points;  /* host [n_known][n_genes] or NULL (resume)        */
  const double* known_fitness;  /* host [n_known] or NULL                          */
  int64_t n_known;              /* 0 = nothing known                               */
  int32_t* final_population;    /* host [population][n_genes] or NULL: receives the
                                   end configurations (Sec. 5): the GA's last
                                   population; random search's last `population`
                                   distinct individuals (rows past the evaluation
                                   count set to -1); untouched by exhaustive search */
  int32_t renew;                /* GA renewal tries (>= 0; 0 = none): an offspring that
                                   repeats an evaluated individual or an earlier
                                   offspring of its generation is mutated again (a
                                   kernel, then one of its genes, drawn uniformly) up
                                   to this many times -- Sec. 3.2 forms pairs so that
                                   crossover yields new offspring, and a repeat is no
                                   new offspring */
} sps_search_desc;

typedef struct {
  double best_fitness;
  int64_t evaluations;       /* distinct individuals evaluated                     */
  int32_t generations;
  int32_t reserved;
} sps_search_result;

typedef int32_t (*sps_valid_fn)(const int32_t* point, void* user);          /* 1 = valid */
typedef double (*sps_fitness_fn)(const int32_t* point, void* user);
typedef void (*sps_trace_fn)(int64_t index, const int32_t* point, double fitness, void* user);

/* Host-only search over a caller-defined space with caller callbacks (no GPU
 * needed).  valid may be NULL (every point valid); trace (may be NULL) is
 * called once per distinct evaluation, in order.  best_point: host int32
 * [n_genes].  INVALID_ARG for a bad space or descriptor, or when no finite
 * fitness was seen. */
sps_status sps_optimize(const sps_space* space, const sps_search_desc* desc, sps_valid_fn valid,
                        sps_fitness_fn fitness, sps_trace_fn trace, void* user, int32_t* best_point,
                        sps_search_result* result);

/* The plan's tuning space: the genes of every kernel its search path launches
 * (brute: de-dispersion then S/N; subband: step one, step two, S/N), each a
 * list of powers of two (Sec. 3.2).  SPS_SPACE_REDUCED keeps six genes of the
 * subband path (5000 points) or five of the brute path.  Call with n_values
 * NULL to get n_genes; values is [n_genes][SPS_TUNE_MAX_VALUES]. */
sps_status sps_tune_space(const sps_plan* plan, int32_t which, int32_t max_genes, int32_t* n_genes,
                          int32_t* n_values, int32_t* kernel_of, int32_t* values);
/* The kernel configuration of a point (the plan's current one for genes the
 * space does not hold); INVALID_ARG when the point breaks a boundary condition
 * (no compiled variant, too many threads or too much shared memory). */
sps_status sps_tune_config(const sps_plan* plan, int32_t which, const int32_t* point, sps_kernel_config* out);
/* Live tuning on the GPU: fitness = median over three trials of the mean time
 * (ms) of `reps` back-to-back sps_search calls on the given buffers (as for
 * sps_search), +inf when a configuration is rejected or slower than limit_ms
 * (0 = no limit).  Leaves the plan on the best configuration found.
 * Synchronises `stream`. */
sps_status sps_tune(sps_plan* plan, int32_t which, const sps_search_desc* desc, const uint8_t* x,
                    int64_t x_pitch, int32_t* D, void* workspace, size_t workspace_bytes, double* snr,
                    int32_t* peak_t, int32_t* peak_val, int32_t reps, double limit_ms, sps_trace_fn trace,
                    void* user, int32_t* best_point, sps_search_result* result, void* stream);

/* ------------------------------------------------------- batched beams */

/* Batched beams.  A fixed set of beams (one plan each, in any mix of shapes
 * and configurations) searched by ONE launch: sps_batch_create captures every
 * beam's search into a CUDA graph whose beams run on `branches` concurrent
 * branches (beams spread over the branches by work, largest first);
 * sps_batch_launch replays the graph on a stream.  Beams on the pre-summed
 * brute-force kernel share their pass: the graph runs their pre-passes, then
 * one pass launch per kernel configuration (and occupancy class) over a device work list of (beam,
 * DM tile, time tile) descriptors of all those beams, then their S/N kernels;
 * other beams run their whole search on a branch.  Results are those of each
 * beam's own sps_search.  The ALERT setting
 * searches hundreds of beams at once (Sec. 1: beams spread over a GPU
 * cluster); the paper has no batched entry point, this is a library one.
 * buffers[b]: the device buffers of beam b as for sps_search (x with its
 * pitch, D, snr, peak_t, peak_val; best may be NULL); they stay owned by the
 * caller and must outlive the batch.  workspace: device, >=
 * sps_batch_workspace_bytes for the same plans and branch count, 256-byte
 * aligned; each branch uses its own region, and each beam of a shared pass
 * its own, so beams run concurrently.  The graph holds the plans' current configurations:
 * sps_batch_launch returns INVALID_ARG, launching nothing, once a plan has been
 * reconfigured since the capture; plans must outlive the batch.  Launches of
 * one batch on different streams must not overlap (they share the workspace). */
typedef struct sps_batch sps_batch;
typedef struct {
  const uint8_t* x;
  int64_t x_pitch;
  int32_t* D;
  double* snr;
  int32_t* peak_t;
  int32_t* peak_val;
  int32_t* best;
} sps_beam_buffers;
sps_status sps_batch_workspace_bytes(const sps_plan* const* plans, int32_t n_beams, int32_t branches,
                                     size_t* bytes);
sps_status sps_batch_create(const sps_plan* const* plans, const sps_beam_buffers* buffers, int32_t n_beams,
                            int32_t branches, void* workspace, size_t workspace_bytes, sps_batch** out);
sps_status sps_batch_launch(sps_batch* batch, void* stream);
/* How many shared-pass launches the graph holds (one per kernel configuration
 * and occupancy class: beams whose stages allow the same number of resident
 * blocks per SM share a launch). */
sps_status sps_batch_list_launches(const sps_batch* batch, int32_t* n);
sps_status sps_batch_destroy(sps_batch* batch);

/* ------------------------------------------------------- real-time serving */

/* A server for beams that stream consecutive batches in real time (Sec. 1:
 * ALERT searches every beam's 1.024 s of data within 1.024 s).  Not in the
 * paper; a library runtime.  Single-threaded: one host thread calls every
 * entry point of a server.
 *   - Memory: the server allocates one device arena of `hbm_budget_bytes` at
 *     creation and nothing afterwards.  Each beam keeps only its overlap tail
 *     there between batches ([channels][N_in - N_t] bytes).  A batch takes its
 *     input buffer, D, S/N tables and workspace from the arena when it is
 *     dispatched and returns them when it completes.
 *   - Admission: sps_server_add_beam admits a beam when its tail, plus one
 *     batch of it, fits beside the tails already resident (UNSUPPORTED
 *     otherwise).  Queued batches are admitted at dispatch time, in arrival
 *     order and each beam's in order, as slots and arena memory free up; a
 *     batch that does not fit yet waits, and later batches of other beams
 *     that fit may pass it.
 *   - Overlap tails: a batch is searched over its beam's tail (zeros before the
 *     first batch) followed by its N_t new samples; its window's last
 *     N_in - N_t samples become the tail of the beam's next batch.
 *   - Each batch runs on one of `max_inflight` concurrent slots (streams): the
 *     tail copy, the host-to-device copy of the new samples, sps_search and
 *     the copies of the S/N table and best back to the host pointers given at
 *     submission, which must stay valid until poll reports the batch.
 *   - Times are seconds on the host's steady clock; a completion time is the
 *     GPU-timeline end of the batch's last copy, mapped to that clock. */
typedef struct sps_server sps_server;
typedef struct {
  size_t hbm_budget_bytes;  /* the arena: every device byte the server uses     */
  int32_t max_inflight;     /* concurrent batches (1 = one batch at a time)    */
} sps_server_desc;
typedef struct {
  size_t budget_bytes;      /* arena size                                      */
  size_t used_bytes;        /* tails + batches in flight                       */
  size_t resident_bytes;    /* overlap tails                                   */
  size_t batch_bytes;       /* blocks of the batches in flight                 */
  int32_t inflight;         /* batches on the GPU                              */
  int32_t queued;           /* batches waiting for their beam, a slot or memory */
  int64_t admitted;         /* batches dispatched so far                       */
  int64_t waits_for_memory; /* dispatch attempts that found the arena too full */
  int64_t failed;           /* batches reported with an error status           */
} sps_server_stats;
/* Creates a server on the current device; OOM when the arena cannot be
 * allocated. */
sps_status sps_server_create(const sps_server_desc* desc, sps_server** out);
/* Admits a beam searched with `plan` (which must outlive the server and keep
 * its configuration); beam ids count from 0 and are never reused. */
sps_status sps_server_add_beam(sps_server* server, const sps_plan* plan, int32_t* beam_id);
/* Removes a beam: further submissions are refused (INVALID_ARG); batches
 * already queued or in flight still run and are reported; its tail returns
 * to the arena once none is left. */
sps_status sps_server_remove_beam(sps_server* server, int32_t beam_id);
/* Queues one batch of a beam: host uint8 [channels][host_pitch], N_t new
 * samples per channel (pinned memory keeps the copy asynchronous).  snr_host:
 * double [n_widths][n_dms]; best_host: int32[4] (either may be NULL).
 * Every check happens before the batch is queued: a non-OK status means it
 * was refused and nothing of it remains.  OK means it is queued, and its
 * outcome -- completion, or an error when it was dispatched -- is reported
 * by sps_server_poll under `tag`.  Then dispatches what it can. */
sps_status sps_server_submit(sps_server* server, int32_t beam_id, const uint8_t* host_x, int64_t host_pitch,
                             double* snr_host, int32_t* best_host, uint64_t tag);
/* Collects completed batches, dispatches what it can, then reports up to
 * `max` finished batches (oldest first): tags, completion times and, if
 * `status` is not NULL, each batch's status (OK, or the error that stopped
 * it).  *n = how many; batches beyond `max` stay for the next call. */
sps_status sps_server_poll(sps_server* server, uint64_t* tags, double* done_s, sps_status* status, int32_t max,
                           int32_t* n);
/* Batches queued, in flight, or finished and not yet reported. */
sps_status sps_server_pending(const sps_server* server, int32_t* n);
/* Arena occupancy and counters. */
sps_status sps_server_get_stats(const sps_server* server, sps_server_stats* out);
/* The host steady clock in seconds (the clock of submission and completion times). */
double sps_server_clock(void);
/* Waits for the batches in flight, then frees the arena; queued batches are dropped. */
sps_status sps_server_destroy(sps_server* server);

/* ---------------------------------------------------------------- misc */

/* Reads (synchronously) the plan's device status word; clears it if `clear`.
 * Bit 0 (1): a kernel's bounded wait for an asynchronous copy ran out.
 * Bit 1 (2): only in the bounds-checked build of the library (compiled with
 * SPS_BOUNDS_CHECK=1): a de-dispersion pass would have read outside a
 * shared-memory stage; the read was not made.
 * Returns TIMEOUT when the word is non-zero. */
sps_status sps_plan_status(const sps_plan* plan, uint32_t* host_status, int32_t clear);

/* Failure-detection self-check (the paper has no counterpart): launches on
 * `stream` one block that waits, through the same bounded mbarrier wait every
 * kernel uses, on a barrier nothing arrives at, for at most `polls` polls
 * (1 .. 2^20).  The wait runs out, sets the timeout bit of the plan's status
 * word (read it with sps_plan_status) and the block returns normally: no
 * fault, the context stays usable.  Asynchronous; INVALID_ARG on a null plan
 * or polls out of range. */
sps_status sps_plan_check_wait_timeout(const sps_plan* plan, int32_t polls, void* stream);

/* Host-only check of the pre-summed kernels' tables (no device needed; the
 * paper has no counterpart): builds the staging tables a plan would build for
 * `delays` (host int32 [rows][channels]; groups of `per` channels: `channels`
 * for brute force, channels / n_subbands for step one) and configuration
 * `cfg` (presum 1 or 2), with series written for build_n_out outputs, then
 * re-derives from the delays what each trial of each tile reads and checks it:
 * its staged offset lies in a window of its chunk, the window holds its own
 * series in the copy of its delay parity and starts where its delay says, the
 * window fits the stage, and the series' written range covers the samples of
 * read_n_out outputs.  OK when every check holds; INVALID_ARG naming the first
 * failure; UNSUPPORTED when the configuration's stage would not fit. */
sps_status sps_presum_tables_verify(const int32_t* delays, int32_t rows, int32_t channels, int32_t per,
                                    int32_t build_n_out, int32_t read_n_out, const sps_dedisp_config* cfg);

/* Measures the device's 32-bit integer add rate (adds/s over all SMs: independent
 * add chains split between the ALU pipe and multiply-adds by one on the FMA
 * pipe, best of three timed runs), the denominator against which the
 * de-dispersion kernels' integer work is compared.  Not in the paper; a
 * measurement helper.  Synchronises `stream`. */
sps_status sps_measure_int_add_rate(double* adds_per_s, void* stream);

const char* sps_status_string(sps_status s);
/* Message of the last failed call on this thread ("" if none). */
const char* sps_last_error(void);
/* ABI version of this header (major * 100 + minor). */
int32_t sps_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPS_H */
