/*
 * sps_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU statement of what the single-pulse
 * search hot path computes: dispersion delays, brute-force ("one-step") and
 * two-step subband incoherent dedispersion, sliding boxcar integration and
 * per-(DM, width) signal-to-noise with peak extraction.  Only tests/, the
 * package's smoke() check and bench.py's CPU-baseline leg may load it; the
 * product path never does.  It shares no code, header or table with the CUDA
 * library.
 *
 * The paper (Mikhailov & Sclocco, AMBER auto-tuning with genetic algorithms)
 * names these steps but prints no formula for them:
 *   - Sec. 1: de-dispersion is the shift and integration of frequency
 *     channels that removes the frequency sweep; then smoothing and S/N.
 *   - Sec. 2 and its first footnote: the pipeline's kernels are a two-step
 *     (subband) de-dispersion, time-series downsampling (smoothing) and S/N.
 *   - Table 2: channel count, channel bandwidth, subbands, DM grid.
 *   - Sec. 5: a one-step de-dispersion path exists beside the two-step one.
 * Every place where the text is silent is taken with the reading stated at
 * the function below (frequencies at channel centres, top channel as the
 * reference, delays rounded half away from zero in FP64, valid-only sliding
 * boxcars, population standard deviation over the whole valid series).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no -ffast-math),
 * so every FP64 expression below is evaluated as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Dispersion constant, s MHz^2 pc^-1 cm^3. */
#define ORACLE_K_DM 4.148808e3

/* Centre frequency of channel c (MHz); channel 0 is the lowest frequency.
 * Table 2 gives MIN_FREQ and CHANNEL_BANDWIDTH; the centre reading is ours. */
double oracle_channel_freq(double f_lo, double f_hi, int32_t channels, int32_t c) {
  double df = (f_hi - f_lo) / (double)channels;
  return f_lo + ((double)c + 0.5) * df;
}

/* Delay, in samples per unit DM, of a frequency f relative to f_ref:
 * K = k_DM * (1/f^2 - 1/f_ref^2) / t_samp, evaluated in this order. */
static double oracle_k_per_dm(double f, double f_ref, double t_samp) {
  double inv_f = 1.0 / (f * f);
  double inv_r = 1.0 / (f_ref * f_ref);
  return ORACLE_K_DM * (inv_f - inv_r) / t_samp;
}

/* Brute-force delay table d[i*C + c] = round_half_away(DM_i * K_c), with the
 * top channel's centre as reference (Sec. 1 "shift"; rounding reading ours). */
void oracle_delay_table(double f_lo, double f_hi, int32_t channels, double t_samp,
                        const double* dms, int32_t n_dms, int32_t* d) {
  double f_ref = oracle_channel_freq(f_lo, f_hi, channels, channels - 1);
  for (int32_t c = 0; c < channels; c++) {
    double kc = oracle_k_per_dm(oracle_channel_freq(f_lo, f_hi, channels, c), f_ref, t_samp);
    for (int32_t i = 0; i < n_dms; i++) d[(int64_t)i * channels + c] = (int32_t)llround(dms[i] * kc);
  }
}

/* Two-step subband delay tables (Sec. 2 first footnote; Table 2 SUBBANDS,
 * SUBBANDING_DMS, DMS).  Subband s holds channels [s*C/S, (s+1)*C/S); its
 * reference is the centre of its top channel.
 *   d1[k*C + c] = round(coarse_k * (k(f_c) - k(f_top(s(c)))))   intra-subband
 *   d2[i*S + s] = round(DM_i     * (k(f_top(s)) - k(f_ref)))    across subbands
 * Step two shifts each subband with the full trial DM_i. */
void oracle_subband_tables(double f_lo, double f_hi, int32_t channels, double t_samp,
                           int32_t n_subbands, const double* coarse_dms, int32_t n_coarse,
                           const double* dms, int32_t n_dms, int32_t* d1, int32_t* d2) {
  int32_t per = channels / n_subbands;
  double f_ref = oracle_channel_freq(f_lo, f_hi, channels, channels - 1);
  for (int32_t c = 0; c < channels; c++) {
    int32_t s = c / per;
    double f_top = oracle_channel_freq(f_lo, f_hi, channels, (s + 1) * per - 1);
    double k1 = oracle_k_per_dm(oracle_channel_freq(f_lo, f_hi, channels, c), f_top, t_samp);
    for (int32_t k = 0; k < n_coarse; k++) d1[(int64_t)k * channels + c] = (int32_t)llround(coarse_dms[k] * k1);
  }
  for (int32_t s = 0; s < n_subbands; s++) {
    double f_top = oracle_channel_freq(f_lo, f_hi, channels, (s + 1) * per - 1);
    double k2 = oracle_k_per_dm(f_top, f_ref, t_samp);
    for (int32_t i = 0; i < n_dms; i++) d2[(int64_t)i * n_subbands + s] = (int32_t)llround(dms[i] * k2);
  }
}

/* Dedispersion with an explicit delay table (Sec. 1; one-step path of Sec. 5):
 *   D[i][t] = sum_{c<C} x[c][t + d[i][c]],  0 <= t < n_t.
 * x is channel-major with a row pitch of `pitch` bytes.  The loop runs over c
 * for a whole output row at a time; integer addition makes the order moot. */
void oracle_dedisperse(const uint8_t* x, int64_t pitch, int32_t channels, int32_t n_t,
                       const int32_t* d, int32_t n_dms, int32_t* D) {
  for (int32_t i = 0; i < n_dms; i++) {
    int32_t* row = D + (int64_t)i * n_t;
    for (int32_t t = 0; t < n_t; t++) row[t] = 0;
    for (int32_t c = 0; c < channels; c++) {
      const uint8_t* xr = x + (int64_t)c * pitch + d[(int64_t)i * channels + c];
      for (int32_t t = 0; t < n_t; t++) row[t] += (int32_t)xr[t];
    }
  }
}

/* Subband step one: Y[k][s][t] = sum_{c in s} x[c][t + d1[k][c]], t < n_1. */
void oracle_subband_step1(const uint8_t* x, int64_t pitch, int32_t channels, int32_t n_subbands,
                          int32_t n_1, const int32_t* d1, int32_t n_coarse, int32_t* Y) {
  int32_t per = channels / n_subbands;
  for (int32_t k = 0; k < n_coarse; k++)
    for (int32_t s = 0; s < n_subbands; s++) {
      int32_t* row = Y + ((int64_t)k * n_subbands + s) * n_1;
      for (int32_t t = 0; t < n_1; t++) row[t] = 0;
      for (int32_t c = s * per; c < (s + 1) * per; c++) {
        const uint8_t* xr = x + (int64_t)c * pitch + d1[(int64_t)k * channels + c];
        for (int32_t t = 0; t < n_1; t++) row[t] += (int32_t)xr[t];
      }
    }
}

/* Subband step two: D[i][t] = sum_s Y[k(i)][s][t + d2[i][s]], t < n_t. */
void oracle_subband_step2(const int32_t* Y, int32_t n_coarse, int32_t n_subbands, int32_t n_1,
                          const int32_t* d2, const int32_t* coarse_of, int32_t n_dms,
                          int32_t n_t, int32_t* D) {
  (void)n_coarse;
  for (int32_t i = 0; i < n_dms; i++) {
    int32_t* row = D + (int64_t)i * n_t;
    for (int32_t t = 0; t < n_t; t++) row[t] = 0;
    for (int32_t s = 0; s < n_subbands; s++) {
      const int32_t* yr = Y + ((int64_t)coarse_of[i] * n_subbands + s) * n_1 + d2[(int64_t)i * n_subbands + s];
      for (int32_t t = 0; t < n_t; t++) row[t] += yr[t];
    }
  }
}

/* Sliding boxcar of width w over one series (the "smoothing" of Sec. 2):
 *   B[t] = sum_{u<w} D[t+u],  0 <= t <= n_t - w  (valid part only). */
void oracle_boxcar(const int32_t* D, int32_t n_t, int32_t w, int32_t* B) {
  for (int32_t t = 0; t + w <= n_t; t++) {
    int64_t s = 0;
    for (int32_t u = 0; u < w; u++) s += D[t + u];
    B[t] = (int32_t)s;
  }
}

/* S/N and peak of every (width, DM) pair (Sec. 2 names the S/N step):
 *   N = n_t - w + 1 valid boxcar samples, mean = sum B / N (FP64),
 *   sigma = sqrt(sum (B - mean)^2 / N)  (population, pulse included),
 *   P = max B, t* = smallest t with B[t] = P,
 *   snr = (P - mean) / sigma, and snr = 0 when sigma = 0.
 * Two passes over B in FP64; outputs are laid out [w][i]. */
void oracle_snr(const int32_t* D, int32_t n_dms, int32_t n_t, const int32_t* widths,
                int32_t n_widths, double* snr, int32_t* peak_t, int32_t* peak_val) {
  int32_t* B = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_t > 0 ? n_t : 1));
  for (int32_t wi = 0; wi < n_widths; wi++) {
    int32_t w = widths[wi];
    int32_t N = n_t - w + 1;
    for (int32_t i = 0; i < n_dms; i++) {
      oracle_boxcar(D + (int64_t)i * n_t, n_t, w, B);
      double sum = 0.0;
      int32_t pv = B[0], pt = 0;
      for (int32_t t = 0; t < N; t++) {
        sum += (double)B[t];
        if (B[t] > pv) { pv = B[t]; pt = t; }
      }
      double mean = sum / (double)N;
      double ss = 0.0;
      for (int32_t t = 0; t < N; t++) {
        double e = (double)B[t] - mean;
        ss += e * e;
      }
      double sigma = sqrt(ss / (double)N);
      int64_t o = (int64_t)wi * n_dms + i;
      snr[o] = sigma > 0.0 ? ((double)pv - mean) / sigma : 0.0;
      peak_t[o] = pt;
      peak_val[o] = pv;
    }
  }
  free(B);
}

/* Global detection: the (DM index, width index) with the largest S/N; ties go
 * to the smaller DM index, then to the smaller width index. */
void oracle_detect(const double* snr, int32_t n_dms, int32_t n_widths, int32_t* best_dm,
                   int32_t* best_w) {
  int32_t bi = 0, bw = 0;
  double best = snr[0];
  for (int32_t i = 0; i < n_dms; i++)
    for (int32_t wi = 0; wi < n_widths; wi++) {
      double v = snr[(int64_t)wi * n_dms + i];
      if (v > best) { best = v; bi = i; bw = wi; }
    }
  *best_dm = bi;
  *best_w = bw;
}
