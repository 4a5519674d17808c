// Host tables of the pre-summed-pair de-dispersion (dedisperse_pair.cu).
//
// Channels of each group are taken in adjacent pairs (a, b = a + 1); an odd
// last channel is a pair with no partner.  For trial i the pair contributes
// Q_delta[t + d(i, b)] with delta = d(i, a) - d(i, b).  The plan needs:
//   series : every (a, b, delta) any trial uses, as rows of the workspace;
//   slots  : per (DM tile, group, chunk of pairs), the series the tile uses and
//            the start of their common window (d(i0, b) rounded down to 8);
//   offs   : per (DM tile, group, pair, trial), the byte offset of the trial's
//            first sample inside the staged chunk (slot, alignment copy, word).
// Tiles start at multiples of 64 samples, so nothing depends on the time tile.
#include <algorithm>
#include <vector>

#include "sps_internal.h"

namespace sps {

sps_status build_pair_tables(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per,
                             const sps_dedisp_config& cfg, int32_t dmax_tile, PairTables* out) {
  const int32_t G = C / per;
  const int32_t P = (per + 1) / 2;
  const int32_t Di = cfg.warps_dm * cfg.dms_per_thread;
  const int32_t di_pad = pair_di_pad(cfg);
  const int32_t cp = pair_chunk(cfg);
  const int32_t n_chunks = (P + cp - 1) / cp;
  const int32_t n_tiles = (rows + Di - 1) / Di;
  const int32_t wb = pair_window_bytes(cfg, dmax_tile);

  auto pair_a = [&](int32_t g, int32_t pl) { return g * per + 2 * pl; };
  auto pair_b = [&](int32_t g, int32_t pl) { return 2 * pl + 1 < per ? g * per + 2 * pl + 1 : -1; };
  auto delta = [&](int32_t i, int32_t a, int32_t b) {
    return b < 0 ? 0 : d[(size_t)i * C + a] - d[(size_t)i * C + b];
  };

  // series: per pair, every delta between its smallest and largest over all trials
  std::vector<int32_t> sbase((size_t)G * P), dmin((size_t)G * P);
  out->series.clear();
  for (int32_t g = 0; g < G; g++)
    for (int32_t pl = 0; pl < P; pl++) {
      const int32_t a = pair_a(g, pl), b = pair_b(g, pl);
      int32_t lo = INT32_MAX, hi = INT32_MIN;
      for (int32_t i = 0; i < rows; i++) {
        const int32_t v = delta(i, a, b);
        lo = std::min(lo, v);
        hi = std::max(hi, v);
      }
      if (lo < 0) return fail(SPS_ERR_INVALID_ARG, "a lower channel arrives before a higher one");
      sbase[(size_t)g * P + pl] = (int32_t)out->series.size();
      dmin[(size_t)g * P + pl] = lo;
      for (int32_t v = lo; v <= hi; v++) out->series.push_back({a, b, v, 0});
    }

  // slot lists per (tile, group, chunk), then the offsets
  int32_t slots_max = 0;
  struct Chunk { std::vector<int2> slots; };
  std::vector<Chunk> chunks((size_t)n_tiles * G * n_chunks);
  std::vector<int32_t> first_slot((size_t)n_tiles * G * P), lo_of((size_t)n_tiles * G * P),
      b0_of((size_t)n_tiles * G * P);
  for (int32_t tile = 0; tile < n_tiles; tile++) {
    const int32_t i0 = tile * Di, i1 = std::min(i0 + Di, rows) - 1;
    for (int32_t g = 0; g < G; g++)
      for (int32_t pl = 0; pl < P; pl++) {
        const int32_t a = pair_a(g, pl), b = pair_b(g, pl), bb = b < 0 ? a : b;
        int32_t lo = INT32_MAX, hi = INT32_MIN;
        for (int32_t i = i0; i <= i1; i++) {
          const int32_t v = delta(i, a, b);
          lo = std::min(lo, v);
          hi = std::max(hi, v);
        }
        const size_t key = ((size_t)tile * G + g) * P + pl;
        Chunk& ck = chunks[((size_t)tile * G + g) * n_chunks + pl / cp];
        const int32_t b0 = d[(size_t)i0 * C + bb] & ~7;
        first_slot[key] = (int32_t)ck.slots.size();
        lo_of[key] = lo;
        b0_of[key] = b0;
        for (int32_t v = lo; v <= hi; v++)
          ck.slots.push_back({sbase[(size_t)g * P + pl] + (v - dmin[(size_t)g * P + pl]), b0});
        slots_max = std::max<int32_t>(slots_max, (int32_t)ck.slots.size());
      }
  }
  out->slots_max = slots_max;
  out->wb = wb;
  out->slots.assign(chunks.size() * (size_t)(slots_max + 1), int2{-1, 0});
  for (size_t q = 0; q < chunks.size(); q++) {
    int2* row = &out->slots[q * (slots_max + 1)];
    for (size_t k = 0; k < chunks[q].slots.size(); k++) row[k] = chunks[q].slots[k];
    row[slots_max] = int2{(int32_t)chunks[q].slots.size(), 0};
  }
  out->offs.assign((size_t)n_tiles * G * P * di_pad, 0u);
  for (int32_t tile = 0; tile < n_tiles; tile++) {
    const int32_t i0 = tile * Di;
    for (int32_t g = 0; g < G; g++)
      for (int32_t pl = 0; pl < P; pl++) {
        const int32_t a = pair_a(g, pl), b = pair_b(g, pl), bb = b < 0 ? a : b;
        const size_t key = ((size_t)tile * G + g) * P + pl;
        for (int32_t r = 0; r < di_pad; r++) {
          const int32_t i = std::min(i0 + std::min(r, Di - 1), rows - 1);
          const int32_t slot = first_slot[key] + (delta(i, a, b) - lo_of[key]);
          const int32_t rel = d[(size_t)i * C + bb] - b0_of[key];
          out->offs[key * di_pad + r] = (uint32_t)((slot * 2 + (rel & 1)) * wb + (rel & ~1) * 2);
        }
      }
  }
  return SPS_OK;
}

}  // namespace sps
