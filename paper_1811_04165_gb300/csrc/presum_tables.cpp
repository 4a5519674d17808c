// Host tables of the pre-summed de-dispersion (dedisperse_presum.cu).
//
// Channels of each group are taken in units of K = 2^presum adjacent channels
// c0 .. c0 + n - 1 (n = K, fewer at the end of a group).  The unit's reference
// is its last channel e = c0 + n - 1, the highest in frequency and so the
// least delayed (Sec. 1: the delay falls with frequency).  For trial i the
// unit contributes
//   S_rel[t + d(i, e)],   S_rel[u] = sum_j x[c0 + j][u + rel_j],
//   rel_j = d(i, c0 + j) - d(i, e) >= 0   (rel_{n-1} = 0),
// so one series serves every trial with the same tuple rel.  The plan needs:
//   series : every (unit, rel) any trial uses, as rows of the workspace;
//   slots  : per (DM tile, group, chunk of units), the series the tile uses and
//            the start of their common window (d(i0, e) rounded down to 8);
//   offs   : per (DM tile, group, unit, trial), the offset of the trial's first
//            sample inside the staged chunk (slot, alignment copy, word), in
//            4-byte words as uint16 (a stage is well below 256 KiB), so that one
//            vector load fetches a warp's offsets for a unit.
// Tiles start at multiples of 64 samples, so nothing depends on the time tile.
#include <algorithm>
#include <array>
#include <vector>

#include "sps_internal.h"

namespace sps {
namespace {

using Rel = std::array<int32_t, 3>;

struct Unit {
  int32_t c0, n;
};

Unit unit_of(int32_t g, int32_t u, int32_t per, int32_t K) {
  return {g * per + K * u, std::min(K, per - K * u)};
}

Rel rel_of(const std::vector<int32_t>& d, int32_t C, int32_t i, Unit un) {
  Rel r{0, 0, 0};
  const int32_t* row = &d[(size_t)i * C];
  for (int32_t j = 0; j + 1 < un.n; j++) r[j] = row[un.c0 + j] - row[un.c0 + un.n - 1];
  return r;
}

// Distinct tuples of one unit over rows [i0, i1], in sorted order.
std::vector<Rel> distinct_rels(const std::vector<int32_t>& d, int32_t C, int32_t i0, int32_t i1, Unit un) {
  std::vector<Rel> v;
  v.reserve((size_t)(i1 - i0 + 1));
  for (int32_t i = i0; i <= i1; i++) v.push_back(rel_of(d, C, i, un));
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
  return v;
}

int32_t index_of(const std::vector<Rel>& v, const Rel& r) {
  return (int32_t)(std::lower_bound(v.begin(), v.end(), r) - v.begin());
}

}  // namespace

int64_t count_presum_series(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per, int32_t K) {
  int64_t n = 0;
  const int32_t U = (per + K - 1) / K;
  for (int32_t g = 0; g < C / per; g++)
    for (int32_t u = 0; u < U; u++) n += (int64_t)distinct_rels(d, C, 0, rows - 1, unit_of(g, u, per, K)).size();
  return n;
}

int32_t presum_slots(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per, int32_t K, int32_t Di,
                     int32_t cu) {
  const int32_t U = (per + K - 1) / K;
  int32_t best = 0;
  for (int32_t i0 = 0; i0 < rows; i0 += Di) {
    const int32_t i1 = std::min(i0 + Di, rows) - 1;
    for (int32_t g = 0; g < C / per; g++)
      for (int32_t u0 = 0; u0 < U; u0 += cu) {
        int32_t count = 0;
        for (int32_t u = u0; u < std::min(u0 + cu, U); u++)
          count += (int32_t)distinct_rels(d, C, i0, i1, unit_of(g, u, per, K)).size();
        best = std::max(best, count);
      }
  }
  return best;
}

sps_status build_presum_tables(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per,
                               const sps_dedisp_config& cfg, int32_t dmax_tile, PresumTables* out) {
  const int32_t K = 1 << cfg.presum;
  const int32_t G = C / per;
  const int32_t U = (per + K - 1) / K;
  const int32_t Di = cfg.warps_dm * cfg.dms_per_thread;
  const int32_t di_pad = presum_di_pad(cfg);
  const int32_t cu = presum_chunk(cfg);
  const int32_t n_chunks = (U + cu - 1) / cu;
  const int32_t n_tiles = (rows + Di - 1) / Di;
  const int32_t wb = presum_window_bytes(cfg, dmax_tile);

  // series: per unit, every tuple over all trials
  std::vector<int32_t> sbase((size_t)G * U);
  std::vector<std::vector<Rel>> all((size_t)G * U);
  out->series.clear();
  out->units.clear();
  out->max_rel = 0;
  for (int32_t g = 0; g < G; g++)
    for (int32_t u = 0; u < U; u++) {
      const Unit un = unit_of(g, u, per, K);
      std::vector<Rel>& v = all[(size_t)g * U + u];
      v = distinct_rels(d, C, 0, rows - 1, un);
      for (const Rel& r : v)
        if (std::min({r[0], r[1], r[2]}) < 0)
          return fail(SPS_ERR_INVALID_ARG, "a lower channel arrives before a higher one");
      sbase[(size_t)g * U + u] = (int32_t)out->series.size();
      for (const Rel& r : v) out->series.push_back({un.c0, un.n, {r[0], r[1], r[2]}, {0, 0, 0}});
      const int32_t max_rel = v.back()[0];  // tuples sorted: the last has the largest first delay
      out->units.push_back({un.c0, un.n, sbase[(size_t)g * U + u], (int32_t)out->series.size(), max_rel, {0, 0, 0}});
      out->max_rel = std::max(out->max_rel, max_rel);
    }

  // slot lists per (tile, group, chunk): each unit's tuples within the tile
  const size_t n_keys = (size_t)n_tiles * G * U;
  std::vector<std::vector<Rel>> tile_rels(n_keys);
  std::vector<int32_t> first_slot(n_keys), b0_of(n_keys);
  std::vector<std::vector<int2>> chunks((size_t)n_tiles * G * n_chunks);
  int32_t slots_max = 0;
  for (int32_t tile = 0; tile < n_tiles; tile++) {
    const int32_t i0 = tile * Di, i1 = std::min(i0 + Di, rows) - 1;
    for (int32_t g = 0; g < G; g++)
      for (int32_t u = 0; u < U; u++) {
        const Unit un = unit_of(g, u, per, K);
        const size_t key = ((size_t)tile * G + g) * U + u;
        std::vector<int2>& ck = chunks[((size_t)tile * G + g) * n_chunks + u / cu];
        tile_rels[key] = distinct_rels(d, C, i0, i1, un);
        b0_of[key] = d[(size_t)i0 * C + un.c0 + un.n - 1] & ~7;
        first_slot[key] = (int32_t)ck.size();
        for (const Rel& r : tile_rels[key])
          ck.push_back({sbase[(size_t)g * U + u] + index_of(all[(size_t)g * U + u], r), b0_of[key]});
        slots_max = std::max<int32_t>(slots_max, (int32_t)ck.size());
      }
  }
  out->slots_max = slots_max;
  out->wb = wb;
  out->slots.assign(chunks.size() * (size_t)(slots_max + 1), int2{-1, 0});
  for (size_t q = 0; q < chunks.size(); q++) {
    int2* row = &out->slots[q * (slots_max + 1)];
    for (size_t k = 0; k < chunks[q].size(); k++) row[k] = chunks[q][k];
    row[slots_max] = int2{(int32_t)chunks[q].size(), 0};
  }

  // offsets: slot of the trial's tuple, alignment copy and word of its first sample
  out->offs.assign(n_keys * di_pad, 0);
  for (int32_t tile = 0; tile < n_tiles; tile++) {
    const int32_t i0 = tile * Di;
    for (int32_t g = 0; g < G; g++)
      for (int32_t u = 0; u < U; u++) {
        const Unit un = unit_of(g, u, per, K);
        const size_t key = ((size_t)tile * G + g) * U + u;
        for (int32_t r = 0; r < di_pad; r++) {
          const int32_t i = std::min(i0 + std::min(r, Di - 1), rows - 1);
          const int32_t slot = first_slot[key] + index_of(tile_rels[key], rel_of(d, C, i, un));
          const int32_t rel = d[(size_t)i * C + un.c0 + un.n - 1] - b0_of[key];
          const int64_t word = ((int64_t)(slot * 2 + (rel & 1)) * wb + (rel & ~1) * 2) / 4;
          if (word > 0xFFFF) return fail(SPS_ERR_UNSUPPORTED, "pre-summed staging window beyond 256 KiB");
          out->offs[key * di_pad + r] = (uint16_t)word;
        }
      }
  }
  return SPS_OK;
}

}  // namespace sps
