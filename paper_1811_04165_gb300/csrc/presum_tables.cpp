// Host tables of the pre-summed de-dispersion (dedisperse_presum.cu).
//
// Channels of each group are taken in units of K = 2^presum adjacent channels
// c0 .. c0 + n - 1 (n = K, fewer at the end of a group).  The unit's reference
// is its last channel e = c0 + n - 1, the highest in frequency and so the
// least delayed (Sec. 1: the delay falls with frequency).  For trial i the
// unit contributes
//   S_rel[t + d(i, e)],   S_rel[u] = sum_j x[c0 + j][u + rel_j],
//   rel_j = d(i, c0 + j) - d(i, e) >= 0   (rel_{n-1} = 0),
// so one series serves every trial with the same tuple rel.  Each series is
// stored twice, copy 1 shifted by one sample, so that a trial whose reference
// delay d is odd reads aligned words of copy 1 at d - 1.  The plan needs:
//   series : every (unit, rel) any trial uses, as rows of the workspace, with
//            the sample range its trials read for outputs t < n_out:
//            [min d', max d' + n_out), d' = the reference delay rounded down
//            to even (copy 1 at d - 1 holds the samples from d on);
//   copies : per (DM tile, group, chunk of units), the windows of series
//            copies the tile reads -- one per (tuple, parity of d) that occurs,
//            each just long enough for its trials -- packed back to back in
//            the shared-memory stage: {row, start, (stage byte / 16) |
//            (bytes / 16) << 16, 0}, and last {count, total bytes};
//   offs   : per (DM tile, group, unit, trial), the offset of the trial's first
//            sample inside the packed stage, in 4-byte words as uint16 (a stage
//            is well below 256 KiB), so that one vector load fetches a warp's
//            offsets for a unit.
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

int32_t ref_delay(const std::vector<int32_t>& d, int32_t C, int32_t i, Unit un) {
  return d[(size_t)i * C + un.c0 + un.n - 1];
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

// The copy windows one unit needs in one DM tile of rows [i0, i1]: for tuple
// k of `rels` and parity j, the trials' smallest and largest even-rounded
// reference delay.  Window = [lo rounded down to 8, hi + Tt) samples.
struct TileCopy {
  int32_t k, j, lo, hi;
};

std::vector<TileCopy> tile_copies(const std::vector<int32_t>& d, int32_t C, int32_t i0, int32_t i1, Unit un,
                                  const std::vector<Rel>& rels) {
  std::vector<TileCopy> out;
  for (int32_t i = i0; i <= i1; i++) {
    const int32_t k = index_of(rels, rel_of(d, C, i, un));
    const int32_t de = ref_delay(d, C, i, un), j = de & 1, e = de & ~1;
    auto it = std::find_if(out.begin(), out.end(), [&](const TileCopy& c) { return c.k == k && c.j == j; });
    if (it == out.end()) {
      out.push_back({k, j, e, e});
    } else {
      it->lo = std::min(it->lo, e);
      it->hi = std::max(it->hi, e);
    }
  }
  std::sort(out.begin(), out.end(), [](const TileCopy& a, const TileCopy& b) {
    return a.k != b.k ? a.k < b.k : a.j < b.j;
  });
  return out;
}

int32_t copy_start(const TileCopy& c) { return c.lo & ~7; }

int32_t copy_bytes(const TileCopy& c, int32_t Tt) { return 2 * ((c.hi - copy_start(c) + Tt + 7) / 8 * 8); }

}  // namespace

int64_t count_presum_series(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per, int32_t K) {
  int64_t n = 0;
  const int32_t U = (per + K - 1) / K;
  for (int32_t g = 0; g < C / per; g++)
    for (int32_t u = 0; u < U; u++) n += (int64_t)distinct_rels(d, C, 0, rows - 1, unit_of(g, u, per, K)).size();
  return n;
}

int32_t presum_stage_data(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per, int32_t K,
                          int32_t Di, int32_t cu, int32_t Tt) {
  const int32_t U = (per + K - 1) / K;
  int64_t best = 0;
  for (int32_t i0 = 0; i0 < rows; i0 += Di) {
    const int32_t i1 = std::min(i0 + Di, rows) - 1;
    for (int32_t g = 0; g < C / per; g++)
      for (int32_t u0 = 0; u0 < U; u0 += cu) {
        int64_t bytes = 0;
        for (int32_t u = u0; u < std::min(u0 + cu, U); u++) {
          const Unit un = unit_of(g, u, per, K);
          for (const TileCopy& c : tile_copies(d, C, i0, i1, un, distinct_rels(d, C, i0, i1, un)))
            bytes += copy_bytes(c, Tt);
        }
        best = std::max(best, bytes);
      }
  }
  return (int32_t)std::min<int64_t>(best, INT32_MAX);
}

sps_status build_presum_tables(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per, int32_t n_out,
                               const sps_dedisp_config& cfg, PresumTables* out) {
  const int32_t K = 1 << cfg.presum;
  const int32_t G = C / per;
  const int32_t U = (per + K - 1) / K;
  const int32_t Di = cfg.warps_dm * cfg.dms_per_thread;
  const int32_t Tt = cfg.warps_time * 32 * cfg.samples_per_thread;
  const int32_t di_pad = presum_di_pad(cfg);
  const int32_t cu = presum_chunk(cfg);
  const int32_t n_chunks = (U + cu - 1) / cu;
  const int32_t n_tiles = (rows + Di - 1) / Di;

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
      std::vector<int32_t> lo(v.size(), INT32_MAX), hi(v.size(), INT32_MIN);
      for (int32_t i = 0; i < rows; i++) {
        const size_t k = (size_t)index_of(v, rel_of(d, C, i, un));
        const int32_t de = ref_delay(d, C, i, un) & ~1;
        lo[k] = std::min(lo[k], de);
        hi[k] = std::max(hi[k], de);
      }
      sbase[(size_t)g * U + u] = (int32_t)out->series.size();
      int32_t ulo = INT32_MAX, uhi = 0;
      for (size_t k = 0; k < v.size(); k++) {
        const int32_t slo = lo[k] & ~7, shi = (hi[k] + n_out + 7) / 8 * 8;
        out->series.push_back({un.c0, un.n, {v[k][0], v[k][1], v[k][2]}, slo, shi, 0});
        ulo = std::min(ulo, slo);
        uhi = std::max(uhi, shi);
      }
      const int32_t max_rel = v.back()[0];  // tuples sorted: the last has the largest first delay
      out->units.push_back({un.c0, un.n, sbase[(size_t)g * U + u], (int32_t)out->series.size(), max_rel, ulo, uhi,
                            0});
      out->max_rel = std::max(out->max_rel, max_rel);
    }

  // copy lists per (tile, group, chunk), packed in order; the offsets of each
  // trial point at its (tuple, parity) copy
  const size_t n_chunk_rows = (size_t)n_tiles * G * n_chunks;
  std::vector<std::vector<int4>> lists(n_chunk_rows);
  std::vector<int32_t> used(n_chunk_rows, 0);
  out->offs.assign((size_t)n_tiles * G * U * di_pad, 0);
  int32_t copies_max = 0, data_bytes = 0;
  for (int32_t tile = 0; tile < n_tiles; tile++) {
    const int32_t i0 = tile * Di, i1 = std::min(i0 + Di, rows) - 1;
    for (int32_t g = 0; g < G; g++)
      for (int32_t u = 0; u < U; u++) {
        const Unit un = unit_of(g, u, per, K);
        const size_t row = ((size_t)tile * G + g) * n_chunks + u / cu;
        const std::vector<Rel> rels = distinct_rels(d, C, i0, i1, un);
        const std::vector<TileCopy> copies = tile_copies(d, C, i0, i1, un, rels);
        std::vector<int32_t> dst(copies.size());
        for (size_t q = 0; q < copies.size(); q++) {
          const TileCopy& c = copies[q];
          const int32_t series = sbase[(size_t)g * U + u] + index_of(all[(size_t)g * U + u], rels[c.k]);
          dst[q] = used[row];
          lists[row].push_back({2 * series + c.j, copy_start(c), (dst[q] >> 4) | ((copy_bytes(c, Tt) >> 4) << 16), 0});
          used[row] += copy_bytes(c, Tt);
        }
        copies_max = std::max<int32_t>(copies_max, (int32_t)lists[row].size());
        data_bytes = std::max(data_bytes, used[row]);
        const size_t key = ((size_t)tile * G + g) * U + u;
        for (int32_t r = 0; r < di_pad; r++) {
          const int32_t i = std::min(i0 + std::min(r, Di - 1), rows - 1);
          const int32_t k = index_of(rels, rel_of(d, C, i, un));
          const int32_t de = ref_delay(d, C, i, un);
          size_t q = 0;
          while (copies[q].k != k || copies[q].j != (de & 1)) q++;
          const int64_t word = ((int64_t)dst[q] + 2 * ((de & ~1) - copy_start(copies[q]))) / 4;
          if (word > 0xFFFF) return fail(SPS_ERR_UNSUPPORTED, "pre-summed staging window beyond 256 KiB");
          out->offs[key * di_pad + r] = (uint16_t)word;
        }
      }
  }
  if (data_bytes >= (1 << 18) || copies_max >= (1 << 14))
    return fail(SPS_ERR_UNSUPPORTED, "pre-summed stage beyond 256 KiB or 16383 windows");
  out->copies_max = copies_max;
  out->data_bytes = data_bytes;
  out->copies.assign(n_chunk_rows * (size_t)(copies_max + 1), int4{-1, 0, 0, 0});
  for (size_t q = 0; q < n_chunk_rows; q++) {
    int4* row = &out->copies[q * (copies_max + 1)];
    for (size_t k = 0; k < lists[q].size(); k++) row[k] = lists[q][k];
    row[copies_max] = int4{(int32_t)lists[q].size(), used[q], 0, 0};
  }
  return SPS_OK;
}

// Checks, from the delay table alone, what the pass kernel will read through a
// set of tables: for every trial of every (tile, group, unit), its staged
// offset falls inside one window of its chunk's list, that window holds the
// trial's own series (same unit, same relative delays) in the copy of the
// trial's delay parity, the window's first sample plus the offset is the
// trial's even-rounded reference delay d', the window lies inside the stage's
// data, and the series' written range [lo, hi) covers d' .. d' + read_n_out - 1
// (every sample a valid output reads).  The first failure is described in *why.
bool verify_presum_tables(const std::vector<int32_t>& d, int32_t rows, int32_t C, int32_t per, int32_t read_n_out,
                          const sps_dedisp_config& cfg, const PresumTables& t, std::string* why) {
  const int32_t K = 1 << cfg.presum;
  const int32_t G = C / per;
  const int32_t U = (per + K - 1) / K;
  const int32_t Di = cfg.warps_dm * cfg.dms_per_thread;
  const int32_t Tt = cfg.warps_time * 32 * cfg.samples_per_thread;
  const int32_t di_pad = presum_di_pad(cfg);
  const int32_t cu = presum_chunk(cfg);
  const int32_t n_chunks = (U + cu - 1) / cu;
  const int32_t n_tiles = (rows + Di - 1) / Di;
  auto say = [&](const char* what, int32_t tile, int32_t g, int32_t u, int32_t r) {
    *why = std::string(what) + " (tile " + std::to_string(tile) + ", group " + std::to_string(g) + ", unit " +
           std::to_string(u) + ", trial " + std::to_string(r) + ")";
    return false;
  };
  for (int32_t tile = 0; tile < n_tiles; tile++)
    for (int32_t g = 0; g < G; g++)
      for (int32_t u = 0; u < U; u++) {
        const int32_t c0 = g * per + K * u, n = std::min(K, per - K * u), e = c0 + n - 1;
        const size_t row = ((size_t)tile * G + g) * n_chunks + u / cu;
        const int4* list = &t.copies[row * (t.copies_max + 1)];
        const int32_t count = list[t.copies_max].x;
        for (int32_t r = 0; r < Di; r++) {
          const int32_t i = tile * Di + r;
          if (i >= rows) break;
          const int32_t* di = &d[(size_t)i * C];
          const int32_t de = di[e], dprime = de & ~1, parity = de & 1;
          const int64_t off = 4 * (int64_t)t.offs[(((size_t)tile * G + g) * U + u) * di_pad + r];  // stage bytes
          int32_t q = 0;
          for (; q < count; q++) {
            const int32_t dst = (list[q].z & 0xFFFF) * 16, bytes = ((uint32_t)list[q].z >> 16) * 16;
            if (off >= dst && off + 2 * (int64_t)Tt <= (int64_t)dst + bytes) break;
          }
          if (q == count) return say("offset outside every window of the chunk", tile, g, u, r);
          const int32_t dst = (list[q].z & 0xFFFF) * 16, bytes = ((uint32_t)list[q].z >> 16) * 16;
          if (dst + bytes > t.data_bytes) return say("window beyond the stage data", tile, g, u, r);
          const int32_t srow = list[q].x, s = srow / 2;
          if (srow < 0 || s >= (int32_t)t.series.size()) return say("window row outside the series table", tile, g, u, r);
          if (srow % 2 != parity) return say("window of the wrong alignment copy", tile, g, u, r);
          const PresumSeries& ps = t.series[s];
          if (ps.c0 != c0 || ps.n != n) return say("window of another unit's series", tile, g, u, r);
          for (int32_t j = 0; j + 1 < n; j++)
            if (ps.rel[j] != di[c0 + j] - de) return say("window of a series with other relative delays", tile, g, u, r);
          if (list[q].y + (off - dst) / 2 != dprime) return say("offset does not land on the trial's delay", tile, g, u, r);
          if (dprime < ps.lo || (int64_t)dprime + read_n_out > ps.hi)
            return say("a valid output reads outside the series' written range", tile, g, u, r);
        }
      }
  return true;
}

}  // namespace sps
