// De-dispersion over pre-summed units of K = 2^presum adjacent channels
// (K = 2 pairs, K = 4 quads; brute force, or subband step one), exactly:
//
//   out[i * G + g][t] = sum_{c in group g} x[c][t + d(i, c)]
//                     = sum_{units (c0 .. e)} S_rel[t + d(i, e)],
//   S_rel[u] = sum_j x[c0 + j][u + rel_j],   rel_j = d(i, c0 + j) - d(i, e) >= 0.
//
// (Sec. 1: shift and integrate channels; Sec. 2, first footnote: step one.)
// Adjacent channels have nearly equal delays, so a tile of consecutive trials
// needs only a few tuples rel per unit.  A pre-pass writes, for every unit and
// every tuple its trials need, the series S_rel as uint16 (two copies, the
// second shifted by one sample, so every 32-bit shared load is aligned), over
// the samples those trials read for valid outputs only; the block then
// stages, per chunk of units, just the windows of the copies its tile reads (a
// host-built list, packed) with bulk asynchronous copies (TMA) into a ring of
// kStages mbarrier-tracked stages.  A 32-bit load holds two samples of a unit
// sum in 16-bit lanes: one add accumulates 2 K channel-samples, with no
// unpacking.  Samples outside a series' written range reach only output lanes
// past the end of the row (a lane's carry runs towards later samples), which
// are never stored.  Unit sums
// are <= 255 K, so 16-bit lanes are exact for 65535 / (255 K) units (128 pairs,
// 64 quads); partial sums fold into int32 registers that often.  A group whose
// size is not a multiple of K ends in a shorter unit.
#include <algorithm>

#include "sps_internal.h"
#include "tma.cuh"

namespace sps {
namespace {

constexpr int kMaxThreads = 512;
constexpr int kStages = 3;  // shared-memory ring depth

// NW words at shared address addr + 128 * m (immediate offsets).
template <int NW, int M = 0>
__device__ __forceinline__ void lds_row(uint32_t addr, uint32_t (&w)[NW]) {
  if constexpr (M < NW) {
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(w[M]) : "r"(addr), "n"(M * 128));
    lds_row<NW, M + 1>(addr, w);
  }
}

// The staged offsets of one unit for a warp's ND trials (uint16 words, one
// vector load), as byte offsets.
template <int ND>
__device__ __forceinline__ void load_offs(const uint16_t* p, uint32_t (&o)[ND]) {
  if constexpr (ND == 1) {
    o[0] = (uint32_t)*p << 2;
  } else {
    uint32_t w[ND / 2];
    if constexpr (ND == 8) {
      const uint4 v = *reinterpret_cast<const uint4*>(p);
      w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else if constexpr (ND == 4) {
      const uint2 v = *reinterpret_cast<const uint2*>(p);
      w[0] = v.x; w[1] = v.y;
    } else {
      w[0] = *reinterpret_cast<const uint32_t*>(p);
    }
#pragma unroll
    for (int k = 0; k < ND / 2; k++) {
      o[2 * k] = (w[k] & 0xFFFFu) << 2;
      o[2 * k + 1] = (w[k] >> 16) << 2;
    }
  }
}

// One block's tile: DM tile `tile`, time tile `ty`, group `g` of the pass `a`.
template <int ND, int NW>
__device__ __forceinline__ void presum_pass_block(const PresumPassArgs& a, int tile, int ty, int g, int wd,
                                                  int cp_max, int wb) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int wt = (int)(blockDim.x >> 5) / wd;
  const int Tt = wt * 64 * NW;
  const int Di = wd * ND;
  const int copies_max = a.copies_max;
  const int stage_bytes = a.data_bytes + cp_max * a.di_pad * 2;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * stage_bytes);
  uint64_t* empty = full + kStages;
  __shared__ volatile int aborted;
  __shared__ volatile int issued_upto;  // chunks [0, issued_upto) have been issued

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = (int)(blockDim.x >> 5);
  const int dm_sub = warp % wd, t_sub = warp / wd;
  const int i0 = tile * Di;
  const int t0 = ty * Tt;
  const int P = a.group_units;
  const int n_chunks = (P + cp_max - 1) / cp_max;
  const uint32_t toff = (uint32_t)(t_sub * 128 * NW + lane * 4);  // bytes
  const int64_t chunk_row = ((int64_t)tile * a.n_groups + g) * n_chunks;
  const bool clip = t0 + wb / 2 + a.max_start > a.q_pitch;  // windows may be cut at the row end
  // bounds-checked build: the largest staged offset whose NW words fit the
  // stage's windows, and the warp's trials inside a row of the offset table
  const int64_t lim = (int64_t)a.data_bytes - (int64_t)(toff + 128 * (NW - 1) + 4);
  if (kBoundsCheck && (dm_sub + 1) * ND > a.di_pad) stage_read_ok(1u, -1, a.status);

  if (tid == 0) {
    aborted = 0;
    issued_upto = 0;
    for (int k = 0; k < kStages; k++) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], nwarps);
    }
    fence_mbar_init();
  }
  __syncthreads();

  // One warp stages a whole chunk: the chunk's copy list names, per window,
  // the series copy (row), its first sample relative to the time tile, its
  // byte in the stage and its length; lane 0 also copies the chunk's offset
  // table and arrives on the stage's "full" barrier with the byte count (the
  // list's last entry, unless a window may be cut at the end of a row).  The
  // issuing warp fetches the count and its first list entry per lane a chunk
  // early (`fetch`).
  // A list entry is {row, start, (stage byte / 16) | (bytes / 16) << 16, 0};
  // the last is {count, total bytes}.
  struct Fetched { uint32_t nt; int row, start, at; };  // nt = count | total << 14
  auto fetch = [&](int ch) {
    const int4* list = a.copies + (chunk_row + ch) * (copies_max + 1);
    Fetched f;
    const int4 h = __ldg(&list[copies_max]);
    f.nt = (uint32_t)h.x | ((uint32_t)h.y << 14);
    const int4 e = lane < copies_max ? __ldg(&list[lane]) : make_int4(0, 0, 0, 0);
    f.row = e.x;
    f.start = e.y;
    f.at = e.z;
    return f;
  };
  auto issue = [&](int ch, const Fetched& f) {
    const int st = ch % kStages;
    uint8_t* sb = smem + st * stage_bytes;
    const int pb = ch * cp_max, cp = min(cp_max, P - pb);
    const int4* list = a.copies + (chunk_row + ch) * (copies_max + 1);
    const uint32_t tbl_bytes = (uint32_t)(cp * a.di_pad * 2);
    const int n = (int)(f.nt & 0x3FFFu);
    auto entry = [&](int q) {
      if (q == lane) return make_int3(f.row, f.start, f.at);
      const int4 e = __ldg(&list[q]);
      return make_int3(e.x, e.y, e.z);
    };
    auto length = [&](const int3& e) {
      const int w = (int)((uint32_t)e.z >> 16) * 16;
      return clip ? min(w, 2 * (a.q_pitch - (t0 + e.y))) : w;
    };
    uint32_t bytes_all = f.nt >> 14;
    if (clip) {
      bytes_all = 0;
      for (int q = lane; q < n; q += 32) bytes_all += (uint32_t)length(entry(q));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bytes_all += __shfl_xor_sync(0xffffffffu, bytes_all, o);
    }
    if (lane == 0) mbar_arrive_expect_tx(&full[st], bytes_all + tbl_bytes);
    __syncwarp();
    for (int q = lane; q < n; q += 32) {
      const int3 e = entry(q);
      const uint16_t* src = a.q + (int64_t)e.x * a.q_pitch + t0 + e.y;
      bulk_g2s(sb + ((uint32_t)e.z & 0xFFFFu) * 16, src, (uint32_t)length(e), &full[st]);
    }
    if (lane == 0) {
      const uint16_t* src = a.offs + (((int64_t)tile * a.n_groups + g) * P + pb) * a.di_pad;
      bulk_g2s(sb + a.data_bytes, src, tbl_bytes, &full[st]);
      issued_upto = ch + 1;
    }
  };

  uint32_t lanes[ND][NW];
  int32_t acc[ND][NW][2];
#pragma unroll
  for (int r = 0; r < ND; r++)
#pragma unroll
    for (int m = 0; m < NW; m++) { lanes[r][m] = 0u; acc[r][m][0] = 0; acc[r][m][1] = 0; }
  auto fold = [&]() {
#pragma unroll
    for (int r = 0; r < ND; r++)
#pragma unroll
      for (int m = 0; m < NW; m++) {
        acc[r][m][0] += (int32_t)(lanes[r][m] & 0xFFFFu);
        acc[r][m][1] += (int32_t)(lanes[r][m] >> 16);
        lanes[r][m] = 0u;
      }
  };

  // Chunks 0 and 1 go out first; after computing chunk ch, warp (ch mod
  // nwarps) stages chunk ch + 2 into the stage chunk ch - 1 used, once every
  // warp has released that stage.  No block-wide barrier: a warp waits only for
  // its data, and the issuer for warps one chunk behind.
  if (warp == 0)
    for (int k = 0; k < min(kStages - 1, n_chunks); k++) issue(k, fetch(k));

  // A warp that sees a wait run out stops waiting for the rest of the block
  // (`bad`) and records it for the block (`aborted`, read once at the end).
  int pending = 0;
  int ch = 0;
  int turn = 0;  // ch mod nwarps
  bool bad = false;
  for (; ch < n_chunks; ch++) {
    const int st = ch % kStages;
    const int cp = min(cp_max, P - ch * cp_max);
    const bool issuer = turn == warp && ch + kStages - 1 < n_chunks;
    if (++turn == nwarps) turn = 0;
    if (pending + cp > a.fold_units) { fold(); pending = 0; }
    Fetched next{};
    if (issuer) next = fetch(ch + kStages - 1);
    if (!bad && !mbar_wait(&full[st], (ch / kStages) & 1, a.status)) {
      bad = true;
      aborted = 1;
    }
    if (!bad) {
      const uint32_t base = smem_u32(smem) + (uint32_t)(st * stage_bytes) + toff;
      const uint16_t* tb =
          reinterpret_cast<const uint16_t*>(smem + st * stage_bytes + a.data_bytes) + dm_sub * ND;
      int p = 0;
      for (; p + 1 < cp; p += 2) {
        uint32_t e0[ND], e1[ND];
        load_offs<ND>(tb + p * a.di_pad, e0);
        load_offs<ND>(tb + (p + 1) * a.di_pad, e1);
#pragma unroll
        for (int r = 0; r < ND; r++) {
          uint32_t A[NW] = {}, B[NW] = {};
          if (stage_read_ok(e0[r], lim, a.status)) lds_row<NW>(base + e0[r], A);
          if (stage_read_ok(e1[r], lim, a.status)) lds_row<NW>(base + e1[r], B);
#pragma unroll
          for (int m = 0; m < NW; m++) lanes[r][m] += A[m] + B[m];
        }
      }
      if (p < cp) {
        uint32_t e0[ND];
        load_offs<ND>(tb + p * a.di_pad, e0);
#pragma unroll
        for (int r = 0; r < ND; r++) {
          uint32_t A[NW] = {};
          if (stage_read_ok(e0[r], lim, a.status)) lds_row<NW>(base + e0[r], A);
#pragma unroll
          for (int m = 0; m < NW; m++) lanes[r][m] += A[m];
        }
      }
    }
    pending += cp;
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
    if (issuer && !bad) {
      const int prev = ch - 1;  // the stage chunk ch + 2 reuses
      if (prev >= 0 && !mbar_wait(&empty[prev % kStages], (prev / kStages) & 1, a.status)) {
        bad = true;
        aborted = 1;
      } else {
        issue(ch + kStages - 1, next);
      }
    }
  }
  __syncthreads();  // every warp has left the loop
  if (aborted) {
    // let the copies still in flight (the last chunks issued) land before the
    // block's shared memory goes away; each wait is bounded
    if (tid == 0)
      for (int k = max(0, issued_upto - kStages); k < issued_upto; k++)
        mbar_wait(&full[k % kStages], (k / kStages) & 1, nullptr);
    return;
  }
  fold();

  // Each lane holds 2 consecutive samples per (trial, word).
  const bool vec = (a.out_pitch & 1) == 0;
#pragma unroll
  for (int r = 0; r < ND; r++) {
    const int i = i0 + dm_sub * ND + r;
    if (i >= a.n_dm) continue;
    const int64_t row = (int64_t)i * a.n_groups + g;
#pragma unroll
    for (int m = 0; m < NW; m++) {
      const int t = t0 + (int)(toff >> 1) + 64 * m;
      if (t >= a.n_out) continue;
      if (a.out_u16) {
        uint16_t* o = static_cast<uint16_t*>(a.out) + row * a.out_pitch + t;
        if (t + 1 < a.n_out && vec) {
          *reinterpret_cast<uint32_t*>(o) = (uint32_t)acc[r][m][0] | ((uint32_t)acc[r][m][1] << 16);
        } else {
          o[0] = (uint16_t)acc[r][m][0];
          if (t + 1 < a.n_out) o[1] = (uint16_t)acc[r][m][1];
        }
      } else {
        int32_t* o = static_cast<int32_t*>(a.out) + row * a.out_pitch + t;
        if (t + 1 < a.n_out && vec) {
          *reinterpret_cast<int2*>(o) = make_int2(acc[r][m][0], acc[r][m][1]);
        } else {
          o[0] = acc[r][m][0];
          if (t + 1 < a.n_out) o[1] = acc[r][m][1];
        }
      }
    }
  }
}

template <int ND, int NW>
__global__ void __launch_bounds__(kMaxThreads, 1)
presum_pass_kernel(PresumPassArgs a, int wd, int cp_max, int wb) {
  presum_pass_block<ND, NW>(a, blockIdx.x, blockIdx.y, blockIdx.z, wd, cp_max, wb);
}

// Batched form: one launch over a work list of tiles from several passes of
// the same configuration (several beams).  work[b] = {pass, DM tile, time
// tile, group}; each pass's arguments (and its window bytes) live in `passes`.
template <int ND, int NW>
__global__ void __launch_bounds__(kMaxThreads, 1)
presum_pass_list_kernel(const PresumPassArgs* __restrict__ passes, const int4* __restrict__ work, int wd,
                        int cp_max) {
  const int4 w = work[blockIdx.x];
  const PresumPassArgs& a = passes[w.x];
  presum_pass_block<ND, NW>(a, w.y, w.z, w.w, wd, cp_max, a.window_bytes);
}

// Adds bytes o + j .. o + j + 15 of W (24 bytes, o in 0 .. 7), for j = 0 and
// 1, into v[j] as eight words of 16-bit lanes.
__device__ __forceinline__ void add_window16x2(const uint32_t (&W)[6], int o, uint32_t (&v)[2][8]) {
#pragma unroll
  for (int j = 0; j < 2; j++) {
    const int oj = o + j;  // 0 .. 8
    const int wi = oj >> 2, sh = (oj & 3) * 8;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t lo = wi == 0 ? W[k] : (wi == 1 ? W[k + 1] : W[k + 2]);
      const uint32_t hi = wi == 0 ? W[k + 1] : (wi == 1 ? W[k + 2] : (k + 3 < 6 ? W[k + 3] : 0u));
      const uint32_t w = __funnelshift_r(lo, hi, sh);
      v[j][2 * k] += __byte_perm(w, 0u, 0x4140);
      v[j][2 * k + 1] += __byte_perm(w, 0u, 0x4342);
    }
  }
}

// Adds bytes O .. O + 8 of W (16 bytes, O in 0 .. 7) into v as 16-bit lanes:
// samples 0 .. 7 as four words (two per word), sample 8 in the low lane of
// v[4]; every word index and shift is a constant.
template <int O>
__device__ __forceinline__ void add_window9_c(const uint32_t (&W)[4], uint32_t (&v)[5]) {
#pragma unroll
  for (int k = 0; k < 2; k++) {
    const int wi = (O >> 2) + k, sh = (O & 3) * 8;
    const uint32_t w = sh ? __funnelshift_r(W[wi], W[wi + 1], sh) : W[wi];
    v[2 * k] += __byte_perm(w, 0u, 0x4140);
    v[2 * k + 1] += __byte_perm(w, 0u, 0x4342);
  }
  constexpr int b8 = O + 8;
  v[4] += __byte_perm(W[b8 >> 2], 0u, 0x4440 | (b8 & 3));
}

template <int O>
__device__ __forceinline__ void add_window9x2_c(const uint32_t (&W0)[4], const uint32_t (&W1)[4], uint32_t (&v0)[5],
                                                uint32_t (&v1)[5]) {
  add_window9_c<O>(W0, v0);
  add_window9_c<O>(W1, v1);
}

// Both halves of a thread share the offset o, and it is the same for every
// thread of a (series, channel), so the switch does not diverge.
__device__ __forceinline__ void add_window9x2_u(const uint32_t (&W0)[4], const uint32_t (&W1)[4], int o,
                                                uint32_t (&v0)[5], uint32_t (&v1)[5]) {
  switch (o) {
    case 0: add_window9x2_c<0>(W0, W1, v0, v1); break;
    case 1: add_window9x2_c<1>(W0, W1, v0, v1); break;
    case 2: add_window9x2_c<2>(W0, W1, v0, v1); break;
    case 3: add_window9x2_c<3>(W0, W1, v0, v1); break;
    case 4: add_window9x2_c<4>(W0, W1, v0, v1); break;
    case 5: add_window9x2_c<5>(W0, W1, v0, v1); break;
    case 6: add_window9x2_c<6>(W0, W1, v0, v1); break;
    default: add_window9x2_c<7>(W0, W1, v0, v1); break;
  }
}

// Eight samples of both copies of series s from u on: copy 0 from the nine
// summed samples v, copy 1 (one sample later) a byte permutation of them.
__device__ __forceinline__ void store_series9(uint16_t* q, int64_t q_pitch, int s, int u, const uint32_t (&v)[5]) {
  uint16_t* row0 = q + (int64_t)s * 2 * q_pitch + u;
  *reinterpret_cast<uint4*>(row0) = make_uint4(v[0], v[1], v[2], v[3]);
  // copy 1: word k = (sample 2 k + 1, sample 2 k + 2)
  *reinterpret_cast<uint4*>(row0 + q_pitch) =
      make_uint4(__byte_perm(v[0], v[1], 0x5432), __byte_perm(v[1], v[2], 0x5432), __byte_perm(v[2], v[3], 0x5432),
                 __byte_perm(v[3], v[4], 0x5432));
}

// Bytes u .. u + 23 of a channel row (u & 7 == 0) as six words; bytes at and
// beyond in_len read as 0.  `row` is 16-byte aligned.
__device__ __forceinline__ void load_row24(const uint8_t* row, int u, int in_len, uint32_t (&W)[6]) {
  if (u >= 0 && u + 24 <= in_len) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const uint2 t = __ldg(reinterpret_cast<const uint2*>(row + u + 8 * k));
      W[2 * k] = t.x;
      W[2 * k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      uint32_t w = 0;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const int p = u + 4 * k + i;
        if (p >= 0 && p < in_len) w |= (uint32_t)__ldg(row + p) << (8 * i);
      }
      W[k] = w;
    }
  }
}

constexpr int kSeriesThreads = 128;
constexpr int kSeriesBlock = kSeriesThreads * 16;  // samples per block

__device__ __forceinline__ void store_series(uint16_t* q, int64_t q_pitch, int s, int u0, const uint32_t (&v)[2][8]) {
#pragma unroll
  for (int j = 0; j < 2; j++) {
    uint4* o = reinterpret_cast<uint4*>(q + ((int64_t)s * 2 + j) * q_pitch + u0);
    o[0] = make_uint4(v[j][0], v[j][1], v[j][2], v[j][3]);
    o[1] = make_uint4(v[j][4], v[j][5], v[j][6], v[j][7]);
  }
}

// Series s, both copies j: q[(2 s + j) * q_pitch + u] = sum_c x[c0 + c][u + j + rel_c]
// (rel of the last channel 0), written for u in the series' range [lo, hi).
// A block takes one unit and kSeriesBlock samples: it stages the unit's
// channel rows once in shared memory (win_bytes per row, covering the block
// plus the unit's largest relative delay), then every thread computes eight
// samples of both copies of each of the unit's series in each half of the
// block (thread k: samples 8 k and 8 (k + kSeriesThreads) on), so that a
// warp's 16-byte stores cover 512 contiguous bytes.  The thread sums nine
// samples of copy 0; copy 1 (one sample later) is a byte permutation of them.
__global__ void __launch_bounds__(kSeriesThreads) presum_series_kernel(const uint8_t* x, int64_t pitch,
                                                                       int32_t in_len, const PresumUnit* units,
                                                                       const PresumSeries* series, uint16_t* q,
                                                                       int32_t q_pitch, int32_t win_bytes) {
  extern __shared__ __align__(16) uint8_t win[];
  const int4 uh = __ldg(reinterpret_cast<const int4*>(units + blockIdx.x));      // {c0, n, s_begin, s_end}
  const int4 ur = __ldg(reinterpret_cast<const int4*>(units + blockIdx.x) + 1);  // {max_rel, lo, hi, 0}
  const int ub = blockIdx.y * kSeriesBlock;
  if (ub >= ur.z || ub + kSeriesBlock <= ur.y) return;  // no series of the unit needs these samples
  // asynchronous 16-byte copies (all in flight at once); bytes at and beyond
  // in_len are zero-filled and never read
  for (int c = 0; c < uh.y; c++) {
    const uint8_t* row = x + (int64_t)(uh.x + c) * pitch;
    for (int k = threadIdx.x; k < win_bytes / 16; k += kSeriesThreads) {
      const int p = ub + 16 * k;
      const int n = min(16, max(0, in_len - p));
      const uint8_t* src = n > 0 ? row + p : row;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(win + c * win_bytes + 16 * k)),
                   "l"(src), "r"(n)
                   : "memory");
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int l0 = 8 * (int)threadIdx.x, l1 = l0 + 8 * kSeriesThreads;  // sample offsets of the halves
  const int u0 = ub + l0, u1 = ub + l1;
  // each series' header {c0, n, rel0, rel1}, {rel2, lo, hi, 0} is fetched one series ahead
  int4 hn = make_int4(0, 0, 0, 0), rn = make_int4(0, 0, 0, 0);
  if (uh.z < uh.w) {
    hn = __ldg(reinterpret_cast<const int4*>(series + uh.z));
    rn = __ldg(reinterpret_cast<const int4*>(series + uh.z) + 1);
  }
  for (int s = uh.z; s < uh.w; s++) {
    const int4 h = hn, r = rn;
    if (s + 1 < uh.w) {
      hn = __ldg(reinterpret_cast<const int4*>(series + s + 1));
      rn = __ldg(reinterpret_cast<const int4*>(series + s + 1) + 1);
    }
    const bool need0 = u0 < q_pitch && u0 + 8 > r.y && u0 < r.z;
    const bool need1 = u1 < q_pitch && u1 + 8 > r.y && u1 < r.z;
    if (!need0 && !need1) continue;
    uint32_t v0[5] = {0u, 0u, 0u, 0u, 0u}, v1[5] = {0u, 0u, 0u, 0u, 0u};
    auto channel = [&](int c, int rel) {
      const uint8_t* base = win + c * win_bytes + (rel & ~7);  // l0, l1 are multiples of 8
      const uint2* s0 = reinterpret_cast<const uint2*>(base + l0);
      const uint2* s1 = reinterpret_cast<const uint2*>(base + l1);
      const uint2 a0 = s0[0], a1 = s0[1], b0 = s1[0], b1 = s1[1];
      const uint32_t W0[4] = {a0.x, a0.y, a1.x, a1.y}, W1[4] = {b0.x, b0.y, b1.x, b1.y};
      add_window9x2_u(W0, W1, rel & 7, v0, v1);
    };
    if (h.y == 4) {  // a full quad (every unit but a short last one of a group)
      channel(0, h.z);
      channel(1, h.w);
      channel(2, r.x);
      channel(3, 0);
    } else {
      for (int c = 0; c < h.y; c++) channel(c, c + 1 == h.y ? 0 : (c == 0 ? h.z : (c == 1 ? h.w : r.x)));
    }
    if (need0) store_series9(q, q_pitch, s, u0, v0);
    if (need1) store_series9(q, q_pitch, s, u1, v1);
  }
}

// The same series straight from global memory, one (series, 16 samples) per
// thread: for units whose relative delays are too long to stage.
__global__ void __launch_bounds__(256) presum_series_direct_kernel(const uint8_t* x, int64_t pitch,
                                                                   int32_t in_len, const PresumSeries* series,
                                                                   int32_t n_series, uint16_t* q,
                                                                   int32_t q_pitch) {
  const int64_t per_row = q_pitch >> 4;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= per_row * n_series) return;
  const int s = (int)(id / per_row);
  const int u0 = (int)(id - (int64_t)s * per_row) << 4;
  const int4 h = __ldg(reinterpret_cast<const int4*>(series + s));
  const int4 r = __ldg(reinterpret_cast<const int4*>(series + s) + 1);  // {rel2, lo, hi, 0}
  if (u0 + 16 <= r.y || u0 >= r.z) return;
  const int rel2 = r.x;
  uint32_t v[2][8];
#pragma unroll
  for (int j = 0; j < 2; j++)
#pragma unroll
    for (int k = 0; k < 8; k++) v[j][k] = 0u;
  for (int c = 0; c < h.y; c++) {
    const int rel = c + 1 == h.y ? 0 : (c == 0 ? h.z : (c == 1 ? h.w : rel2));
    const int u = u0 + rel, b = u & ~7;
    uint32_t W[6];
    load_row24(x + (int64_t)(h.x + c) * pitch, b, in_len, W);
    add_window16x2(W, u - b, v);
  }
  store_series(q, q_pitch, s, u0, v);
}

typedef void (*PresumKernel)(PresumPassArgs, int, int, int);
typedef void (*PresumListKernel)(const PresumPassArgs*, const int4*, int, int);

template <int ND, int NW>
constexpr PresumKernel k() { return presum_pass_kernel<ND, NW>; }
template <int ND, int NW>
constexpr PresumListKernel kl() { return presum_pass_list_kernel<ND, NW>; }

struct Variant { int nd, nw; PresumKernel fn; PresumListKernel list; };
#define SPS_PRESUM_VARIANT(ND, NW) {ND, NW, k<ND, NW>(), kl<ND, NW>()}
const Variant kVariants[] = {
    SPS_PRESUM_VARIANT(1, 2), SPS_PRESUM_VARIANT(1, 4), SPS_PRESUM_VARIANT(1, 8), SPS_PRESUM_VARIANT(1, 16),
    SPS_PRESUM_VARIANT(2, 2), SPS_PRESUM_VARIANT(2, 4), SPS_PRESUM_VARIANT(2, 8), SPS_PRESUM_VARIANT(2, 16),
    SPS_PRESUM_VARIANT(4, 2), SPS_PRESUM_VARIANT(4, 4), SPS_PRESUM_VARIANT(4, 8),
    SPS_PRESUM_VARIANT(8, 2), SPS_PRESUM_VARIANT(8, 4),
};
#undef SPS_PRESUM_VARIANT

const Variant* find_variant(int nd, int nw) {
  for (const Variant& v : kVariants)
    if (v.nd == nd && v.nw == nw) return &v;
  return nullptr;
}

PresumKernel find(int nd, int nw) {
  const Variant* v = find_variant(nd, nw);
  return v ? v->fn : nullptr;
}

}  // namespace

int presum_window_bytes(const sps_dedisp_config& c, int32_t dmax_tile) {
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  return 2 * ((Tt + dmax_tile + 7 + 7) / 8 * 8);
}

int presum_di_pad(const sps_dedisp_config& c) { return (c.warps_dm * c.dms_per_thread + 7) / 8 * 8; }

int presum_chunk(const sps_dedisp_config& c) { return std::max(1, c.chunk >> c.presum); }

bool presum_config_supported(const sps_dedisp_config& c, std::string* why) {
  if (c.presum < 1 || c.presum > 2) {
    *why = "presum must be 1 (pairs) or 2 (quads) for this kernel";
    return false;
  }
  if (c.samples_per_thread % 2 || !find(c.dms_per_thread, c.samples_per_thread / 2)) {
    *why = "no compiled pre-summed variant for this (dms_per_thread, samples_per_thread)";
    return false;
  }
  const int threads = 32 * c.warps_dm * c.warps_time;
  if (c.warps_dm < 1 || c.warps_time < 1 || threads > kMaxThreads) {
    *why = "warps_dm * warps_time must lie in [1, 16]";
    return false;
  }
  if (c.chunk < 2 || c.chunk > 64 || (c.chunk & 1)) {
    *why = "chunk must be even and in [2, 64]";
    return false;
  }
  return true;
}

size_t presum_smem_bytes(const sps_dedisp_config& c, int32_t data_bytes) {
  const size_t stage = (size_t)data_bytes + (size_t)presum_chunk(c) * presum_di_pad(c) * 2;
  return kStages * stage + 16 * kStages;
}

sps_status launch_presum_series(const uint8_t* x, int64_t pitch, int32_t in_len, const PresumUnit* units,
                                int32_t n_units, int32_t unit_channels, int32_t max_rel, const PresumSeries* series,
                                int32_t n_series, uint16_t* q, int32_t q_pitch, cudaStream_t st) {
  if (n_series == 0) return SPS_OK;
  // staged window per channel row: the block's samples, the largest relative
  // delay, and the 16-byte reach of the last thread's loads
  const int64_t win = ((int64_t)kSeriesBlock + max_rel + 16 + 15) / 16 * 16;
  const int64_t smem = win * unit_channels;
  if (smem <= 96 * 1024) {
    SPS_CUDA(cudaFuncSetAttribute(presum_series_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)n_units, (unsigned)((q_pitch + kSeriesBlock - 1) / kSeriesBlock));
    presum_series_kernel<<<grid, kSeriesThreads, (size_t)smem, st>>>(x, pitch, in_len, units, series, q, q_pitch,
                                                                    (int32_t)win);
  } else {
    const int64_t threads = (int64_t)(q_pitch >> 4) * n_series;
    presum_series_direct_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(x, pitch, in_len, series,
                                                                                   n_series, q, q_pitch);
  }
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

sps_status launch_presum_pass(const PresumPassArgs& a, const sps_dedisp_config& c, cudaStream_t st) {
  std::string why;
  if (!presum_config_supported(c, &why)) return fail(SPS_ERR_INVALID_ARG, why);
  PresumKernel fn = find(c.dms_per_thread, c.samples_per_thread / 2);
  const int Di = c.warps_dm * c.dms_per_thread;
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  const size_t smem = presum_smem_bytes(c, a.data_bytes);
  dim3 grid((a.n_dm + Di - 1) / Di, (a.n_out + Tt - 1) / Tt, a.n_groups);
  if (grid.y > 65535 || grid.z > 65535) return fail(SPS_ERR_UNSUPPORTED, "too many time tiles or groups");
  SPS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<grid, 32 * c.warps_dm * c.warps_time, smem, st>>>(a, c.warps_dm, presum_chunk(c),
                                                        presum_window_bytes(c, a.dmax_tile));
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

int64_t presum_pass_blocks(const PresumPassArgs& a, const sps_dedisp_config& c) {
  const int Di = c.warps_dm * c.dms_per_thread;
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  return (int64_t)((a.n_dm + Di - 1) / Di) * ((a.n_out + Tt - 1) / Tt) * a.n_groups;
}

void presum_pass_work(const PresumPassArgs& a, const sps_dedisp_config& c, int32_t pass, std::vector<int4>* work) {
  const int Di = c.warps_dm * c.dms_per_thread;
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  const int tiles = (a.n_dm + Di - 1) / Di, ty = (a.n_out + Tt - 1) / Tt;
  for (int g = 0; g < a.n_groups; g++)
    for (int y = 0; y < ty; y++)
      for (int t = 0; t < tiles; t++) work->push_back(make_int4(pass, t, y, g));
}

sps_status launch_presum_pass_list(const PresumPassArgs* d_passes, const int4* d_work, int64_t n_work,
                                   const sps_dedisp_config& c, int32_t max_data_bytes, cudaStream_t st) {
  std::string why;
  if (!presum_config_supported(c, &why)) return fail(SPS_ERR_INVALID_ARG, why);
  if (n_work < 1 || n_work > 0x7fffffff) return fail(SPS_ERR_UNSUPPORTED, "work list size out of range");
  const Variant* v = find_variant(c.dms_per_thread, c.samples_per_thread / 2);
  const size_t smem = presum_smem_bytes(c, max_data_bytes);
  SPS_CUDA(cudaFuncSetAttribute(v->list, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  v->list<<<(unsigned)n_work, 32 * c.warps_dm * c.warps_time, smem, st>>>(d_passes, d_work, c.warps_dm,
                                                                         presum_chunk(c));
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

}  // namespace sps
