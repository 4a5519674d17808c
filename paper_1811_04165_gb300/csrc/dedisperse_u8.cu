// Brute-force de-dispersion and subband step one over uint8 channels.
//
//   out[i * G + g][t] = sum_{c in group g} x[c][t + d(i, c)]
//
// (Sec. 1: shift and integrate channels; Sec. 2, first footnote: step one sums
// the channels of each subband at the coarse DMs.)  Brute force is G = 1 over
// all channels.
//
// Design for sm_103a.  The work is integer shift-and-add, bound by shared
// memory wavefronts and integer issue, not by HBM (about 300 adds per input
// byte at 1536 channels), so there are no tensor cores here.
//   * A block owns Di = warps_dm * ND DM trials by Tt = warps_time * 128 * NW
//     samples and walks its channels `chunk` at a time.  For each channel the
//     window [t0 + d(i0, c), t0 + Tt + d(i_last, c)) is staged once and read by
//     all Di trials.
//   * Four copies of each window are staged, copy j shifted by j bytes, so that
//     every 4-sample read is one aligned, conflict-free 32-bit shared load
//     whatever the delay's alignment.  A pre-pass (expand_kernel) writes the
//     shifted copies 1..3 of the whole batch once; all four copies and the
//     chunk's shared-memory offset table arrive by bulk asynchronous copies
//     (TMA) into a two-stage ring guarded by mbarriers, so the warps only add.
//   * SWAR: the words of 4 samples are summed whole (one three-input add per
//     two channels), and their odd bytes, moved into 16-bit lanes by one byte
//     permute, are summed apart with integer multiply-adds by 1 on the FMA
//     pipe (the integer ALU pipe, 64 lanes per SM, would otherwise saturate).
//     With sums b_k of byte k over <= 257 channels of 255, both below 2^16,
//       raw = b0 + 2^8 b1 + 2^16 b2 + 2^24 b3,   odd = b1 + 2^16 b3,
//       raw - (odd << 8) = b0 + 2^16 b2   (mod 2^32),
//     so the even bytes' 16-bit lanes come back exactly; partial sums are
//     folded into int32 registers every <= 256 channels.
//   * Shared loads use 32-bit shared-window addresses with immediate offsets.
//   * The offset of (trial, channel) inside the staged windows does not depend
//     on the time tile (tiles start at multiples of 128), so the plan
//     precomputes it once per configuration.
//   * In subband step one a block may walk several groups (subbands) as one
//     stream of chunks, storing each group's sums while the next chunks land.
#include <algorithm>

#include "sps_internal.h"
#include "tma.cuh"

namespace sps {
namespace {

constexpr int kMaxThreads = 512;

__device__ __forceinline__ uint32_t odd_bytes(uint32_t w) { return __byte_perm(w, 0u, 0x4341); }

// c + a * one with one == 1 known only at run time: an integer multiply-add on
// the FMA pipe instead of an add on the integer ALU pipe.
__device__ __forceinline__ uint32_t madd(uint32_t a, uint32_t one, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(one), "r"(c));
  return d;
}

// NW words at shared address addr + 128 * m, m < NW (immediate offsets).
template <int NW, int M = 0>
__device__ __forceinline__ void lds_row(uint32_t addr, uint32_t (&w)[NW]) {
  if constexpr (M < NW) {
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(w[M]) : "r"(addr), "n"(M * 128));
    lds_row<NW, M + 1>(addr, w);
  }
}

// WALK: the block walks gpb > 1 groups in turn (subband step one); without it
// the block has one group, compiled as a plain loop over its chunks.
template <int ND, int NW, bool WALK>
__global__ void __launch_bounds__(kMaxThreads, 1)
u8_pass_kernel(U8PassArgs a, int wd, int cc_max, int wb, int gpb) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int wt = (int)(blockDim.x >> 5) / wd;
  const int Tt = wt * 128 * NW;
  const int Di = wd * ND;
  const int copy_stride = cc_max * wb;
  const int stage_bytes = 4 * copy_stride + cc_max * a.di_pad * 4;
  int32_t* b0s = reinterpret_cast<int32_t*>(smem + 2 * stage_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * stage_bytes + ((gpb * a.group_channels * 4 + 15) & ~15));
  __shared__ int aborted;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int dm_sub = warp % wd, t_sub = warp / wd;
  const int tile = blockIdx.x;
  const int i0 = tile * Di;
  const int t0 = blockIdx.y * Tt;
  // the block's groups g0 .. g0 + ng - 1, walked as one stream of chunks so
  // that the stage ring keeps running from one group into the next
  const int g0 = blockIdx.z * gpb;
  const int ng = min(gpb, a.n_groups - g0);
  const int G = a.group_channels;
  const int c_lo = g0 * G;
  const int chunks_g = (G + cc_max - 1) / cc_max;  // chunks per group
  const int n_chunks = ng * chunks_g;
  const int pairs = (G + 1) >> 1;
  const uint32_t toff = (uint32_t)(t_sub * 128 * NW + lane * 4);
  // bounds-checked build: the largest staged offset whose NW words fit the four
  // copies of the stage, and the warp's trials inside a row of the offset table
  const int64_t lim = (int64_t)4 * copy_stride - (int64_t)(toff + 128 * (NW - 1) + 4);
  if (kBoundsCheck && (dm_sub + 1) * ND > a.di_pad) stage_read_ok(1u, -1, a.status);
  const uint32_t one = a.one;

  for (int c = tid; c < ng * G; c += blockDim.x) b0s[c] = a.b0[(int64_t)tile * a.channels + c_lo + c];
  if (tid == 0) {
    aborted = 0;
    mbar_init(&bars[0], blockDim.x >> 5);
    mbar_init(&bars[1], blockDim.x >> 5);
    fence_mbar_init();
  }
  __syncthreads();

  // Every warp stages its share of chunk `ch` (channels warp, warp + nwarps,
  // ...) into stage ch & 1: the four shifted copies of each channel window;
  // warp 0 also copies the chunk's offset table.  Each warp's lane 0 arrives
  // on the stage barrier with the bytes its warp issued.  Chunk ch is chunk
  // ch % chunks_g of the block's group ch / chunks_g; cb is its first channel
  // inside the block's channel range.
  const int nwarps = (int)(blockDim.x >> 5);
  auto issue = [&](int ch) {
    const int st = ch & 1;
    uint8_t* sb = smem + st * stage_bytes;
    const int gi = WALK ? ch / chunks_g : 0, cg = WALK ? ch - gi * chunks_g : ch;
    const int cb = gi * G + cg * cc_max, cc = min(cc_max, G - cg * cc_max);
    const int npair = (cc + 1) >> 1;
    const uint32_t tbl_bytes = (uint32_t)(npair * a.di_pad * 8);
    // lanes 4q..4q+3 of a warp handle copies 0..3 of channels warp + (q + 8k) * nwarps
    const int q = lane >> 2, j = lane & 3;
    uint32_t mine = 0;
    for (int l = warp + q * nwarps; l < cc; l += 8 * nwarps)
      mine += (uint32_t)min(wb, a.win_limit - (t0 + b0s[cb + l]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if (lane == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&bars[st], mine + (warp == 0 ? tbl_bytes : 0u));
    }
    __syncwarp();
    for (int l = warp + q * nwarps; l < cc; l += 8 * nwarps) {
      const int c = c_lo + cb + l;
      const int start = t0 + b0s[cb + l];
      const uint32_t bytes = (uint32_t)min(wb, a.win_limit - start);
      const uint8_t* src = j == 0 ? a.x + (int64_t)c * a.pitch + start
                                  : a.x4 + ((int64_t)(j - 1) * a.channels + c) * a.pitch4 + start;
      bulk_g2s(sb + j * copy_stride + l * wb, src, bytes, &bars[st]);
    }
    if (warp == 0 && lane == 0) {
      const uint32_t* src =
          a.offs + (((int64_t)tile * a.n_groups + g0 + gi) * pairs + ((cg * cc_max) >> 1)) * a.di_pad * 2;
      bulk_g2s(sb + 4 * copy_stride, src, tbl_bytes, &bars[st]);
    }
  };

  uint32_t raw[ND][NW], hi[ND][NW];  // whole-word sums; odd bytes in 16-bit lanes
  int32_t acc[ND][NW][4];
#pragma unroll
  for (int r = 0; r < ND; r++)
#pragma unroll
    for (int m = 0; m < NW; m++) {
      raw[r][m] = 0u; hi[r][m] = 0u;
#pragma unroll
      for (int q = 0; q < 4; q++) acc[r][m][q] = 0;
    }
  auto fold = [&]() {
#pragma unroll
    for (int r = 0; r < ND; r++)
#pragma unroll
      for (int m = 0; m < NW; m++) {
        const uint32_t lo = raw[r][m] - (hi[r][m] << 8);  // even bytes in 16-bit lanes
        // whole lane words (low + 2^16 high, mod 2^32) and the high lanes; the
        // low sums are recovered after the last fold as word sum - 2^16 high sum
        acc[r][m][0] += (int32_t)lo;
        acc[r][m][2] += (int32_t)(lo >> 16);
        acc[r][m][1] += (int32_t)hi[r][m];
        acc[r][m][3] += (int32_t)(hi[r][m] >> 16);
        raw[r][m] = 0u; hi[r][m] = 0u;
      }
  };

  // A group's sums: the last fold, the low lanes recovered, the rows stored
  // (each lane holds 4 consecutive samples per (trial, word)), the registers
  // cleared for the block's next group.
  const bool vec = (a.out_pitch & 3) == 0;
  auto finish_group = [&](int g) {
    fold();
#pragma unroll
    for (int r = 0; r < ND; r++)
#pragma unroll
      for (int m = 0; m < NW; m++) {
        acc[r][m][0] = (int32_t)((uint32_t)acc[r][m][0] - ((uint32_t)acc[r][m][2] << 16));
        acc[r][m][1] = (int32_t)((uint32_t)acc[r][m][1] - ((uint32_t)acc[r][m][3] << 16));
      }
#pragma unroll
    for (int r = 0; r < ND; r++) {
      const int i = i0 + dm_sub * ND + r;
      if (i >= a.n_dm) continue;
      const int64_t row = (int64_t)i * a.n_groups + g;
#pragma unroll
      for (int m = 0; m < NW; m++) {
        const int t = t0 + (int)toff + 128 * m;
        if (t >= a.n_out) continue;
        if (a.out_u16) {
          uint16_t* o = static_cast<uint16_t*>(a.out) + row * a.out_pitch + t;
          if (t + 3 < a.n_out && vec) {
            uint2 v;
            v.x = (uint32_t)acc[r][m][0] | ((uint32_t)acc[r][m][1] << 16);
            v.y = (uint32_t)acc[r][m][2] | ((uint32_t)acc[r][m][3] << 16);
            *reinterpret_cast<uint2*>(o) = v;
          } else {
            for (int q = 0; q < 4 && t + q < a.n_out; q++) o[q] = (uint16_t)acc[r][m][q];
          }
        } else {
          int32_t* o = static_cast<int32_t*>(a.out) + row * a.out_pitch + t;
          if (t + 3 < a.n_out && vec) {
            *reinterpret_cast<int4*>(o) = make_int4(acc[r][m][0], acc[r][m][1], acc[r][m][2], acc[r][m][3]);
          } else {
            for (int q = 0; q < 4 && t + q < a.n_out; q++) o[q] = acc[r][m][q];
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < ND; r++)
#pragma unroll
      for (int m = 0; m < NW; m++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[r][m][q] = 0;
  };

  issue(0);
  if (n_chunks > 1) issue(1);

  int pending = 0;
  int ch = 0;
  int gi = 0, cg = 0;  // group and chunk inside it of chunk ch (WALK)
  for (; ch < n_chunks; ch++) {
    const int st = ch & 1;
    const int cc = min(cc_max, G - (WALK ? cg : ch) * cc_max);
    if (pending + cc > 256) { fold(); pending = 0; }
    if (!mbar_wait(&bars[st], (ch >> 1) & 1, a.status)) aborted = 1;
    if (!aborted) {
      const uint32_t base = smem_u32(smem) + (uint32_t)(st * stage_bytes) + toff;
      const uint2* tb = reinterpret_cast<const uint2*>(smem + st * stage_bytes + 4 * copy_stride) + dm_sub * ND;
      int cl = 0;
      for (; cl + 1 < cc; cl += 2) {
        const uint2* e = tb + (cl >> 1) * a.di_pad;
#pragma unroll
        for (int r = 0; r < ND; r++) {
          const uint2 o = e[r];
          uint32_t W1[NW] = {}, W2[NW] = {};
          if (stage_read_ok(o.x, lim, a.status)) lds_row<NW>(base + o.x, W1);
          if (stage_read_ok(o.y, lim, a.status)) lds_row<NW>(base + o.y, W2);
#pragma unroll
          for (int m = 0; m < NW; m++) {
            raw[r][m] += W1[m] + W2[m];
            hi[r][m] = madd(odd_bytes(W2[m]), one, madd(odd_bytes(W1[m]), one, hi[r][m]));
          }
        }
      }
      if (cl < cc) {
        const uint2* e = tb + (cl >> 1) * a.di_pad;
#pragma unroll
        for (int r = 0; r < ND; r++) {
          uint32_t W1[NW] = {};
          if (stage_read_ok(e[r].x, lim, a.status)) lds_row<NW>(base + e[r].x, W1);
#pragma unroll
          for (int m = 0; m < NW; m++) {
            raw[r][m] += W1[m];
            hi[r][m] = madd(odd_bytes(W1[m]), one, hi[r][m]);
          }
        }
      }
    }
    pending += cc;
    __syncthreads();
    if (aborted) break;
    if (ch + 2 < n_chunks) issue(ch + 2);
    if constexpr (WALK) {
      if (++cg == chunks_g) {
        // the group's last chunk: its sums go out while the next chunks land
        finish_group(g0 + gi);
        pending = 0;
        cg = 0;
        gi++;
      }
    }
  }
  if (aborted) {
    // let copies already in flight land before the block's shared memory goes away
    if (tid == 0)
      for (int k = ch; k < min(ch + 2, n_chunks); k++) mbar_wait(&bars[k & 1], (k >> 1) & 1, a.status);
    return;
  }
  if constexpr (!WALK) finish_group(g0);
}

// Bytes [p, p + 20) of a channel row, zero at and beyond `len`.
__device__ __forceinline__ void load_raw20(const uint8_t* row, int64_t p, int32_t len, uint32_t r[5]) {
  if (p + 20 <= len) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(row + p));
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    r[4] = __ldg(reinterpret_cast<const uint32_t*>(row + p + 16));
  } else {
#pragma unroll
    for (int k = 0; k < 5; k++) {
      uint32_t w = 0;
#pragma unroll
      for (int b = 0; b < 4; b++) {
        int64_t q = p + 4 * k + b;
        uint32_t v = q < len ? (uint32_t)__ldg(row + q) : 0u;
        w |= v << (8 * b);
      }
      r[k] = w;
    }
  }
}

// x4[j - 1][c][p] = x[c][p + j] for j = 1..3 (0 at and beyond in_len).
__global__ void __launch_bounds__(256) expand_kernel(const uint8_t* x, int64_t pitch, int32_t in_len,
                                                     int32_t channels, uint8_t* x4, int64_t pitch4) {
  const int64_t spr = pitch4 >> 4;
  const int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (seg >= spr * channels) return;
  const int64_t c = seg / spr, p = (seg - c * spr) << 4;
  uint32_t r[5];
  load_raw20(x + c * pitch, p, in_len, r);
  const int64_t plane = (int64_t)channels * pitch4;
  uint8_t* dst = x4 + c * pitch4 + p;
  *reinterpret_cast<uint4*>(dst) =
      make_uint4(__byte_perm(r[0], r[1], 0x4321), __byte_perm(r[1], r[2], 0x4321),
                 __byte_perm(r[2], r[3], 0x4321), __byte_perm(r[3], r[4], 0x4321));
  *reinterpret_cast<uint4*>(dst + plane) =
      make_uint4(__byte_perm(r[0], r[1], 0x5432), __byte_perm(r[1], r[2], 0x5432),
                 __byte_perm(r[2], r[3], 0x5432), __byte_perm(r[3], r[4], 0x5432));
  *reinterpret_cast<uint4*>(dst + 2 * plane) =
      make_uint4(__byte_perm(r[0], r[1], 0x6543), __byte_perm(r[1], r[2], 0x6543),
                 __byte_perm(r[2], r[3], 0x6543), __byte_perm(r[3], r[4], 0x6543));
}

typedef void (*U8Kernel)(U8PassArgs, int, int, int, int);

template <int ND, int NW>
constexpr U8Kernel k() { return u8_pass_kernel<ND, NW, false>; }
template <int ND, int NW>
constexpr U8Kernel kw() { return u8_pass_kernel<ND, NW, true>; }

struct Variant { int nd, nw; U8Kernel fn, walk; };
const Variant kVariants[] = {
    {1, 1, k<1, 1>(), kw<1, 1>()}, {1, 2, k<1, 2>(), kw<1, 2>()}, {1, 4, k<1, 4>(), kw<1, 4>()},
    {1, 8, k<1, 8>(), kw<1, 8>()}, {2, 1, k<2, 1>(), kw<2, 1>()}, {2, 2, k<2, 2>(), kw<2, 2>()},
    {2, 4, k<2, 4>(), kw<2, 4>()}, {2, 8, k<2, 8>(), kw<2, 8>()}, {4, 1, k<4, 1>(), kw<4, 1>()},
    {4, 2, k<4, 2>(), kw<4, 2>()}, {4, 4, k<4, 4>(), kw<4, 4>()}, {8, 1, k<8, 1>(), kw<8, 1>()},
    {8, 2, k<8, 2>(), kw<8, 2>()},
};

U8Kernel find(int nd, int nw, bool walk = false) {
  for (const Variant& v : kVariants)
    if (v.nd == nd && v.nw == nw) return walk ? v.walk : v.fn;
  return nullptr;
}

}  // namespace

int u8_window_bytes(const sps_dedisp_config& c, int32_t dmax_tile) {
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  return (Tt + dmax_tile + 15 + 15) / 16 * 16;
}

int u8_di_pad(const sps_dedisp_config& c) { return (c.warps_dm * c.dms_per_thread + 1) / 2 * 2; }

bool u8_config_supported(const sps_dedisp_config& c, std::string* why) {
  if (c.samples_per_thread % 4 || !find(c.dms_per_thread, c.samples_per_thread / 4)) {
    *why = "no compiled variant for this (dms_per_thread, samples_per_thread)";
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

// Groups one block walks in turn.  In subband step one a block that walks
// several subbands keeps its stage ring running from one into the next instead
// of filling it anew (measured on the beam's 32 subbands, batches streamed on
// two streams: 0.249 ms per two-step search with one group per block, 0.238
// with four); up to four, while the grid keeps at least 512 blocks (here
// `tiles` = DM tiles x time tiles).  Brute force has one group.
int u8_groups_per_block(int32_t n_groups, int64_t tiles) {
  int g = 1;
  while (g < 4 && 2 * g <= n_groups && tiles * ((n_groups + 2 * g - 1) / (2 * g)) >= 512) g *= 2;
  return g;
}

size_t u8_smem_bytes(const sps_dedisp_config& c, int32_t dmax_tile, int32_t group_channels, int32_t n_groups) {
  const size_t stage = 4 * (size_t)c.chunk * u8_window_bytes(c, dmax_tile) + (size_t)c.chunk * u8_di_pad(c) * 4;
  // room for the channel window starts of the most groups a block may walk
  const size_t b0 = (size_t)std::min<int32_t>(4, std::max<int32_t>(1, n_groups)) * group_channels;
  return 2 * stage + ((b0 * 4 + 15) & ~(size_t)15) + 16;
}

sps_status launch_expand(const uint8_t* x, int64_t pitch, int32_t in_len, int32_t channels, uint8_t* x4,
                         int64_t pitch4, cudaStream_t st) {
  const int64_t segs = (pitch4 >> 4) * channels;
  expand_kernel<<<(unsigned)((segs + 255) / 256), 256, 0, st>>>(x, pitch, in_len, channels, x4, pitch4);
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

sps_status launch_u8_pass(const U8PassArgs& a, const sps_dedisp_config& c, cudaStream_t st) {
  std::string why;
  if (!u8_config_supported(c, &why)) return fail(SPS_ERR_INVALID_ARG, why);
  const int Di = c.warps_dm * c.dms_per_thread;
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  const size_t smem = u8_smem_bytes(c, a.dmax_tile, a.group_channels, a.n_groups);
  const int64_t tiles = (int64_t)((a.n_dm + Di - 1) / Di) * ((a.n_out + Tt - 1) / Tt);
  const int gpb = u8_groups_per_block(a.n_groups, tiles);
  U8Kernel fn = find(c.dms_per_thread, c.samples_per_thread / 4, gpb > 1);
  dim3 grid((a.n_dm + Di - 1) / Di, (a.n_out + Tt - 1) / Tt, (a.n_groups + gpb - 1) / gpb);
  if (grid.y > 65535 || grid.z > 65535) return fail(SPS_ERR_UNSUPPORTED, "too many time tiles or groups");
  SPS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<grid, 32 * c.warps_dm * c.warps_time, smem, st>>>(a, c.warps_dm, c.chunk, u8_window_bytes(c, a.dmax_tile),
                                                          gpb);
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

}  // namespace sps
