// Subband step two over 16-bit subband series (Sec. 2, first footnote):
//
//   D[i][t] = sum_s Y[k(i)][s][t + d2(i, s)],   t < N_t,
//
// each trial shifting the step-one subband series of its coarse DM with its
// own (full) DM.  A block owns one tile of trials that share a coarse DM, by
// Tt samples, and stages the needed window of each subband series once for
// all trials of the tile.
//
// Step-one sums of <= 257 channels fit 16 bits, so Y is uint16 and a 32-bit
// shared load carries two consecutive samples already in 16-bit lanes: one
// add accumulates two samples.  Two copies of each window (the second shifted
// by one sample) keep every load aligned: copy 0 arrives by bulk asynchronous
// copy (TMA), copy 1 is built from it in shared memory.  Chunks of subbands
// run through two stages: while the block computes one chunk, the next one's
// copies land.  The staged offset of every (trial, subband) of the tile is
// computed once, before the first chunk.  Lanes are folded into int32 every
// `flush_every` subbands, before a 16-bit lane could overflow.
#include <algorithm>

#include "sps_internal.h"
#include "tma.cuh"

namespace sps {
namespace {

constexpr int kMaxThreads = 512;

template <int ND, int NW>
__global__ void __launch_bounds__(kMaxThreads, 1)
step2_kernel(Step2Args a, int wd, int cs_max, int wb) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int Di = wd * ND;
  const int wt = (int)(blockDim.x >> 5) / wd;
  const int Tt = wt * 64 * NW;
  const int S = a.n_subbands;
  const int copy_stride = cs_max * wb;  // one copy of a chunk's windows
  const int stage_bytes = 2 * copy_stride;
  // after the two stages: the offset table [Di][S] and two barriers
  uint32_t* tbl = reinterpret_cast<uint32_t*>(smem + 2 * stage_bytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * stage_bytes + (Di * S * 4 + 15) / 16 * 16);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = (int)(blockDim.x >> 5);
  const int dm_sub = warp % wd, t_sub = warp / wd;
  const int t0 = blockIdx.x * Tt;
  const int k = a.tiles[3 * blockIdx.y], ib = a.tiles[3 * blockIdx.y + 1], nd = a.tiles[3 * blockIdx.y + 2];
  const int n_chunks = (S + cs_max - 1) / cs_max;
  const uint32_t toff = (uint32_t)(t_sub * 128 * NW + lane * 4);  // bytes
  // bounds-checked build: the largest staged offset whose NW words fit the
  // stage's two copies
  const int64_t lim = (int64_t)stage_bytes - (int64_t)(toff + 128 * (NW - 1) + 4);
  const int32_t* d2row0 = a.d2 + (int64_t)ib * S;
  const uint16_t* ybase = a.y + (int64_t)k * S * a.y_pitch;

  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // warp 0: copy 0 of every window of chunk c into its stage, lane sl taking subband sl
  auto issue = [&](int c) {
    const int st = c & 1, sb = c * cs_max, cs = min(cs_max, S - sb);
    uint32_t bytes = 0;
    int64_t start = 0;
    if (lane < cs) {
      start = (int64_t)((t0 + __ldg(&d2row0[sb + lane])) & ~7);
      bytes = (uint32_t)min((int64_t)wb, 2 * (a.y_pitch - start));
    }
    uint32_t total = bytes;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (lane == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&full[st], total);
    }
    __syncwarp();
    if (lane < cs)
      bulk_g2s(smem + st * stage_bytes + lane * wb, ybase + (int64_t)(sb + lane) * a.y_pitch + start, bytes,
               &full[st]);
  };

  uint32_t lanes[ND][NW];
  int32_t acc[ND][NW][2];
#pragma unroll
  for (int r = 0; r < ND; r++)
#pragma unroll
    for (int m = 0; m < NW; m++) { lanes[r][m] = 0u; acc[r][m][0] = 0; acc[r][m][1] = 0; }

  // acc[.][.][0] sums whole lane words (low lanes + 2^16 high lanes, mod 2^32),
  // acc[.][.][1] the high lanes; the low sums are recovered at the end as
  // acc0 - 2^16 acc1 (exact: they stay far below 2^32)
  auto fold = [&]() {
#pragma unroll
    for (int r = 0; r < ND; r++)
#pragma unroll
      for (int m = 0; m < NW; m++) {
        acc[r][m][0] += (int32_t)lanes[r][m];
        acc[r][m][1] += (int32_t)(lanes[r][m] >> 16);
        lanes[r][m] = 0u;
      }
  };

  if (warp == 0) issue(0);
  // while chunk 0 lands: the staged offset of every (trial, subband).  Window
  // start of subband s = the tile's first trial's delay rounded down to 8
  // samples; a trial's offset = its copy (parity of rel), the subband's slot in
  // the chunk, and its even sample offset inside the window.
  for (int e = tid; e < Di * S; e += blockDim.x) {
    const int r = e / S, s = e - r * S;
    const int i = ib + min(r, nd - 1);
    const int start = (t0 + __ldg(&d2row0[s])) & ~7;
    const int rel = t0 + __ldg(&a.d2[(int64_t)i * S + s]) - start;  // elements
    tbl[e] = (uint32_t)((rel & 1) * copy_stride + (s % cs_max) * wb + 2 * (rel & ~1));
  }
  __syncthreads();
  int pending = 0;
  const int wwords = wb >> 2;
  for (int c = 0; c < n_chunks; c++) {
    const int st = c & 1, sb = c * cs_max, cs = min(cs_max, S - sb);
    uint8_t* stage = smem + st * stage_bytes;
    const bool ok = mbar_wait(&full[st], (c >> 1) & 1, a.status);
    if (__syncthreads_or(ok ? 0 : 1)) {
      // this chunk's copies (the only ones issued and not yet waited for) may
      // still be in flight: one more bounded wait before the block leaves
      if (tid == 0) mbar_wait(&full[st], (c >> 1) & 1, nullptr);
      return;
    }
    // copy 1 = copy 0 one sample later; a warp per subband window
    const uint32_t* c0 = reinterpret_cast<const uint32_t*>(stage);
    uint32_t* c1 = reinterpret_cast<uint32_t*>(stage + copy_stride);
    for (int sl = warp; sl < cs; sl += nwarps)
      for (int j = lane; j < wwords; j += 32) {
        const int e = sl * wwords + j;
        c1[e] = __byte_perm(c0[e], j + 1 < wwords ? c0[e + 1] : 0u, 0x5432);
      }
    __syncthreads();  // copy 1 is ready; the other stage's chunk is no longer read
    if (warp == 0 && c + 1 < n_chunks) issue(c + 1);

    const uint32_t* trow = tbl + dm_sub * ND * S + sb;
    for (int sl = 0; sl < cs; sl++) {
#pragma unroll
      for (int r = 0; r < ND; r++) {
        const uint32_t off = trow[r * S + sl];
        if (!stage_read_ok(off, lim, a.status)) continue;
        const uint8_t* p = stage + off + toff;
#pragma unroll
        for (int m = 0; m < NW; m++) lanes[r][m] += *reinterpret_cast<const uint32_t*>(p + 128 * m);
      }
      if (++pending == a.flush_every) { fold(); pending = 0; }
    }
  }
  fold();
#pragma unroll
  for (int r = 0; r < ND; r++)
#pragma unroll
    for (int m = 0; m < NW; m++) acc[r][m][0] = (int32_t)((uint32_t)acc[r][m][0] - ((uint32_t)acc[r][m][1] << 16));

  const bool vec = (a.n_t & 1) == 0;
#pragma unroll
  for (int r = 0; r < ND; r++) {
    const int rr = dm_sub * ND + r;
    if (rr >= nd) continue;
    int32_t* orow = a.D + (int64_t)(ib + rr) * a.n_t;
#pragma unroll
    for (int m = 0; m < NW; m++) {
      const int t = t0 + (int)(toff >> 1) + 64 * m;
      if (t >= a.n_t) continue;
      if (t + 1 < a.n_t && vec) {
        *reinterpret_cast<int2*>(orow + t) = make_int2(acc[r][m][0], acc[r][m][1]);
      } else {
        orow[t] = acc[r][m][0];
        if (t + 1 < a.n_t) orow[t + 1] = acc[r][m][1];
      }
    }
  }
}

typedef void (*Step2Kernel)(Step2Args, int, int, int);

template <int ND, int NW>
constexpr Step2Kernel k() { return step2_kernel<ND, NW>; }

struct Variant { int nd, nw; Step2Kernel fn; };
const Variant kVariants[] = {
    {1, 2, k<1, 2>()}, {1, 4, k<1, 4>()}, {1, 8, k<1, 8>()},
    {2, 2, k<2, 2>()}, {2, 4, k<2, 4>()}, {2, 8, k<2, 8>()},
    {4, 2, k<4, 2>()}, {4, 4, k<4, 4>()}, {4, 8, k<4, 8>()},
    {8, 2, k<8, 2>()}, {8, 4, k<8, 4>()},
};

Step2Kernel find(int nd, int nw) {
  for (const Variant& v : kVariants)
    if (v.nd == nd && v.nw == nw) return v.fn;
  return nullptr;
}

// bytes per staged copy of one subband window (elements rounded up to 8)
int copy_bytes(const sps_dedisp_config& c, int32_t dmax_tile) {
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  return 2 * ((Tt + dmax_tile + 7 + 7) / 8 * 8);
}

}  // namespace

bool step2_config_supported(const sps_dedisp_config& c, std::string* why) {
  if (c.samples_per_thread % 2 || !find(c.dms_per_thread, c.samples_per_thread / 2)) {
    *why = "no compiled step-two variant for this (dms_per_thread, samples_per_thread)";
    return false;
  }
  const int threads = 32 * c.warps_dm * c.warps_time;
  if (c.warps_dm < 1 || c.warps_time < 1 || threads > kMaxThreads) {
    *why = "warps_dm * warps_time must lie in [1, 16]";
    return false;
  }
  if (c.chunk < 1 || c.chunk > 32) {
    *why = "chunk must lie in [1, 32] (one issuing lane per subband of a chunk)";
    return false;
  }
  return true;
}

size_t step2_smem_bytes(const sps_dedisp_config& c, int32_t dmax_tile, int32_t n_subbands) {
  const size_t Di = (size_t)c.warps_dm * c.dms_per_thread;
  const size_t stage = 2 * (size_t)c.chunk * copy_bytes(c, dmax_tile);
  // two stages, the offset table and the barriers
  return 2 * stage + (Di * n_subbands * 4 + 15) / 16 * 16 + 16;
}

sps_status launch_step2(const Step2Args& a, const sps_dedisp_config& c, cudaStream_t st) {
  std::string why;
  if (!step2_config_supported(c, &why)) return fail(SPS_ERR_INVALID_ARG, why);
  Step2Kernel fn = find(c.dms_per_thread, c.samples_per_thread / 2);
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  const size_t smem = step2_smem_bytes(c, a.dmax_tile, a.n_subbands);
  dim3 grid((a.n_t + Tt - 1) / Tt, a.n_tiles, 1);
  if (grid.y > 65535) return fail(SPS_ERR_UNSUPPORTED, "too many step-two tiles");
  SPS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<grid, 32 * c.warps_dm * c.warps_time, smem, st>>>(a, c.warps_dm, c.chunk, copy_bytes(c, a.dmax_tile));
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

}  // namespace sps
