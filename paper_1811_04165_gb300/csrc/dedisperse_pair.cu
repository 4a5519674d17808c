// De-dispersion over pre-summed adjacent-channel pairs (brute force, or
// subband step one), exactly:
//
//   out[i * G + g][t] = sum_{c in group g} x[c][t + d(i, c)]
//                     = sum_{pairs (a, b)} Q_delta[t + d(i, b)],
//   Q_delta[u] = x[a][u + delta] + x[b][u],   delta = d(i, a) - d(i, b) >= 0.
//
// (Sec. 1: shift and integrate channels; Sec. 2, first footnote: step one.)
// Adjacent channels have nearly equal delays, so for a tile of consecutive
// trials each pair needs only one or two values of delta.  A pre-pass writes,
// for every pair and every delta its trials need, the series Q_delta as uint16
// (two copies, the second shifted by one sample, so every 32-bit shared load
// is aligned); the block then stages, per chunk of pairs, just the series its
// tile uses (a host-built slot list) with bulk asynchronous copies (TMA) into a
// two-stage mbarrier ring.  A 32-bit load holds two samples of a pair sum in
// 16-bit lanes: one add accumulates four channel-samples, with no unpacking.
// Pair sums are <= 510, so 16-bit lanes are exact for 128 pairs; partial sums
// fold into int32 registers every <= 128 pairs (256 channels).  An unpaired last
// channel of a group is a pair with an empty partner (delta 0).
#include <algorithm>

#include "sps_internal.h"
#include "tma.cuh"

namespace sps {
namespace {

constexpr int kMaxThreads = 512;

// NW words at shared address addr + 128 * m (immediate offsets).
template <int NW, int M = 0>
__device__ __forceinline__ void lds_row(uint32_t addr, uint32_t (&w)[NW]) {
  if constexpr (M < NW) {
    asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(w[M]) : "r"(addr), "n"(M * 128));
    lds_row<NW, M + 1>(addr, w);
  }
}

template <int ND, int NW>
__global__ void __launch_bounds__(kMaxThreads, 1)
pair_pass_kernel(PairPassArgs a, int wd, int cp_max, int wb, int slots_max) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int wt = (int)(blockDim.x >> 5) / wd;
  const int Tt = wt * 64 * NW;
  const int Di = wd * ND;
  const int stage_bytes = slots_max * 2 * wb + cp_max * a.di_pad * 4;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * stage_bytes);
  __shared__ int aborted;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = (int)(blockDim.x >> 5);
  const int dm_sub = warp % wd, t_sub = warp / wd;
  const int tile = blockIdx.x;
  const int i0 = tile * Di;
  const int t0 = blockIdx.y * Tt;
  const int g = blockIdx.z;
  const int P = a.group_pairs;
  const int n_chunks = (P + cp_max - 1) / cp_max;
  const uint32_t toff = (uint32_t)(t_sub * 128 * NW + lane * 4);  // bytes
  const int64_t chunk_row = ((int64_t)tile * a.n_groups + g) * n_chunks;

  if (tid == 0) {
    aborted = 0;
    mbar_init(&bars[0], nwarps);
    mbar_init(&bars[1], nwarps);
    fence_mbar_init();
  }
  __syncthreads();

  // Every warp stages its share of chunk `ch`: the slot list of the chunk names
  // the series (and window start) of each slot; copy j of slot k lands at
  // (2k + j) * wb.  Warp 0 also copies the chunk's offset table.
  auto issue = [&](int ch) {
    const int st = ch & 1;
    uint8_t* sb = smem + st * stage_bytes;
    const int pb = ch * cp_max, cp = min(cp_max, P - pb);
    const int2* list = a.slots + (chunk_row + ch) * (slots_max + 1);
    const int n_slots = __ldg(&list[slots_max].x);
    const uint32_t tbl_bytes = (uint32_t)(cp * a.di_pad * 4);
    uint32_t mine = 0;
    for (int q = warp * 32 + lane; q < 2 * n_slots; q += 32 * nwarps) {
      const int start = t0 + __ldg(&list[q >> 1].y);
      mine += (uint32_t)min(wb, 2 * (a.q_pitch - start));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if (lane == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(&bars[st], mine + (warp == 0 ? tbl_bytes : 0u));
    }
    __syncwarp();
    for (int q = warp * 32 + lane; q < 2 * n_slots; q += 32 * nwarps) {
      const int2 e = __ldg(&list[q >> 1]);
      const int start = t0 + e.y;
      const uint32_t bytes = (uint32_t)min(wb, 2 * (a.q_pitch - start));
      const uint16_t* src = a.q + ((int64_t)e.x * 2 + (q & 1)) * a.q_pitch + start;
      bulk_g2s(sb + q * wb, src, bytes, &bars[st]);
    }
    if (warp == 0 && lane == 0) {
      const uint32_t* src = a.offs + (((int64_t)tile * a.n_groups + g) * P + pb) * a.di_pad;
      bulk_g2s(sb + slots_max * 2 * wb, src, tbl_bytes, &bars[st]);
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

  issue(0);
  if (n_chunks > 1) issue(1);

  int pending = 0;
  int ch = 0;
  for (; ch < n_chunks; ch++) {
    const int st = ch & 1;
    const int cp = min(cp_max, P - ch * cp_max);
    if (pending + cp > 128) { fold(); pending = 0; }
    if (!mbar_wait(&bars[st], (ch >> 1) & 1, a.status)) aborted = 1;
    if (!aborted) {
      const uint32_t base = smem_u32(smem) + (uint32_t)(st * stage_bytes) + toff;
      const uint32_t* tb =
          reinterpret_cast<const uint32_t*>(smem + st * stage_bytes + slots_max * 2 * wb) + dm_sub * ND;
      int p = 0;
      for (; p + 1 < cp; p += 2) {
        const uint32_t* e0 = tb + p * a.di_pad;
        const uint32_t* e1 = e0 + a.di_pad;
#pragma unroll
        for (int r = 0; r < ND; r++) {
          uint32_t A[NW], B[NW];
          lds_row<NW>(base + e0[r], A);
          lds_row<NW>(base + e1[r], B);
#pragma unroll
          for (int m = 0; m < NW; m++) lanes[r][m] += A[m] + B[m];
        }
      }
      if (p < cp) {
        const uint32_t* e0 = tb + p * a.di_pad;
#pragma unroll
        for (int r = 0; r < ND; r++) {
          uint32_t A[NW];
          lds_row<NW>(base + e0[r], A);
#pragma unroll
          for (int m = 0; m < NW; m++) lanes[r][m] += A[m];
        }
      }
    }
    pending += cp;
    __syncthreads();
    if (aborted) break;
    if (ch + 2 < n_chunks) issue(ch + 2);
  }
  if (aborted) {
    if (tid == 0)
      for (int k = ch; k < min(ch + 2, n_chunks); k++) mbar_wait(&bars[k & 1], (k >> 1) & 1, a.status);
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

// Series s, copy j: q[(2 s + j) * q_pitch + u] = x[a][u + j + delta] + x[b][u + j]
// (b < 0: no partner), bytes at and beyond in_len read as 0.  One thread writes
// 8 samples (16 bytes).
__global__ void __launch_bounds__(256) pair_series_kernel(const uint8_t* x, int64_t pitch, int32_t in_len,
                                                          const int4* series, int32_t n_series, uint16_t* q,
                                                          int32_t q_pitch) {
  const int64_t per_row = q_pitch >> 3;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= per_row * 2 * n_series) return;
  const int64_t row = id / per_row;  // 2 s + j
  const int u0 = (int)(id - row * per_row) << 3;
  const int s = (int)(row >> 1), j = (int)(row & 1);
  const int4 e = __ldg(&series[s]);  // {a, b, delta, -}
  const uint8_t* xa = x + (int64_t)e.x * pitch;
  const uint8_t* xb = e.y >= 0 ? x + (int64_t)e.y * pitch : nullptr;
  uint32_t v[8];
#pragma unroll
  for (int k = 0; k < 8; k++) {
    const int ua = u0 + k + j + e.z, ub = u0 + k + j;
    uint32_t s0 = ua < in_len ? (uint32_t)__ldg(xa + ua) : 0u;
    if (xb && ub < in_len) s0 += (uint32_t)__ldg(xb + ub);
    v[k] = s0;
  }
  uint4 out = make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16), v[6] | (v[7] << 16));
  *reinterpret_cast<uint4*>(q + row * q_pitch + u0) = out;
}

typedef void (*PairKernel)(PairPassArgs, int, int, int, int);

template <int ND, int NW>
constexpr PairKernel k() { return pair_pass_kernel<ND, NW>; }

struct Variant { int nd, nw; PairKernel fn; };
const Variant kVariants[] = {
    {1, 2, k<1, 2>()}, {1, 4, k<1, 4>()}, {1, 8, k<1, 8>()}, {1, 16, k<1, 16>()},
    {2, 2, k<2, 2>()}, {2, 4, k<2, 4>()}, {2, 8, k<2, 8>()}, {2, 16, k<2, 16>()},
    {4, 2, k<4, 2>()}, {4, 4, k<4, 4>()}, {4, 8, k<4, 8>()},
    {8, 2, k<8, 2>()}, {8, 4, k<8, 4>()},
};

PairKernel find(int nd, int nw) {
  for (const Variant& v : kVariants)
    if (v.nd == nd && v.nw == nw) return v.fn;
  return nullptr;
}

}  // namespace

int pair_window_bytes(const sps_dedisp_config& c, int32_t dmax_tile) {
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  return 2 * ((Tt + dmax_tile + 7 + 7) / 8 * 8);
}

int pair_di_pad(const sps_dedisp_config& c) { return (c.warps_dm * c.dms_per_thread + 3) / 4 * 4; }

int pair_chunk(const sps_dedisp_config& c) { return std::max(1, c.chunk / 2); }

bool pair_config_supported(const sps_dedisp_config& c, std::string* why) {
  if (c.samples_per_thread % 2 || !find(c.dms_per_thread, c.samples_per_thread / 2)) {
    *why = "no compiled pair variant for this (dms_per_thread, samples_per_thread)";
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

size_t pair_smem_bytes(const sps_dedisp_config& c, int32_t dmax_tile, int32_t slots_max) {
  const size_t stage = (size_t)slots_max * 2 * pair_window_bytes(c, dmax_tile) +
                       (size_t)pair_chunk(c) * pair_di_pad(c) * 4;
  return 2 * stage + 16;
}

sps_status launch_pair_series(const uint8_t* x, int64_t pitch, int32_t in_len, const int4* series,
                              int32_t n_series, uint16_t* q, int32_t q_pitch, cudaStream_t st) {
  const int64_t threads = (int64_t)(q_pitch >> 3) * 2 * n_series;
  pair_series_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(x, pitch, in_len, series, n_series, q,
                                                                         q_pitch);
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

sps_status launch_pair_pass(const PairPassArgs& a, const sps_dedisp_config& c, cudaStream_t st) {
  std::string why;
  if (!pair_config_supported(c, &why)) return fail(SPS_ERR_INVALID_ARG, why);
  PairKernel fn = find(c.dms_per_thread, c.samples_per_thread / 2);
  const int Di = c.warps_dm * c.dms_per_thread;
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  const size_t smem = pair_smem_bytes(c, a.dmax_tile, a.slots_max);
  dim3 grid((a.n_dm + Di - 1) / Di, (a.n_out + Tt - 1) / Tt, a.n_groups);
  if (grid.y > 65535 || grid.z > 65535) return fail(SPS_ERR_UNSUPPORTED, "too many time tiles or groups");
  SPS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<grid, 32 * c.warps_dm * c.warps_time, smem, st>>>(a, c.warps_dm, pair_chunk(c),
                                                        pair_window_bytes(c, a.dmax_tile), a.slots_max);
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

}  // namespace sps
