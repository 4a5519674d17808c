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
// by one sample) keep every load aligned.  Lanes are folded into int32 every
// `flush_every` subbands, before a 16-bit lane could overflow.
#include <algorithm>

#include "sps_internal.h"

namespace sps {
namespace {

constexpr int kMaxThreads = 512;

// Elements [p, p + 10) of a Y row, zero at and beyond `len`.
__device__ __forceinline__ void load_y10(const uint16_t* row, int64_t p, int32_t len, uint32_t r[5]) {
  if (p + 10 <= len) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(row + p));
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    r[4] = __ldg(reinterpret_cast<const uint32_t*>(row + p + 8));
  } else {
#pragma unroll
    for (int k = 0; k < 5; k++) {
      int64_t q = p + 2 * k;
      uint32_t e0 = q < len ? (uint32_t)__ldg(row + q) : 0u;
      uint32_t e1 = q + 1 < len ? (uint32_t)__ldg(row + q + 1) : 0u;
      r[k] = e0 | (e1 << 16);
    }
  }
}

template <int ND, int NW>
__global__ void __launch_bounds__(kMaxThreads, 1)
step2_kernel(Step2Args a, int wd, int cs_max, int wb) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int Di = wd * ND;
  const int wt = (int)(blockDim.x >> 5) / wd;
  const int Tt = wt * 64 * NW;
  const int copy_stride = cs_max * wb;
  uint32_t* tbl = reinterpret_cast<uint32_t*>(smem + 2 * copy_stride);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int dm_sub = warp % wd, t_sub = warp / wd;
  const int t0 = blockIdx.x * Tt;
  const int k = a.tiles[3 * blockIdx.y], ib = a.tiles[3 * blockIdx.y + 1], nd = a.tiles[3 * blockIdx.y + 2];
  const int S = a.n_subbands;
  const uint32_t toff = (uint32_t)(t_sub * 128 * NW + lane * 4);  // bytes
  const int32_t* d2row0 = a.d2 + (int64_t)ib * S;
  const uint16_t* ybase = a.y + (int64_t)k * S * a.y_pitch;

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

  int pending = 0;
  const int segs = wb >> 4;
  for (int sb = 0; sb < S; sb += cs_max) {
    const int cs = min(cs_max, S - sb);
    __syncthreads();
    for (int e = tid; e < cs * segs; e += blockDim.x) {
      const int sl = e / segs, q = e - sl * segs;
      const int s = sb + sl;
      const int64_t start = (int64_t)((t0 + d2row0[s]) & ~7);
      uint32_t r[5];
      load_y10(ybase + (int64_t)s * a.y_pitch, start + 8 * q, a.y_len, r);
      uint8_t* dst = smem + sl * wb + 16 * q;
      *reinterpret_cast<uint4*>(dst) = make_uint4(r[0], r[1], r[2], r[3]);
      *reinterpret_cast<uint4*>(dst + copy_stride) =
          make_uint4(__byte_perm(r[0], r[1], 0x5432), __byte_perm(r[1], r[2], 0x5432),
                     __byte_perm(r[2], r[3], 0x5432), __byte_perm(r[3], r[4], 0x5432));
    }
    for (int e = tid; e < Di * cs; e += blockDim.x) {
      const int r = e / cs, sl = e - r * cs;
      const int i = ib + min(r, nd - 1);
      const int s = sb + sl;
      const int start = (t0 + d2row0[s]) & ~7;
      const int rel = t0 + a.d2[(int64_t)i * S + s] - start;  // elements
      tbl[r * cs_max + sl] = (uint32_t)((rel & 1) * copy_stride + sl * wb + 2 * (rel & ~1));
    }
    __syncthreads();

    const uint32_t* trow = tbl + dm_sub * ND * cs_max;
    for (int sl = 0; sl < cs; sl++) {
#pragma unroll
      for (int r = 0; r < ND; r++) {
        const uint8_t* p = smem + trow[r * cs_max + sl] + toff;
#pragma unroll
        for (int m = 0; m < NW; m++) lanes[r][m] += *reinterpret_cast<const uint32_t*>(p + 128 * m);
      }
      if (++pending == a.flush_every) { fold(); pending = 0; }
    }
  }
  fold();

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
  if (c.chunk < 1 || c.chunk > 256) {
    *why = "chunk must lie in [1, 256]";
    return false;
  }
  return true;
}

size_t step2_smem_bytes(const sps_dedisp_config& c, int32_t dmax_tile) {
  const size_t Di = (size_t)c.warps_dm * c.dms_per_thread;
  return 2 * (size_t)c.chunk * copy_bytes(c, dmax_tile) + Di * c.chunk * 4;
}

sps_status launch_step2(const Step2Args& a, const sps_dedisp_config& c, cudaStream_t st) {
  std::string why;
  if (!step2_config_supported(c, &why)) return fail(SPS_ERR_INVALID_ARG, why);
  Step2Kernel fn = find(c.dms_per_thread, c.samples_per_thread / 2);
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  const size_t smem = step2_smem_bytes(c, a.dmax_tile);
  dim3 grid((a.n_t + Tt - 1) / Tt, a.n_tiles, 1);
  if (grid.y > 65535) return fail(SPS_ERR_UNSUPPORTED, "too many step-two tiles");
  SPS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<grid, 32 * c.warps_dm * c.warps_time, smem, st>>>(a, c.warps_dm, c.chunk, copy_bytes(c, a.dmax_tile));
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

}  // namespace sps
