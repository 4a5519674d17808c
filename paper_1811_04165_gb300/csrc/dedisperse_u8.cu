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
//     samples and walks the channels `chunk` at a time.  For each channel the
//     window [t0 + d(i0, c), t0 + Tt + d(i_last, c)) is staged once (16-byte
//     global loads) and read by all Di trials.
//   * Four copies of each window are kept, copy j shifted by j bytes, so that
//     every 4-sample read is one aligned, conflict-free 32-bit shared load
//     whatever the delay's alignment.
//   * SWAR: a word of 4 samples is split into even and odd bytes in 16-bit
//     lanes (one AND, one byte permute) and two channels are added per 3-input
//     add.  16-bit lanes stay exact for 257 channels of 255; partial sums are
//     folded into int32 registers every <= 256 channels.
//   * A per-chunk table of shared-memory offsets (one per trial and channel)
//     turns each trial's access into a broadcast load plus immediate offsets.
#include <algorithm>

#include "sps_internal.h"

namespace sps {
namespace {

constexpr uint32_t kEvenBytes = 0x00FF00FFu;
constexpr int kMaxThreads = 512;

__device__ __forceinline__ uint32_t odd_bytes(uint32_t w) { return __byte_perm(w, 0u, 0x4341); }

// Bytes [p, p + 20) of channel row `c`, zero at and beyond `len`.
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

template <int ND, int NW>
__global__ void __launch_bounds__(kMaxThreads, 1)
u8_pass_kernel(U8PassArgs a, int wd, int cc_max, int wb) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int Di = wd * ND;
  const int wt = (int)(blockDim.x >> 5) / wd;
  const int Tt = wt * 128 * NW;
  const int copy_stride = cc_max * wb;
  uint32_t* tbl = reinterpret_cast<uint32_t*>(smem + 4 * copy_stride);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int dm_sub = warp % wd, t_sub = warp / wd;
  const int t0 = blockIdx.x * Tt;
  const int i0 = blockIdx.y * Di;
  const int g = blockIdx.z;
  const int c_lo = g * a.group_channels, c_hi = c_lo + a.group_channels;
  const uint32_t toff = (uint32_t)(t_sub * 128 * NW + lane * 4);
  const int32_t* drow0 = a.delays + (int64_t)i0 * a.channels;

  uint32_t lo[ND][NW], hi[ND][NW];
  int32_t acc[ND][NW][4];
#pragma unroll
  for (int r = 0; r < ND; r++)
#pragma unroll
    for (int m = 0; m < NW; m++) {
      lo[r][m] = 0u; hi[r][m] = 0u;
#pragma unroll
      for (int q = 0; q < 4; q++) acc[r][m][q] = 0;
    }

  auto fold = [&]() {
#pragma unroll
    for (int r = 0; r < ND; r++)
#pragma unroll
      for (int m = 0; m < NW; m++) {
        acc[r][m][0] += (int32_t)(lo[r][m] & 0xFFFFu);
        acc[r][m][2] += (int32_t)(lo[r][m] >> 16);
        acc[r][m][1] += (int32_t)(hi[r][m] & 0xFFFFu);
        acc[r][m][3] += (int32_t)(hi[r][m] >> 16);
        lo[r][m] = 0u; hi[r][m] = 0u;
      }
  };

  int pending = 0;
  const int segs = wb >> 4;
  for (int cb = c_lo; cb < c_hi; cb += cc_max) {
    const int cc = min(cc_max, c_hi - cb);
    if (pending + cc > 256) { fold(); pending = 0; }
    __syncthreads();  // the previous chunk's readers are done with the buffers

    // Stage the windows: copy j holds raw byte (start + p + j) at position p.
    for (int e = tid; e < cc * segs; e += blockDim.x) {
      const int cl = e / segs, q = e - cl * segs;
      const int c = cb + cl;
      const int64_t start = (int64_t)((t0 + drow0[c]) & ~15);
      uint32_t r[5];
      load_raw20(a.x + (int64_t)c * a.pitch, start + 16 * q, a.in_len, r);
      uint8_t* dst = smem + cl * wb + 16 * q;
      *reinterpret_cast<uint4*>(dst) = make_uint4(r[0], r[1], r[2], r[3]);
      *reinterpret_cast<uint4*>(dst + copy_stride) =
          make_uint4(__byte_perm(r[0], r[1], 0x4321), __byte_perm(r[1], r[2], 0x4321),
                     __byte_perm(r[2], r[3], 0x4321), __byte_perm(r[3], r[4], 0x4321));
      *reinterpret_cast<uint4*>(dst + 2 * copy_stride) =
          make_uint4(__byte_perm(r[0], r[1], 0x5432), __byte_perm(r[1], r[2], 0x5432),
                     __byte_perm(r[2], r[3], 0x5432), __byte_perm(r[3], r[4], 0x5432));
      *reinterpret_cast<uint4*>(dst + 3 * copy_stride) =
          make_uint4(__byte_perm(r[0], r[1], 0x6543), __byte_perm(r[1], r[2], 0x6543),
                     __byte_perm(r[2], r[3], 0x6543), __byte_perm(r[3], r[4], 0x6543));
    }
    // Offsets: trial r of the block reads channel cl at copy (rel & 3), byte (rel & ~3).
    for (int e = tid; e < Di * cc; e += blockDim.x) {
      const int r = e / cc, cl = e - r * cc;
      const int i = min(i0 + r, a.n_dm - 1);
      const int c = cb + cl;
      const int d0 = drow0[c];
      const int di = a.delays[(int64_t)i * a.channels + c];
      const int start = (t0 + d0) & ~15;
      const int rel = t0 + di - start;
      tbl[r * cc_max + cl] = (uint32_t)((rel & 3) * copy_stride + cl * wb + (rel & ~3));
    }
    __syncthreads();

    const uint32_t* trow = tbl + dm_sub * ND * cc_max;
    int cl = 0;
    for (; cl + 1 < cc; cl += 2) {
#pragma unroll
      for (int r = 0; r < ND; r++) {
        const uint2 o = *reinterpret_cast<const uint2*>(trow + r * cc_max + cl);
        const uint8_t* p1 = smem + o.x + toff;
        const uint8_t* p2 = smem + o.y + toff;
#pragma unroll
        for (int m = 0; m < NW; m++) {
          const uint32_t w1 = *reinterpret_cast<const uint32_t*>(p1 + 128 * m);
          const uint32_t w2 = *reinterpret_cast<const uint32_t*>(p2 + 128 * m);
          lo[r][m] += (w1 & kEvenBytes) + (w2 & kEvenBytes);
          hi[r][m] += odd_bytes(w1) + odd_bytes(w2);
        }
      }
    }
    if (cl < cc) {
#pragma unroll
      for (int r = 0; r < ND; r++) {
        const uint8_t* p1 = smem + trow[r * cc_max + cl] + toff;
#pragma unroll
        for (int m = 0; m < NW; m++) {
          const uint32_t w1 = *reinterpret_cast<const uint32_t*>(p1 + 128 * m);
          lo[r][m] += w1 & kEvenBytes;
          hi[r][m] += odd_bytes(w1);
        }
      }
    }
    pending += cc;
  }
  fold();

  // Each lane holds 4 consecutive samples per (trial, word).
  const bool vec = (a.out_pitch & 3) == 0;
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
}

typedef void (*U8Kernel)(U8PassArgs, int, int, int);

template <int ND, int NW>
constexpr U8Kernel k() { return u8_pass_kernel<ND, NW>; }

struct Variant { int nd, nw; U8Kernel fn; };
const Variant kVariants[] = {
    {1, 1, k<1, 1>()}, {1, 2, k<1, 2>()}, {1, 4, k<1, 4>()}, {1, 8, k<1, 8>()},
    {2, 1, k<2, 1>()}, {2, 2, k<2, 2>()}, {2, 4, k<2, 4>()}, {2, 8, k<2, 8>()},
    {4, 1, k<4, 1>()}, {4, 2, k<4, 2>()}, {4, 4, k<4, 4>()},
    {8, 1, k<8, 1>()}, {8, 2, k<8, 2>()},
};

U8Kernel find(int nd, int nw) {
  for (const Variant& v : kVariants)
    if (v.nd == nd && v.nw == nw) return v.fn;
  return nullptr;
}

int copy_bytes(const sps_dedisp_config& c, int32_t dmax_tile) {
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  return (Tt + dmax_tile + 15 + 15) / 16 * 16;
}

}  // namespace

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
  if (c.chunk < 2 || c.chunk > 256 || (c.chunk & 1)) {
    *why = "chunk must be even and in [2, 256]";
    return false;
  }
  return true;
}

size_t u8_smem_bytes(const sps_dedisp_config& c, int32_t dmax_tile) {
  const size_t Di = (size_t)c.warps_dm * c.dms_per_thread;
  return 4 * (size_t)c.chunk * copy_bytes(c, dmax_tile) + Di * c.chunk * 4;
}

sps_status launch_u8_pass(const U8PassArgs& a, const sps_dedisp_config& c, cudaStream_t st) {
  std::string why;
  if (!u8_config_supported(c, &why)) return fail(SPS_ERR_INVALID_ARG, why);
  U8Kernel fn = find(c.dms_per_thread, c.samples_per_thread / 4);
  const int Di = c.warps_dm * c.dms_per_thread;
  const int Tt = c.warps_time * 32 * c.samples_per_thread;
  const size_t smem = u8_smem_bytes(c, a.dmax_tile);
  dim3 grid((a.n_out + Tt - 1) / Tt, (a.n_dm + Di - 1) / Di, a.n_groups);
  if (grid.y > 65535 || grid.z > 65535) return fail(SPS_ERR_UNSUPPORTED, "too many DM tiles or groups");
  SPS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fn<<<grid, 32 * c.warps_dm * c.warps_time, smem, st>>>(a, c.warps_dm, c.chunk, copy_bytes(c, a.dmax_tile));
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

}  // namespace sps
