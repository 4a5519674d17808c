// RFI channel zapping (Sec. 2, footnote: channels to zap because of
// terrestrial interference): a copy of the input whose zapped rows are zero,
// bytes at and beyond in_len zero too; the search then reads the copy.
#include "sps_internal.h"

namespace sps {
namespace {

__global__ void __launch_bounds__(256) zap_copy_kernel(const uint8_t* x, int64_t pitch, int32_t in_len,
                                                       const uint8_t* zap, int32_t channels, uint8_t* out,
                                                       int64_t out_pitch) {
  const int64_t per_row = out_pitch >> 4;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= per_row * channels) return;
  const int c = (int)(id / per_row);
  const int p = (int)(id - (int64_t)c * per_row) << 4;
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (!__ldg(zap + c)) {
    const uint8_t* row = x + (int64_t)c * pitch;
    if (p + 16 <= in_len) {
      v = __ldg(reinterpret_cast<const uint4*>(row + p));
    } else {
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      for (int b = 0; b < 16 && p + b < in_len; b++) w[b >> 2] |= (uint32_t)__ldg(row + p + b) << (8 * (b & 3));
      v = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  *reinterpret_cast<uint4*>(out + (int64_t)c * out_pitch + p) = v;
}

}  // namespace

sps_status launch_zap_copy(const uint8_t* x, int64_t pitch, int32_t in_len, const uint8_t* zap, int32_t channels,
                           uint8_t* out, int64_t out_pitch, cudaStream_t st) {
  const int64_t threads = (out_pitch >> 4) * channels;
  zap_copy_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(x, pitch, in_len, zap, channels, out, out_pitch);
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

}  // namespace sps
