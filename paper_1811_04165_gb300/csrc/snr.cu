// Boxcar integration and S/N with peak extraction (Sec. 2: smoothing of the
// de-dispersed series, then S/N; the sliding-boxcar reading of "smoothing").
//
// For each DM row the block forms the prefix sums P[t] = sum_{u<t} D[u] once in
// shared memory (32-bit wrap-around arithmetic: every boxcar
// B_w[t] = P[t + w] - P[t] is below 2^31, so the wrapped difference is exact),
// then for every width accumulates, over the N = N_t - w + 1 valid samples,
// the exact integer moments S1 = sum B (64-bit), S2 = sum B^2 (128-bit), the
// maximum and its first position.  One FP64 expression gives
//   snr = (N P - S1) / sqrt(N S2 - S1^2),
// i.e. (peak - mean) / population sigma, since N S2 - S1^2 = N^2 sigma^2.
// Nothing is materialised; the integrate kernel writes B for checking.
#include <algorithm>

#include "sps_internal.h"

namespace sps {
namespace {

constexpr int kMaxThreads = 1024;

// Block-wide exclusive prefix sum (uint32, wrap-around) of one value per thread.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < nw ? scratch[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) scratch[lane] = s;
  }
  __syncthreads();
  uint32_t base = warp ? scratch[warp - 1] : 0u;
  __syncthreads();
  return base + x - v;
}

// Fill P[0..n_t] with the prefix sums of one row (P[0] = 0).
__device__ void row_prefix(const int32_t* row, int n_t, uint32_t* P, uint32_t* scratch) {
  const int per = (n_t + blockDim.x - 1) / blockDim.x;
  const int b = min(n_t, (int)threadIdx.x * per), e = min(n_t, b + per);
  uint32_t s = 0;
  for (int t = b; t < e; t++) s += (uint32_t)__ldg(row + t);
  uint32_t run = block_exclusive_scan(s, scratch);
  for (int t = b; t < e; t++) {
    P[t] = run;
    run += (uint32_t)__ldg(row + t);
  }
  if (threadIdx.x == blockDim.x - 1) P[n_t] = run;
  if (n_t == 0 && threadIdx.x == 0) P[0] = 0;
  __syncthreads();
}

struct Moments {
  unsigned long long s1;
  unsigned long long s2lo, s2hi;
  int32_t best;
  int32_t best_t;
};

__device__ __forceinline__ void add128(unsigned long long& lo, unsigned long long& hi,
                                       unsigned long long vlo, unsigned long long vhi) {
  unsigned long long nlo = lo + vlo;
  hi += vhi + (nlo < lo ? 1ull : 0ull);
  lo = nlo;
}

__device__ __forceinline__ void merge(Moments& a, const Moments& b) {
  a.s1 += b.s1;
  add128(a.s2lo, a.s2hi, b.s2lo, b.s2hi);
  if (b.best > a.best || (b.best == a.best && b.best_t < a.best_t)) { a.best = b.best; a.best_t = b.best_t; }
}

__device__ Moments shfl_moments(const Moments& m, int o) {
  Moments r;
  r.s1 = __shfl_down_sync(0xffffffffu, m.s1, o);
  r.s2lo = __shfl_down_sync(0xffffffffu, m.s2lo, o);
  r.s2hi = __shfl_down_sync(0xffffffffu, m.s2hi, o);
  r.best = __shfl_down_sync(0xffffffffu, m.best, o);
  r.best_t = __shfl_down_sync(0xffffffffu, m.best_t, o);
  return r;
}

// (N P - S1) / sqrt(N S2 - S1^2) from exact moments; 0 for a constant series.
__device__ double snr_from_moments(int64_t N, const Moments& m) {
  const unsigned long long s1 = m.s1;
  // var_num = N*S2 - S1^2 in 128 bits (non-negative by Cauchy-Schwarz)
  const unsigned __int128 s2 = ((unsigned __int128)m.s2hi << 64) | m.s2lo;
  const unsigned __int128 var_num = (unsigned __int128)N * s2 - (unsigned __int128)s1 * s1;
  if (var_num == 0) return 0.0;
  const int64_t num = N * (int64_t)m.best - (int64_t)s1;
  const double v = __dadd_rn(__dmul_rn((double)(unsigned long long)(var_num >> 64), 18446744073709551616.0),
                             (double)(unsigned long long)var_num);
  return __ddiv_rn((double)num, __dsqrt_rn(v));
}

__global__ void __launch_bounds__(kMaxThreads, 1) snr_kernel(SnrArgs a) {
  extern __shared__ __align__(16) uint32_t P[];
  __shared__ uint32_t scratch[32];
  __shared__ Moments part[32];
  const int i = blockIdx.x;
  const int n_t = a.n_t;
  row_prefix(a.D + (int64_t)i * n_t, n_t, P, scratch);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;

  for (int wi = 0; wi < a.n_widths; wi++) {
    const int w = __ldg(a.widths + wi);
    const int N = n_t - w + 1;
    Moments m{0ull, 0ull, 0ull, -1, 0x7fffffff};
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
      const int32_t B = (int32_t)(P[t + w] - P[t]);
      m.s1 += (unsigned long long)(uint32_t)B;
      const unsigned long long sq = (unsigned long long)(uint32_t)B * (uint32_t)B;
      add128(m.s2lo, m.s2hi, sq, 0ull);
      if (B > m.best) { m.best = B; m.best_t = t; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) merge(m, shfl_moments(m, o));
    if (lane == 0) part[warp] = m;
    __syncthreads();
    if (warp == 0) {
      Moments r = lane < nw ? part[lane] : Moments{0ull, 0ull, 0ull, -1, 0x7fffffff};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) merge(r, shfl_moments(r, o));
      if (lane == 0) {
        const int64_t o = (int64_t)wi * a.n_dms + i;
        a.snr[o] = snr_from_moments(N, r);
        a.peak_t[o] = r.best_t;
        a.peak_val[o] = r.best;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kMaxThreads, 1)
integrate_kernel(const int32_t* D, int n_dms, int n_t, const int32_t* widths, int n_widths, int32_t* B) {
  extern __shared__ __align__(16) uint32_t P[];
  __shared__ uint32_t scratch[32];
  const int i = blockIdx.x;
  row_prefix(D + (int64_t)i * n_t, n_t, P, scratch);
  for (int wi = 0; wi < n_widths; wi++) {
    const int w = __ldg(widths + wi);
    const int N = n_t - w + 1;
    int32_t* out = B + ((int64_t)wi * n_dms + i) * n_t;
    for (int t = threadIdx.x; t < n_t; t += blockDim.x) out[t] = t < N ? (int32_t)(P[t + w] - P[t]) : 0;
  }
}

// Largest S/N over (width, DM); ties -> smaller DM index, then smaller width index.
__device__ __forceinline__ bool better(double v, int i, int w, double bv, int bi, int bw) {
  if (v != bv) return v > bv;
  if (i != bi) return i < bi;
  return w < bw;
}

__global__ void __launch_bounds__(1024, 1)
detect_kernel(const double* snr, const int32_t* peak_t, const int32_t* peak_val, int n_dms, int n_widths,
              int32_t* best) {
  __shared__ double sv[32];
  __shared__ int si[32], sw[32];
  double bv = -1.0;
  int bi = 0x7fffffff, bw = 0x7fffffff;
  const int64_t n = (int64_t)n_dms * n_widths;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const int w = (int)(e / n_dms), i = (int)(e - (int64_t)w * n_dms);
    const double v = snr[e];
    if (better(v, i, w, bv, bi, bw)) { bv = v; bi = i; bw = w; }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double v = __shfl_down_sync(0xffffffffu, bv, o);
    int i = __shfl_down_sync(0xffffffffu, bi, o), w = __shfl_down_sync(0xffffffffu, bw, o);
    if (better(v, i, w, bv, bi, bw)) { bv = v; bi = i; bw = w; }
  }
  if (lane == 0) { sv[warp] = bv; si[warp] = bi; sw[warp] = bw; }
  __syncthreads();
  if (warp == 0) {
    bv = lane < nw ? sv[lane] : -1.0;
    bi = lane < nw ? si[lane] : 0x7fffffff;
    bw = lane < nw ? sw[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double v = __shfl_down_sync(0xffffffffu, bv, o);
      int i = __shfl_down_sync(0xffffffffu, bi, o), w = __shfl_down_sync(0xffffffffu, bw, o);
      if (better(v, i, w, bv, bi, bw)) { bv = v; bi = i; bw = w; }
    }
    if (lane == 0) {
      const int64_t o = (int64_t)bw * n_dms + bi;
      best[0] = bi;
      best[1] = bw;
      best[2] = peak_t[o];
      best[3] = peak_val[o];
    }
  }
}

size_t prefix_smem(int n_t) { return ((size_t)n_t + 1) * sizeof(uint32_t); }

}  // namespace

bool snr_config_supported(const sps_snr_config& c, std::string* why) {
  if (c.threads < 32 || c.threads > kMaxThreads || (c.threads & 31)) {
    *why = "threads must be a multiple of 32 in [32, 1024]";
    return false;
  }
  return true;
}

sps_status launch_snr(const SnrArgs& a, const sps_snr_config& c, cudaStream_t st) {
  std::string why;
  if (!snr_config_supported(c, &why)) return fail(SPS_ERR_INVALID_ARG, why);
  const size_t smem = prefix_smem(a.n_t);
  int dev = 0, max_smem = 0;
  SPS_CUDA(cudaGetDevice(&dev));
  SPS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem + 32 * sizeof(Moments) + 128 > (size_t)max_smem)
    return fail(SPS_ERR_UNSUPPORTED, "rows too long for the shared-memory prefix");
  SPS_CUDA(cudaFuncSetAttribute(snr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  snr_kernel<<<a.n_dms, c.threads, smem, st>>>(a);
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

sps_status launch_integrate(const int32_t* D, int32_t n_dms, int32_t n_t, const int32_t* widths,
                            int32_t n_widths, int32_t* B, cudaStream_t st) {
  const size_t smem = prefix_smem(n_t);
  SPS_CUDA(cudaFuncSetAttribute(integrate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  integrate_kernel<<<n_dms, 256, smem, st>>>(D, n_dms, n_t, widths, n_widths, B);
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

sps_status launch_detect(const double* snr, const int32_t* peak_t, const int32_t* peak_val, int32_t n_dms,
                         int32_t n_widths, int32_t* best, cudaStream_t st) {
  detect_kernel<<<1, 1024, 0, st>>>(snr, peak_t, peak_val, n_dms, n_widths, best);
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

}  // namespace sps
