// Boxcar integration and S/N with peak extraction (Sec. 2: smoothing of the
// de-dispersed series, then S/N; the sliding-boxcar reading of "smoothing").
//
// One block per DM row.  The row arrives in shared memory by one bulk copy
// (TMA) and is turned in place into prefix sums P[t] = sum_{u<t} D[u] (32-bit
// wrap-around arithmetic: every boxcar B_w[t] = P[t + w] - P[t] is below 2^31,
// so the wrapped difference is exact).  A single pass over t then serves all
// widths of the pass at once, accumulating per width the exact integer moment
// S2 = sum B^2 (128-bit at block level), the maximum and its first position
// over the N = N_t - w + 1 valid samples.  S1 = sum B needs no pass: every
// sample u lies in w boxcars except near the ends, so
//   S1 = w T - sum_{j=1}^{w-1} P[j] - sum_{j=1}^{w-1} (T - P[N_t - j]),
// T = P[N_t] (for decimation by f it telescopes to P[floor(N_t / f) f]); each
// thread adds w times its share of T and subtracts its share of the end
// terms, all exact in 64 bits.  One FP64 expression gives
//   snr = (N P - S1) / sqrt(N S2 - S1^2),
// i.e. (peak - mean) / population sigma, since N S2 - S1^2 = N^2 sigma^2.
// Nothing is materialised; the integrate kernel writes B for checking.
#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "sps_internal.h"
#include "tma.cuh"

namespace sps {
namespace {

constexpr int kMaxThreads = 512;
constexpr int kWidthsPerPass = 8;
constexpr int kPad = 4;  // P[k] lives at buf[kPad - 1 + k]; the row lands at buf[kPad]

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

// Load row i into buf[kPad .. kPad + n_t) and turn it into prefix sums in place:
// afterwards buf[kPad - 1 + k] = sum_{u<k} D[u] for k = 0..n_t.  *seg = the sum
// of the samples this thread scanned (the threads' segments tile the row).
__device__ bool load_prefix(const int32_t* row, int n_t, uint32_t* buf, uint32_t* scratch, uint64_t* bar,
                            bool use_tma, uint32_t* status, uint32_t* seg) {
  bool ok = true;
  if (use_tma) {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
      mbar_arrive_expect_tx(bar, (uint32_t)n_t * 4u);
      bulk_g2s(buf + kPad, row, (uint32_t)n_t * 4u, bar);
    }
    __syncthreads();
    ok = mbar_wait(bar, 0, status);
    if (__syncthreads_or(ok ? 0 : 1)) {
      // a copy that did not land in time may still be in flight: give it one
      // more bounded wait before the block's shared memory is released
      if (threadIdx.x == 0) mbar_wait(bar, 0, status);
      return false;
    }
  } else {
    for (int t = threadIdx.x; t < n_t; t += blockDim.x) buf[kPad + t] = (uint32_t)__ldg(row + t);
  }
  if (threadIdx.x == 0) buf[kPad - 1] = 0u;
  __syncthreads();
  // odd segment lengths keep the strided shared accesses free of bank conflicts
  const int per = ((n_t + blockDim.x - 1) / blockDim.x) | 1;
  const int b = min(n_t, (int)threadIdx.x * per), e = min(n_t, b + per);
  uint32_t s = 0;
  for (int t = b; t < e; t++) s += buf[kPad + t];
  *seg = s;
  uint32_t run = block_exclusive_scan(s, scratch);
  for (int t = b; t < e; t++) {
    run += buf[kPad + t];
    buf[kPad + t] = run;
  }
  __syncthreads();
  return ok;
}

struct Moments {
  unsigned long long s1;
  unsigned long long s2lo, s2hi;
  int32_t best;
  int32_t best_t;
};

__device__ __forceinline__ void add128(unsigned long long& lo, unsigned long long& hi, unsigned long long v) {
  const unsigned long long n = lo + v;
  hi += n < lo ? 1ull : 0ull;
  lo = n;
}

__device__ __forceinline__ void merge(Moments& a, const Moments& b) {
  a.s1 += b.s1;
  const unsigned long long n = a.s2lo + b.s2lo;
  a.s2hi += b.s2hi + (n < a.s2lo ? 1ull : 0ull);
  a.s2lo = n;
  if (b.best > a.best || (b.best == a.best && b.best_t < a.best_t)) { a.best = b.best; a.best_t = b.best_t; }
}

__device__ Moments shfl_down(const Moments& m, int o) {
  Moments r;
  r.s1 = __shfl_down_sync(0xffffffffu, m.s1, o);
  r.s2lo = __shfl_down_sync(0xffffffffu, m.s2lo, o);
  r.s2hi = __shfl_down_sync(0xffffffffu, m.s2hi, o);
  r.best = __shfl_down_sync(0xffffffffu, m.best, o);
  r.best_t = __shfl_down_sync(0xffffffffu, m.best_t, o);
  return r;
}

// (N P - S1) / sqrt(N S2 - S1^2) from exact moments; 0 for a constant series.
// Both integers are exact; the variance numerator is rounded once to double and
// the quotient taken as num * rsqrt(var) (FP64, within 2 ulp): a few FP64
// operations, which matter on this part's narrow FP64 path.
__device__ double snr_from_moments(int64_t N, const Moments& m) {
  const unsigned __int128 s2 = ((unsigned __int128)m.s2hi << 64) | m.s2lo;
  const unsigned __int128 var_num = (unsigned __int128)N * s2 - (unsigned __int128)m.s1 * m.s1;
  if (var_num == 0) return 0.0;
  const int64_t num = N * (int64_t)m.best - (int64_t)m.s1;
  const double v = fma((double)(unsigned long long)(var_num >> 64), 18446744073709551616.0,
                       (double)(unsigned long long)var_num);
  return (double)num * rsqrt(v);
}

// One pass over widths [w_begin, w_begin + NWP) (ascending).  `flush`: samples a
// thread may add into its 32-bit S1 and 64-bit S2 partials before they could
// overflow (from the largest possible boxcar value).  The pass tracks only the
// maximum; the first position of the block's maximum is found afterwards by the
// few threads whose own maximum equals it.
//
// `narrow`: the host has shown that a warp's S2 total fits 64 bits (32 threads'
// samples times the largest square), so warps reduce S1 and S2 as 64-bit sums
// and the maximum with one redux; otherwise the full 128-bit merge runs.
//
// DEC: the widths are downsampling factors f; the series is X_f[j] =
// P[(j+1) f] - P[j f] for j < N_t / f (Table 2 DOWNSAMPLING), and peak_t is
// reported as f j.
//
// FAST: the host has shown that no thread's partials ever need flushing and
// that warp sums fit 64 bits (`narrow`), so a thread keeps only its 32-bit S1,
// 64-bit S2 and maximum per width; at most 64 registers, twice the blocks per SM.
template <int NWP, bool DEC, bool FAST>
__global__ void __launch_bounds__(kMaxThreads, FAST ? 2 : 1) snr_kernel(SnrArgs a, int w_begin, int flush,
                                                                        int use_tma, int narrow) {
  extern __shared__ __align__(16) uint32_t buf[];
  __shared__ uint32_t scratch[32];
  __shared__ uint64_t bar;
  __shared__ Moments part[kMaxThreads / 32][NWP];  // one entry per warp and width
  __shared__ int gmax[NWP], first[NWP];
  const int i = blockIdx.x;
  const int n_t = a.n_t;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t seg = 0;
  if (!load_prefix(a.D + (int64_t)i * n_t, n_t, buf, scratch, &bar, use_tma != 0, a.status, &seg)) return;
  const uint32_t* P = buf + kPad - 1;

  int W[NWP];
  uint32_t mx[NWP];
  unsigned long long s2p[NWP], s2lo[NWP], s2hi[NWP];
#pragma unroll
  for (int k = 0; k < NWP; k++) {
    W[k] = __ldg(a.widths + w_begin + k);
    mx[k] = 0u; s2p[k] = 0ull; s2lo[k] = 0ull; s2hi[k] = 0ull;
  }
  if (threadIdx.x < NWP) first[threadIdx.x] = 0x7fffffff;
  auto flush_partials = [&]() {
    if constexpr (!FAST) {
#pragma unroll
      for (int k = 0; k < NWP; k++) {
        add128(s2lo[k], s2hi[k], s2p[k]);
        s2p[k] = 0ull;
      }
    }
  };
  if constexpr (DEC) {
    // each factor strides its own samples; partials are flushed per factor
#pragma unroll
    for (int k = 0; k < NWP; k++) {
      const int N = n_t / W[k];
      int count = 0;
      for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const uint32_t B = P[(j + 1) * W[k]] - P[j * W[k]];
        s2p[k] += (unsigned long long)B * B;
        mx[k] = max(mx[k], B);
        if (!FAST && ++count == flush) { flush_partials(); count = 0; }
      }
    }
  } else {
    const int n_all = n_t - W[NWP - 1] + 1;  // every width of the pass is valid below this
    const int n_any = n_t - W[0] + 1;
    int count = 0;
    int t = threadIdx.x;
    for (; t < n_all; t += blockDim.x) {
      const uint32_t p0 = P[t];
#pragma unroll
      for (int k = 0; k < NWP; k++) {
        const uint32_t B = P[t + W[k]] - p0;
        s2p[k] += (unsigned long long)B * B;
        mx[k] = max(mx[k], B);
      }
      if (!FAST && ++count == flush) { flush_partials(); count = 0; }
    }
    for (; t < n_any; t += blockDim.x) {
      const uint32_t p0 = P[t];
#pragma unroll
      for (int k = 0; k < NWP; k++) {
        if (t + W[k] <= n_t) {
          const uint32_t B = P[t + W[k]] - p0;
          s2p[k] += (unsigned long long)B * B;
          mx[k] = max(mx[k], B);
        }
      }
      if (!FAST && ++count == flush) { flush_partials(); count = 0; }
    }
  }
  flush_partials();
  // this thread's share of S1 (wrap-around 64-bit terms; the block total is exact)
  unsigned long long s1t[NWP];
  if constexpr (DEC) {
    // S1 = P[N f]: T less the samples after the last whole window (fewer than f)
#pragma unroll
    for (int k = 0; k < NWP; k++)
      s1t[k] = (unsigned long long)seg -
               (threadIdx.x == 0 ? (unsigned long long)(P[n_t] - P[n_t / W[k] * W[k]]) : 0ull);
  } else {
#pragma unroll
    for (int k = 0; k < NWP; k++) s1t[k] = (unsigned long long)W[k] * seg;
    // end terms: P[j] and T - P[N_t - j] for 1 <= j < w, each below 2^31
    for (int j = (int)threadIdx.x + 1; j < W[NWP - 1]; j += blockDim.x) {
      const unsigned long long v = (unsigned long long)P[j] + (unsigned long long)(P[n_t] - P[n_t - j]);
#pragma unroll
      for (int k = 0; k < NWP; k++)
        if (j < W[k]) s1t[k] -= v;
    }
  }
  if (FAST || narrow) {
#pragma unroll
    for (int k = 0; k < NWP; k++) {
      unsigned long long s1 = s1t[k], s2 = FAST ? s2p[k] : s2lo[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      }
      const uint32_t m = __reduce_max_sync(0xffffffffu, mx[k]);
      if (lane == 0) part[warp][k] = Moments{s1, s2, 0ull, (int32_t)m, 0};
    }
  } else {
#pragma unroll
    for (int k = 0; k < NWP; k++) {
      Moments m{s1t[k], s2lo[k], s2hi[k], (int32_t)mx[k], 0};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) merge(m, shfl_down(m, o));
      if (lane == 0) part[warp][k] = m;
    }
  }
  __syncthreads();
  if (threadIdx.x < NWP) {
    const int k = threadIdx.x;
    int best = part[0][k].best;
    for (int q = 1; q < nw; q++) best = max(best, part[q][k].best);
    gmax[k] = best;
  }
  __syncthreads();
  // first position of the maximum: the warp of each thread holding it searches
  // that thread's samples (u = owner + m * blockDim.x) together, 32 at a time
#pragma unroll
  for (int k = 0; k < NWP; k++) {
    const int N = DEC ? n_t / W[k] : n_t - W[k] + 1;
    unsigned owners = __ballot_sync(0xffffffffu, (int32_t)mx[k] == gmax[k]);
    while (owners) {
      const int o = __ffs(owners) - 1;
      owners &= owners - 1;
      const int owner = warp * 32 + o;
      for (int m0 = 0; owner + m0 * (int)blockDim.x < N; m0 += 32) {
        const int u = owner + (m0 + lane) * (int)blockDim.x;
        const uint32_t v = u < N ? (DEC ? P[(u + 1) * W[k]] - P[u * W[k]] : P[u + W[k]] - P[u]) : 0u;
        const bool hit = u < N && (int32_t)v == gmax[k];
        const unsigned h = __ballot_sync(0xffffffffu, hit);
        if (h) {
          if (lane == 0) atomicMin(&first[k], owner + (m0 + __ffs(h) - 1) * (int)blockDim.x);
          break;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < NWP) {
    const int k = threadIdx.x;
    Moments r = part[0][k];
    for (int q = 1; q < nw; q++) merge(r, part[q][k]);
    const int64_t o = (int64_t)(w_begin + k) * a.n_dms + i;
    a.snr[o] = snr_from_moments(DEC ? n_t / W[k] : n_t - W[k] + 1, r);
    a.peak_t[o] = DEC ? first[k] * W[k] : first[k];
    a.peak_val[o] = gmax[k];
  }
}

__global__ void __launch_bounds__(kMaxThreads, 1)
integrate_kernel(const int32_t* D, int n_dms, int n_t, const int32_t* widths, int n_widths, int32_t* B,
                 int use_tma, int decimate, uint32_t* status) {
  extern __shared__ __align__(16) uint32_t buf[];
  __shared__ uint32_t scratch[32];
  __shared__ uint64_t bar;
  const int i = blockIdx.x;
  uint32_t seg = 0;
  if (!load_prefix(D + (int64_t)i * n_t, n_t, buf, scratch, &bar, use_tma != 0, status, &seg)) return;
  const uint32_t* P = buf + kPad - 1;
  for (int wi = 0; wi < n_widths; wi++) {
    const int w = __ldg(widths + wi);
    const int N = decimate ? n_t / w : n_t - w + 1;
    int32_t* out = B + ((int64_t)wi * n_dms + i) * n_t;
    for (int t = threadIdx.x; t < n_t; t += blockDim.x)
      out[t] = t < N ? (int32_t)(decimate ? P[(t + 1) * w] - P[t * w] : P[t + w] - P[t]) : 0;
  }
}

// Largest S/N over (width, DM); ties -> smaller DM index, then smaller width
// index.  Every S/N this library writes is a finite double >= +0 (the peak is
// never below the mean; a constant series gives 0), and the bit patterns of
// such doubles, read as signed 64-bit integers, order exactly as the values, so
// the comparison runs on the integer pipe (the FP64 pipe of this part is
// narrow).  The sentinel LLONG_MIN loses to every entry.
__device__ __forceinline__ bool better(long long v, int i, int w, long long bv, int bi, int bw) {
  if (v != bv) return v > bv;
  if (i != bi) return i < bi;
  return w < bw;
}

// The detection over the whole S/N table by one cluster of kDetectBlocks
// blocks: every thread takes entries e = w n_dms + i at a stride of the
// cluster's thread count (a couple each for a beam), the blocks reduce their
// threads, and block 0 reduces the blocks' results through distributed shared
// memory and writes best = {i, w, peak_t, peak_val}.  Launched after the S/N
// kernel on the same stream, so the table is complete and visible; no fence,
// counter or zeroed buffer is involved.
constexpr int kDetectBlocks = 8;
constexpr int kDetectThreads = 1024;

__global__ void __cluster_dims__(kDetectBlocks, 1, 1) __launch_bounds__(kDetectThreads, 1)
detect_kernel(const double* snr, const int32_t* peak_t, const int32_t* peak_val, int n_dms, int n_widths,
              int32_t* best) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ long long sv[32];
  __shared__ int si[32], sw[32];
  __shared__ long long cv[kDetectBlocks];  // block 0: the blocks' results
  __shared__ int ci[kDetectBlocks], cw[kDetectBlocks];
  cluster.barrier_arrive();  // matched before the remote writes into block 0
  const int rank = (int)cluster.block_rank();
  const int total = n_widths * n_dms;  // below 2^31 (checked by the launcher)
  const int stride = kDetectBlocks * (int)blockDim.x;
  const long long* key = reinterpret_cast<const long long*>(snr);
  long long bv = LLONG_MIN;
  int bi = 0x7fffffff, bw = 0x7fffffff;
  constexpr int kIn = 4;  // table reads in flight per thread
  for (int e0 = rank * (int)blockDim.x + (int)threadIdx.x; e0 < total; e0 += kIn * stride) {
    long long v[kIn];
#pragma unroll
    for (int u = 0; u < kIn; u++) v[u] = e0 + u * stride < total ? key[e0 + u * stride] : LLONG_MIN;
#pragma unroll
    for (int u = 0; u < kIn; u++) {
      const int e = e0 + u * stride;
      if (e >= total) break;
      const int w = e / n_dms, i = e - w * n_dms;
      if (better(v[u], i, w, bv, bi, bw)) { bv = v[u]; bi = i; bw = w; }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long v = __shfl_down_sync(0xffffffffu, bv, o);
    const int i = __shfl_down_sync(0xffffffffu, bi, o), w = __shfl_down_sync(0xffffffffu, bw, o);
    if (better(v, i, w, bv, bi, bw)) { bv = v; bi = i; bw = w; }
  }
  if (lane == 0) { sv[warp] = bv; si[warp] = bi; sw[warp] = bw; }
  __syncthreads();
  if (warp == 0) {
    bv = lane < nw ? sv[lane] : LLONG_MIN;
    bi = lane < nw ? si[lane] : 0x7fffffff;
    bw = lane < nw ? sw[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long v = __shfl_down_sync(0xffffffffu, bv, o);
      const int i = __shfl_down_sync(0xffffffffu, bi, o), w = __shfl_down_sync(0xffffffffu, bw, o);
      if (better(v, i, w, bv, bi, bw)) { bv = v; bi = i; bw = w; }
    }
  }
  cluster.barrier_wait();  // every block of the cluster has started
  if (warp == 0 && lane == 0) {
    *cluster.map_shared_rank(&cv[rank], 0) = bv;
    *cluster.map_shared_rank(&ci[rank], 0) = bi;
    *cluster.map_shared_rank(&cw[rank], 0) = bw;
  }
  cluster.sync();  // every block's result is in block 0's shared memory
  if (rank == 0 && threadIdx.x == 0) {
    bv = cv[0];
    bi = ci[0];
    bw = cw[0];
    for (int q = 1; q < kDetectBlocks; q++)
      if (better(cv[q], ci[q], cw[q], bv, bi, bw)) { bv = cv[q]; bi = ci[q]; bw = cw[q]; }
    const int64_t o = (int64_t)bw * n_dms + bi;
    best[0] = bi;
    best[1] = bw;
    best[2] = peak_t[o];
    best[3] = peak_val[o];
  }
}

// ---------------------------------------------------------------------------
// Vector form for width sets {1, 2, 4, ..., 2^(NW-1)} (the smoothing widths
// of the search; AMBER's are powers of two as well).
//
// One block per row.  The row arrives by one bulk copy (TMA) and is scanned in
// place into prefix sums (P[k] at buf[3 + k], 16-byte shared accesses).  The
// outputs are then taken four at a time: group j holds t = 4j - 3 .. 4j, whose
// P[t] are the aligned word quadruple buf[4j .. 4j + 3]; with the widths known
// at compile time every P[t + w] is a 16-byte load too (buf[4j + 4] serves
// w = 1, 2 and 4, buf[4j + w] the wider ones), consecutive lanes reading
// consecutive quadruples.  A group costs NW - 1 shared loads for 4 NW boxcars,
// each boxcar a subtract, a maximum (integer ALU) and one 32 x 32 -> 64-bit
// multiply-add (mad.wide, FMA pipe).  Only the first and last groups test
// validity (outputs outside [0, N_t - w] are skipped).  S1 comes in closed
// form as in snr_kernel.
//
// The detection follows as its own one-cluster launch (detect_kernel).

// Scans the row at buf[4 .. 4 + n_t) in place into P[k] = buf[3 + k] (k = 0 ..
// n_t); returns the sum of the samples this thread scanned.  Each thread scans
// a run of `per` samples (a multiple of 4 with per / 4 odd, so the 16-byte
// accesses of a warp are conflict-free).
__device__ uint32_t scan_row_v4(uint32_t* buf, int n_t, uint32_t* scratch) {
  if (threadIdx.x == 0) buf[3] = 0u;
  int per = ((n_t + blockDim.x - 1) / blockDim.x + 3) / 4 * 4;
  if ((per / 4) % 2 == 0) per += 4;
  const int b = min(n_t, (int)threadIdx.x * per), e = min(n_t, b + per);
  const int ev = b + (e - b) / 4 * 4;  // vector part [b, ev)
  uint32_t s = 0;
  for (int t = b; t < ev; t += 4) {
    const uint4 v = *reinterpret_cast<const uint4*>(buf + 4 + t);
    s += v.x + v.y + v.z + v.w;
  }
  for (int t = ev; t < e; t++) s += buf[4 + t];
  uint32_t run = block_exclusive_scan(s, scratch);
  for (int t = b; t < ev; t += 4) {
    uint4 v = *reinterpret_cast<const uint4*>(buf + 4 + t);
    v.x += run;
    v.y += v.x;
    v.z += v.y;
    v.w += v.z;
    run = v.w;
    *reinterpret_cast<uint4*>(buf + 4 + t) = v;
  }
  for (int t = ev; t < e; t++) {
    run += buf[4 + t];
    buf[4 + t] = run;
  }
  __syncthreads();
  return s;
}

// S2 += B * B, a 32 x 32 -> 64-bit product added to a 64-bit sum (written in
// C++: measured slightly faster on sm_103a than the explicit mad.wide.u32).
__device__ __forceinline__ void add_square(unsigned long long& acc, uint32_t b) {
  acc += (unsigned long long)b * b;
}

// Sum over the warp of a 64-bit value below 2^64 (every lane gets it), by three
// 22/22/20-bit limbs whose warp sums fit 32 bits (redux.sync).
__device__ __forceinline__ unsigned long long warp_sum64_redux(unsigned long long v) {
  const uint32_t r0 = __reduce_add_sync(0xffffffffu, (uint32_t)v & 0x3FFFFFu);
  const uint32_t r1 = __reduce_add_sync(0xffffffffu, (uint32_t)(v >> 22) & 0x3FFFFFu);
  const uint32_t r2 = __reduce_add_sync(0xffffffffu, (uint32_t)(v >> 44));
  return (unsigned long long)r0 + ((unsigned long long)r1 << 22) + ((unsigned long long)r2 << 44);
}

__device__ __forceinline__ uint32_t quad(const uint4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Moments, maxima and first peak positions of one scanned row for widths 1, 2,
// ..., 2^(NW-1), written to the row's S/N, peak_t and peak_val entries.
template <int NW>
__device__ void row_stats_v4(const SnrArgs& a, const uint32_t* buf, int row, uint32_t segsum) {
  constexpr int WMAX = 1 << (NW - 1);
  __shared__ unsigned long long ps2[kMaxThreads / 32][NW], ptot[kMaxThreads / 32], s1v[NW];
  __shared__ uint32_t pmx[kMaxThreads / 32][NW];
  __shared__ int gmax[NW], first[NW];
  const int n_t = a.n_t;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t* P = buf + 3;  // P[k], k = 0 .. n_t
  const int n_grp = (n_t + 3 + 3) / 4;  // groups of t = 4j - 3 .. 4j covering 0 .. n_t - 1
  uint32_t mx[NW];
  unsigned long long s2[NW];
#pragma unroll
  for (int k = 0; k < NW; k++) { mx[k] = 0u; s2[k] = 0ull; }
  if (threadIdx.x < NW) first[threadIdx.x] = 0x7fffffff;
  for (int j = threadIdx.x; j < n_grp; j += blockDim.x) {
    const int t0 = 4 * j - 3;
    if (t0 >= 0 && t0 + 3 + WMAX <= n_t) {
      // every output of the group is valid for every width
      const uint4 A = *reinterpret_cast<const uint4*>(buf + 4 * j);      // P[t0 .. t0 + 3]
      const uint4 N = *reinterpret_cast<const uint4*>(buf + 4 * j + 4);  // P[t0 + 4 .. t0 + 7]
#pragma unroll
      for (int k = 0; k < NW; k++) {
        const int w = 1 << k;
        uint4 Q;
        if (w >= 8) Q = *reinterpret_cast<const uint4*>(buf + 4 * j + w);  // P[t0 + w .. t0 + w + 3]
#pragma unroll
        for (int i = 0; i < 4; i++) {
          // P[t0 + i + w] - P[t0 + i]
          const uint32_t hi = w >= 8 ? quad(Q, i) : (i + w < 4 ? quad(A, i + w) : quad(N, i + w - 4));
          const uint32_t B = hi - quad(A, i);
          add_square(s2[k], B);
          mx[k] = max(mx[k], B);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < NW; k++) {
        const int w = 1 << k;
#pragma unroll 1
        for (int i = 0; i < 4; i++) {
          const int t = t0 + i;
          if (t >= 0 && t + w <= n_t) {
            const uint32_t B = P[t + w] - P[t];
            add_square(s2[k], B);
            mx[k] = max(mx[k], B);
          }
        }
      }
    }
  }
  // warp sums: S2 per width, the maximum, and the row total (for S1)
#pragma unroll
  for (int k = 0; k < NW; k++) {
    const unsigned long long v2 = warp_sum64_redux(s2[k]);
    const uint32_t m = __reduce_max_sync(0xffffffffu, mx[k]);
    if (lane == 0) { ps2[warp][k] = v2; pmx[warp][k] = m; }
  }
  {
    const unsigned long long t = warp_sum64_redux(segsum);
    if (lane == 0) ptot[warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < NW) {
    const int k = threadIdx.x;
    uint32_t m = pmx[0][k];
    for (int q = 1; q < nw; q++) m = max(m, pmx[q][k]);
    gmax[k] = (int)m;
  }
  __syncthreads();
  if (warp == nw - 1) {
    // S1 = w T - sum_{j<w} P[j] - sum_{j<w} (T - P[N_t - j]): every sample lies
    // in w boxcars except within w - 1 of either end.  Each lane reads the end
    // terms of j = lane + 1 and lane + 33 once (each below 2^31) and adds them
    // into every width they belong to; one limb sum per width.
    unsigned long long T = 0ull;
    for (int q = 0; q < nw; q++) T += ptot[q];
    uint32_t e0 = 0u, e1 = 0u;
    const int j0 = lane + 1, j1 = lane + 33;
    if (j0 < WMAX) e0 = P[j0] + (P[n_t] - P[n_t - j0]);
    if (j1 < WMAX) e1 = P[j1] + (P[n_t] - P[n_t - j1]);
#pragma unroll
    for (int k = 0; k < NW; k++) {
      const unsigned long long e = warp_sum64_redux((unsigned long long)(j0 < (1 << k) ? e0 : 0u) +
                                                    (unsigned long long)(j1 < (1 << k) ? e1 : 0u));
      if (lane == 0) s1v[k] = (unsigned long long)(1u << k) * T - e;
    }
  }
  // first position of each maximum: the warp of each thread holding it searches
  // that thread's groups, 8 groups (32 outputs) at a time, in order
#pragma unroll
  for (int k = 0; k < NW; k++) {
    const int w = 1 << k;
    unsigned owners = __ballot_sync(0xffffffffu, (int)mx[k] == gmax[k]);
    while (owners) {
      const int o = __ffs(owners) - 1;
      owners &= owners - 1;
      const int owner = warp * 32 + o;
      for (int m0 = 0; owner + m0 * (int)blockDim.x < n_grp; m0 += 8) {
        // lane -> group owner + (m0 + lane / 4) * blockDim, output lane % 4 of it
        const int j = owner + (m0 + (lane >> 2)) * (int)blockDim.x;
        const int t = 4 * j - 3 + (lane & 3);
        const bool hit = j < n_grp && t >= 0 && t + w <= n_t && (int)(P[t + w] - P[t]) == gmax[k];
        const unsigned h = __ballot_sync(0xffffffffu, hit);
        if (h) {
          const int l = __ffs(h) - 1;
          if (lane == 0) atomicMin(&first[k], 4 * (owner + (m0 + (l >> 2)) * (int)blockDim.x) - 3 + (l & 3));
          break;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < NW) {
    const int k = threadIdx.x;
    Moments r{s1v[k], ps2[0][k], 0ull, gmax[k], 0};
    for (int q = 1; q < nw; q++) r.s2lo += ps2[q][k];
    const int64_t o = (int64_t)k * a.n_dms + row;
    a.snr[o] = snr_from_moments(n_t - (1 << k) + 1, r);
    a.peak_t[o] = first[k];
    a.peak_val[o] = gmax[k];
  }
}

template <int NW>
__global__ void __launch_bounds__(kMaxThreads, 2) snr_pow2_kernel(SnrArgs a) {
  extern __shared__ __align__(16) uint32_t buf[];
  __shared__ uint32_t scratch[32];
  __shared__ uint64_t bar;
  const int row = blockIdx.x;
  const int n_t = a.n_t;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, (uint32_t)n_t * 4u);
    bulk_g2s(buf + 4, a.D + (int64_t)row * n_t, (uint32_t)n_t * 4u, &bar);
  }
  __syncthreads();
  const bool ok = mbar_wait(&bar, 0, a.status);
  if (__syncthreads_or(ok ? 0 : 1)) {
    // a copy that did not land in time may still be in flight: one more
    // bounded wait before the block's shared memory is released
    if (threadIdx.x == 0) mbar_wait(&bar, 0, a.status);
    return;
  }
  const uint32_t segsum = scan_row_v4(buf, n_t, scratch);
  row_stats_v4<NW>(a, buf, row, segsum);
}

// ---------------------------------------------------------------------------
// Streaming form for width sets {1, 2, 4, ..., 2^(NW-1)}, for rows too long to
// stage whole in shared memory (the row form above is faster when they fit).
//
// One block per DM row; the row's outputs are cut into chunks of 256 samples
// and each warp takes a contiguous run of chunks (its segment), so the warps
// never wait for one another until the row is done.  A warp streams its
// segment: lane l holds the chunk's samples base + 4l .. base + 4l + 3 and
// base + 128 + 4l .. base + 131 + 4l, copied by 16-byte asynchronous copies
// (cp.async) three chunks ahead into the warp's staging slots.  The chunk is
// scanned into 32-bit wrap-around prefix sums P (relative to the segment's
// first sample: a boxcar is a difference, B_w[t] = P[t + w] - P[t], exact since
// B < 2^31) by lane-local adds and warp shuffles, and stored in the warp's ring
// of two chunk slots (slot 0's first 64 words mirrored after slot 1, so that
// every P[t + w] of a chunk is one aligned 16-byte load at a fixed offset).  A
// chunk's boxcars need the next chunk's prefix, so the scan runs one chunk
// ahead (the segment's last chunk reads one chunk past it).  Per boxcar: a
// subtract and a maximum, and the square added to a 64-bit sum.
//
// The first position of each maximum: each lane keeps, per width, its largest
// boxcar and the first chunk where it reached it (a chunk's maximum compared
// once with the running one).  After the block has the row's maximum, the
// earliest chunk holding it is re-scanned from D by one warp, which takes the
// first sample equal to the maximum.  S1 = sum B needs no pass: with T the row
// total, S1_w = w T - sum_{u < w-1} (w-1-u) D[u] - sum_{u > N_t-w} (u-N_t+w) D[u]
// (every sample lies in w boxcars except within w - 1 of either end).
constexpr int kChunk = 256;               // outputs per chunk, eight per lane
constexpr int kRing = 2 * kChunk + 64;    // two chunk slots and the mirror of slot 0's first 64 words

// D[idx .. idx + 3] of the row, zeros past its end (n_t is a multiple of 4, so a
// quadruple lies wholly inside or wholly outside the row).
__device__ __forceinline__ uint4 load_quad(const int32_t* __restrict__ row, int idx, int n_t) {
  return idx < n_t ? __ldg(reinterpret_cast<const uint4*>(row + idx)) : make_uint4(0u, 0u, 0u, 0u);
}

// Asynchronous 16-byte copy of D[idx .. idx + 3] into shared memory, zeros
// past the row's end (the source is then not read).
__device__ __forceinline__ void copy_quad(uint32_t* dst, const int32_t* __restrict__ row, int idx, int n_t) {
  const bool in = idx < n_t;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(row + (in ? idx : 0)),
               "r"(in ? 16 : 0)
               : "memory");
}

// Chunk j's quadruples of this lane into staging slot j % 3 (nothing past
// chunk `last`); always one commit group, so that group counts stay uniform.
__device__ __forceinline__ void stage_chunk(uint32_t* stage, const int32_t* __restrict__ row, int j, int last,
                                            int n_t) {
  const int lane = threadIdx.x & 31;
  if (j <= last) {
    uint32_t* s = stage + (j % 3) * kChunk + 4 * lane;
    copy_quad(s, row, kChunk * j + 4 * lane, n_t);
    copy_quad(s + 128, row, kChunk * j + 128 + 4 * lane, n_t);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void wait_staged() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The lane's two staged quadruples of chunk j.
__device__ __forceinline__ void staged_quads(const uint32_t* stage, int j, uint4& a, uint4& b) {
  const uint32_t* s = stage + (j % 3) * kChunk + 4 * (threadIdx.x & 31);
  a = *reinterpret_cast<const uint4*>(s);
  b = *reinterpret_cast<const uint4*>(s + 128);
}

// Prefix sums of one chunk.  `a`, `b`: the lane's quadruples D[base + 4l ..] and
// D[base + 128 + 4l ..]; `run`: P at the chunk's first sample, advanced past the
// chunk.  p0[i] = P[base + 4l + i], p1[i] = P[base + 128 + 4l + i]; returns the
// chunk's sum (the same in every lane).
__device__ __forceinline__ uint32_t scan_chunk(const uint4& a, const uint4& b, uint32_t& run, uint4& p0, uint4& p1) {
  const int lane = threadIdx.x & 31;
  const uint32_t sa = a.x + a.y + a.z + a.w, sb = b.x + b.y + b.z + b.w;
  uint32_t xa = sa, xb = sb;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t ya = __shfl_up_sync(0xffffffffu, xa, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
    if (lane >= o) { xa += ya; xb += yb; }
  }
  const uint32_t ta = __shfl_sync(0xffffffffu, xa, 31), tb = __shfl_sync(0xffffffffu, xb, 31);
  p0.x = run + xa - sa;
  p0.y = p0.x + a.x;
  p0.z = p0.y + a.y;
  p0.w = p0.z + a.z;
  p1.x = run + ta + xb - sb;
  p1.y = p1.x + b.x;
  p1.z = p1.y + b.y;
  p1.w = p1.z + b.z;
  run += ta + tb;
  return ta + tb;
}

// Stores a scanned chunk in ring slot `slot` (and slot 0's mirror).
__device__ __forceinline__ void store_chunk(uint32_t* ring, int slot, const uint4& p0, const uint4& p1) {
  const int lane = threadIdx.x & 31;
  uint32_t* s = ring + slot * kChunk + 4 * lane;
  *reinterpret_cast<uint4*>(s) = p0;
  *reinterpret_cast<uint4*>(s + 128) = p1;
  if (slot == 0 && lane < 16) *reinterpret_cast<uint4*>(ring + 2 * kChunk + 4 * lane) = p0;
}



// Boxcars of one chunk for every width.  `ptr` = the chunk's slot + 4 lane;
// `c` the chunk index; `mc` (in shared memory, one word per width and lane)
// receives the chunk where the lane's maximum of a width first grew to its
// current value.  EDGE: some output of the chunk is not valid for some width
// (t + w > n_t): those are skipped.
template <int NW, bool EDGE>
__device__ __forceinline__ void chunk_boxcars(const uint32_t* ptr, int base, int n_t, int c,
                                              unsigned long long (&s2)[NW], int (&mx)[NW], int* mc) {
  const int lane = threadIdx.x & 31;
  const uint4 A0 = *reinterpret_cast<const uint4*>(ptr);
  const uint4 A1 = *reinterpret_cast<const uint4*>(ptr + 128);
  const uint4 N0 = *reinterpret_cast<const uint4*>(ptr + 4);
  const uint4 N1 = *reinterpret_cast<const uint4*>(ptr + 132);
#pragma unroll
  for (int k = 0; k < NW; k++) {
    const int w = 1 << k;
    uint4 Q0, Q1;
    if (w >= 8) {
      Q0 = *reinterpret_cast<const uint4*>(ptr + w);
      Q1 = *reinterpret_cast<const uint4*>(ptr + 128 + w);
    }
    int cm = -1;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const uint4& A = h ? A1 : A0;
      const uint4& N = h ? N1 : N0;
      const uint4& Q = h ? Q1 : Q0;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        // P[t + w] for t = base + 128 h + 4 lane + i
        const uint32_t hi = w >= 8 ? quad(Q, i) : (i + w < 4 ? quad(A, i + w) : quad(N, i + w - 4));
        const uint32_t B = hi - quad(A, i);
        if (EDGE) {
          const bool ok = base + 128 * h + 4 * lane + i + w <= n_t;
          add_square(s2[k], ok ? B : 0u);
          if (ok) cm = max(cm, (int)B);
        } else {
          add_square(s2[k], B);
          cm = max(cm, (int)B);
        }
      }
    }
    if (cm > mx[k]) {
      mx[k] = cm;
      mc[k * 32] = c;
    }
  }
}

// First sample t of chunk c whose width-w boxcar equals m (the row's maximum),
// found by one warp from D; the ring serves as its scratch.  Every lane returns it.
__device__ int first_in_chunk(const int32_t* __restrict__ row, int n_t, uint32_t* ring, int c, int w, int m) {
  const int lane = threadIdx.x & 31;
  const int base = kChunk * c;
  uint32_t run = 0u;
  uint4 p0, p1;
  scan_chunk(load_quad(row, base + 4 * lane, n_t), load_quad(row, base + 128 + 4 * lane, n_t), run, p0, p1);
  store_chunk(ring, 0, p0, p1);
  scan_chunk(load_quad(row, base + kChunk + 4 * lane, n_t), load_quad(row, base + kChunk + 128 + 4 * lane, n_t),
             run, p0, p1);
  store_chunk(ring, 1, p0, p1);
  __syncwarp();
  int first = 0x7fffffff;
#pragma unroll
  for (int h = 1; h >= 0; h--) {
#pragma unroll
    for (int i = 3; i >= 0; i--) {
      const int off = 128 * h + 4 * lane + i;
      const int t = base + off;
      if (t + w <= n_t && (int)(ring[off + w] - ring[off]) == m) first = t;
    }
  }
  first = __reduce_min_sync(0xffffffffu, first);
  __syncwarp();
  return first;
}

// Sum over the warp of a 64-bit value (every lane gets it).
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int NW>
__global__ void __launch_bounds__(kMaxThreads, 2) snr_stream_kernel(SnrArgs a) {
  constexpr int kWarps = kMaxThreads / 32;
  // per warp: a ring of prefix sums, three staging slots of D, NW x 32 first-chunk words
  extern __shared__ __align__(16) uint32_t dyn[];
  __shared__ unsigned long long ws2[kWarps][NW], wtot[kWarps], gs1[NW];
  __shared__ int wmx[kWarps][NW], gmax[NW], gchunk[NW], gfirst[NW];
  const int row = blockIdx.x, n_t = a.n_t;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int32_t* __restrict__ Drow = a.D + (int64_t)row * n_t;
  uint32_t* ring = dyn + warp * (kRing + 3 * kChunk + NW * 32);
  uint32_t* stage = ring + kRing;
  int* mc = reinterpret_cast<int*>(stage + 3 * kChunk) + lane;
  const int n_chunks = (n_t + kChunk - 1) / kChunk;
  const int cb = warp * n_chunks / nwarps, ce = (warp + 1) * n_chunks / nwarps;

  unsigned long long s2[NW];
  int mx[NW];
#pragma unroll
  for (int k = 0; k < NW; k++) { s2[k] = 0ull; mx[k] = -1; }
  if (threadIdx.x < NW) gchunk[threadIdx.x] = 0x7fffffff;
#pragma unroll
  for (int k = 0; k < NW; k++) mc[k * 32] = 0;
  unsigned long long tot = 0ull;  // the segment's sum
  if (cb < ce) {
    // chunks cb .. ce (ce: the lookahead) stream through three staging slots
    stage_chunk(stage, Drow, cb, ce, n_t);
    stage_chunk(stage, Drow, cb + 1, ce, n_t);
    stage_chunk(stage, Drow, cb + 2, ce, n_t);
    uint32_t run = 0u;
    uint4 da, db, p0, p1;
    wait_staged<2>();
    staged_quads(stage, cb, da, db);
    tot += scan_chunk(da, db, run, p0, p1);
    store_chunk(ring, cb & 1, p0, p1);
    for (int c = cb; c < ce; c++) {
      // chunk c + 1 (the lookahead past the segment's end included) into the other slot
      wait_staged<1>();
      staged_quads(stage, c + 1, da, db);
      const uint32_t ct = scan_chunk(da, db, run, p0, p1);
      if (c + 1 < ce) tot += ct;
      store_chunk(ring, (c + 1) & 1, p0, p1);
      stage_chunk(stage, Drow, c + 3, ce, n_t);  // into chunk c's staging slot, read before
      __syncwarp();
      const int base = kChunk * c;
      const uint32_t* ptr = ring + (c & 1) * kChunk + 4 * lane;
      if (base + kChunk - 1 + (1 << (NW - 1)) <= n_t)
        chunk_boxcars<NW, false>(ptr, base, n_t, c, s2, mx, mc);
      else
        chunk_boxcars<NW, true>(ptr, base, n_t, c, s2, mx, mc);
      __syncwarp();  // slot c & 1 is rewritten next
    }
    wait_staged<0>();
  }
  // the warp's moments and maxima
#pragma unroll
  for (int k = 0; k < NW; k++) {
    const unsigned long long v2 = warp_sum64(s2[k]);
    const int m = __reduce_max_sync(0xffffffffu, mx[k]);
    if (lane == 0) { ws2[warp][k] = v2; wmx[warp][k] = m; }
  }
  if (lane == 0) wtot[warp] = tot;
  __syncthreads();
  if (threadIdx.x < NW) {
    const int k = threadIdx.x;
    int m = wmx[0][k];
    for (int q = 1; q < nwarps; q++) m = max(m, wmx[q][k]);
    gmax[k] = m;
  }
  __syncthreads();
  // the earliest chunk holding each width's maximum
#pragma unroll
  for (int k = 0; k < NW; k++)
    if (mx[k] == gmax[k]) atomicMin(&gchunk[k], mc[k * 32]);
  __syncthreads();
  for (int k = warp; k < NW; k += nwarps) {
    // (every width has a valid output: the plan keeps widths within the row)
    const int f = gchunk[k] >= 0 && gchunk[k] < n_chunks
                      ? first_in_chunk(Drow, n_t, ring, gchunk[k], 1 << k, gmax[k]) : 0;
    if (lane == 0) gfirst[k] = f;
  }
  if (warp == nwarps - 1) {
    // S1 from the row total and the samples within 63 of either end
    unsigned long long T = 0ull;
    for (int q = 0; q < nwarps; q++) T += wtot[q];
    uint32_t lo[2], hi[2];
#pragma unroll
    for (int j = 0; j < 2; j++) {
      const int u = lane + 32 * j, v = n_t - 64 + lane + 32 * j;
      lo[j] = u < n_t ? (uint32_t)__ldg(Drow + u) : 0u;
      hi[j] = v >= 0 ? (uint32_t)__ldg(Drow + v) : 0u;
    }
#pragma unroll
    for (int k = 0; k < NW; k++) {
      const int w = 1 << k;
      unsigned long long e = 0ull;
#pragma unroll
      for (int j = 0; j < 2; j++) {
        const int u = lane + 32 * j, v = n_t - 64 + lane + 32 * j;
        if (u < w - 1) e += (unsigned long long)(w - 1 - u) * lo[j];
        if (v >= 0 && v > n_t - w) e += (unsigned long long)(v - n_t + w) * hi[j];
      }
      e = warp_sum64(e);
      if (lane == 0) gs1[k] = (unsigned long long)w * T - e;
    }
  }
  __syncthreads();
  if (threadIdx.x < NW) {
    const int k = threadIdx.x;
    unsigned long long v2 = 0ull;
    for (int q = 0; q < nwarps; q++) v2 += ws2[q][k];
    const Moments r{gs1[k], v2, 0ull, gmax[k], 0};
    const int64_t o = (int64_t)k * a.n_dms + row;
    a.snr[o] = snr_from_moments(n_t - (1 << k) + 1, r);
    a.peak_t[o] = gfirst[k];
    a.peak_val[o] = gmax[k];
  }
}


size_t prefix_smem(int n_t) { return ((size_t)n_t + kPad + 3) / 4 * 4 * sizeof(uint32_t); }

bool tma_ok(const int32_t* D, int n_t) { return ((uintptr_t)D & 15) == 0 && (n_t & 3) == 0; }

bool row_fits(int n_t, size_t extra) {
  int dev = 0, max_smem = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  return prefix_smem(n_t) + extra <= (size_t)max_smem;
}

sps_status check_row_fits(int n_t, size_t extra) {
  int dev = 0, max_smem = 0;
  SPS_CUDA(cudaGetDevice(&dev));
  SPS_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (prefix_smem(n_t) + extra > (size_t)max_smem)
    return fail(SPS_ERR_UNSUPPORTED, "rows too long for the shared-memory prefix");
  return SPS_OK;
}

}  // namespace

bool snr_config_supported(const sps_snr_config& c, std::string* why) {
  if (c.threads < 32 || c.threads > kMaxThreads || (c.threads & 31)) {
    *why = "threads must be a multiple of 32 in [32, 512]";
    return false;
  }
  return true;
}

typedef void (*SnrKernel)(SnrArgs, int, int, int, int);

template <bool DEC, bool FAST>
SnrKernel snr_variant(int nwp) {
  switch (nwp) {
    case 1: return snr_kernel<1, DEC, FAST>;
    case 2: return snr_kernel<2, DEC, FAST>;
    case 3: return snr_kernel<3, DEC, FAST>;
    case 4: return snr_kernel<4, DEC, FAST>;
    case 5: return snr_kernel<5, DEC, FAST>;
    case 6: return snr_kernel<6, DEC, FAST>;
    case 7: return snr_kernel<7, DEC, FAST>;
    default: return snr_kernel<8, DEC, FAST>;
  }
}

typedef void (*Pow2Kernel)(SnrArgs);

Pow2Kernel pow2_variant(int nw) {
  switch (nw) {
    case 1: return snr_pow2_kernel<1>;
    case 2: return snr_pow2_kernel<2>;
    case 3: return snr_pow2_kernel<3>;
    case 4: return snr_pow2_kernel<4>;
    case 5: return snr_pow2_kernel<5>;
    case 6: return snr_pow2_kernel<6>;
    default: return snr_pow2_kernel<7>;
  }
}

// The vector kernel serves sliding boxcars of widths 1, 2, ..., 2^(NW-1)
// (NW <= 7) on rows that a bulk copy can stage (16-byte aligned, a multiple
// of 4 samples) whose sums of squares fit 64 bits; it has no decimating form.
bool pow2_form(const SnrArgs& a) {
  if (a.decimate || a.pow2_widths < 1 || a.pow2_widths > 7 || !tma_ok(a.D, a.n_t)) return false;
  const long double bmax = (long double)std::max<int64_t>(1, a.max_boxcar);
  return (long double)a.n_t * bmax * bmax < 1.8e19L;
}

// Bytes of the row buffer: the groups' quadruples and the widest width's reach.
size_t pow2_smem(int n_t, int nw) {
  const int n_grp = (n_t + 6) / 4;
  return ((size_t)4 * n_grp + 4 + (1 << (nw - 1)) + 4) * sizeof(uint32_t);
}

typedef void (*StreamKernel)(SnrArgs);

StreamKernel stream_variant(int nw) {
  switch (nw) {
    case 1: return snr_stream_kernel<1>;
    case 2: return snr_stream_kernel<2>;
    case 3: return snr_stream_kernel<3>;
    case 4: return snr_stream_kernel<4>;
    case 5: return snr_stream_kernel<5>;
    case 6: return snr_stream_kernel<6>;
    default: return snr_stream_kernel<7>;
  }
}

// The streaming form also needs each 256-sample chunk's sum to fit 32 bits.
bool stream_form(const SnrArgs& a) {
  const long double bmax = (long double)std::max<int64_t>(1, a.max_boxcar);
  const long double smax = bmax / (long double)(1 << (a.pow2_widths - 1));  // largest sample
  return smax * kChunk < 4.2e9L;
}

// Shared memory of the streaming kernel: per warp a ring, three staging slots
// and NW x 32 first-chunk words.
size_t stream_smem(int nw, int threads) {
  return (size_t)(threads / 32) * (kRing + 3 * kChunk + nw * 32) * sizeof(uint32_t);
}

sps_status launch_snr(const SnrArgs& a, const sps_snr_config& c, cudaStream_t st) {
  std::string why;
  if (!snr_config_supported(c, &why)) return fail(SPS_ERR_INVALID_ARG, why);
  if (pow2_form(a) && !row_fits(a.n_t, pow2_smem(a.n_t, a.pow2_widths) - prefix_smem(a.n_t) + 8192) &&
      stream_form(a)) {
    // rows too long to stage whole: the streaming form, any row length
    const size_t smem = stream_smem(a.pow2_widths, c.threads);
    StreamKernel fn = stream_variant(a.pow2_widths);
    SPS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    fn<<<a.n_dms, c.threads, smem, st>>>(a);
    SPS_CUDA(cudaGetLastError());
    if (a.best && (int64_t)a.n_widths * a.n_dms >= (int64_t)1 << 31)
      return fail(SPS_ERR_UNSUPPORTED, "S/N table too large for the detection's 32-bit indices");
    if (a.best) {
      detect_kernel<<<kDetectBlocks, kDetectThreads, 0, st>>>(a.snr, a.peak_t, a.peak_val, a.n_dms, a.n_widths,
                                                              a.best);
      SPS_CUDA(cudaGetLastError());
    }
    return SPS_OK;
  }
  if (pow2_form(a)) {
    const size_t smem = pow2_smem(a.n_t, a.pow2_widths);
    if (sps_status s = check_row_fits(a.n_t, smem - prefix_smem(a.n_t) + 8192)) return s;
    Pow2Kernel fn = pow2_variant(a.pow2_widths);
    SPS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    fn<<<a.n_dms, c.threads, smem, st>>>(a);
    SPS_CUDA(cudaGetLastError());
    if (a.best && (int64_t)a.n_widths * a.n_dms >= (int64_t)1 << 31)
      return fail(SPS_ERR_UNSUPPORTED, "S/N table too large for the detection's 32-bit indices");
    if (a.best) {
      detect_kernel<<<kDetectBlocks, kDetectThreads, 0, st>>>(a.snr, a.peak_t, a.peak_val, a.n_dms, a.n_widths,
                                                              a.best);
      SPS_CUDA(cudaGetLastError());
    }
    return SPS_OK;
  }
  if (sps_status s = check_row_fits(a.n_t, sizeof(Moments) * (kMaxThreads / 32) * kWidthsPerPass + 512)) return s;
  // largest boxcar value: 255 * channels * widest width (< 2^31, checked by the plan);
  // a thread's 64-bit S2 partial takes `flush` squares before it must be flushed
  const unsigned long long bmax = std::max<unsigned long long>(1ull, (unsigned long long)a.max_boxcar);
  const unsigned long long f2 = 0xFFFFFFFFFFFFFFFFull / (bmax * bmax);
  const int flush = (int)std::max<unsigned long long>(1ull, std::min<unsigned long long>(f2, 1ull << 30));
  // a warp's S2: 32 threads x ceil(n_t / threads) samples x bmax^2, in 64 bits?
  const unsigned long long per_thread = (unsigned long long)((a.n_t + c.threads - 1) / c.threads);
  const long double warp_s2 = 32.0L * (long double)per_thread * (long double)bmax * (long double)bmax;
  const int narrow = warp_s2 < 1.8e19L ? 1 : 0;
  // no thread ever flushes: its sample count stays within `flush`
  const bool fast = narrow && per_thread <= (unsigned long long)flush;
  const size_t smem = prefix_smem(a.n_t);
  for (int w0 = 0; w0 < a.n_widths; w0 += kWidthsPerPass) {
    const int nwp = std::min(kWidthsPerPass, a.n_widths - w0);
    SnrKernel fn = a.decimate ? (fast ? snr_variant<true, true>(nwp) : snr_variant<true, false>(nwp))
                              : (fast ? snr_variant<false, true>(nwp) : snr_variant<false, false>(nwp));
    SPS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    fn<<<a.n_dms, c.threads, smem, st>>>(a, w0, flush, tma_ok(a.D, a.n_t) ? 1 : 0, narrow);
    SPS_CUDA(cudaGetLastError());
  }
  if (a.best) {
    detect_kernel<<<kDetectBlocks, kDetectThreads, 0, st>>>(a.snr, a.peak_t, a.peak_val, a.n_dms, a.n_widths,
                                                            a.best);
    SPS_CUDA(cudaGetLastError());
  }
  return SPS_OK;
}

sps_status launch_integrate(const int32_t* D, int32_t n_dms, int32_t n_t, const int32_t* widths,
                            int32_t n_widths, int32_t decimate, int32_t* B, uint32_t* status, cudaStream_t st) {
  if (sps_status s = check_row_fits(n_t, 256)) return s;
  const size_t smem = prefix_smem(n_t);
  SPS_CUDA(cudaFuncSetAttribute(integrate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  integrate_kernel<<<n_dms, 256, smem, st>>>(D, n_dms, n_t, widths, n_widths, B, tma_ok(D, n_t) ? 1 : 0, decimate,
                                             status);
  SPS_CUDA(cudaGetLastError());
  return SPS_OK;
}

}  // namespace sps
