// stats.cu -- byte statistics of a device buffer for the ciphertext
// analysis of Sec. 4: the frequency histogram (Fig. 2), from which the
// Shannon entropy follows, and the lagged products behind the
// auto-correlation of Fig. 3.  Every quantity is an exact integer sum, so
// the result does not depend on the order in which threads add.
//
// One pass over the data: HBM-bound.  Each CTA keeps a private histogram in
// shared memory (one copy per warp, against contention on the same bins),
// reads its tile with 16-byte loads, and adds its partial sums to the
// global 64-bit totals with one atomic per bin and per sum.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lc.h"

namespace lc {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint64_t kTile = 64 * 1024;  // bytes per CTA per iteration

// acc layout (uint64): [0, 256) histogram, 256 sum, 257 sum of squares,
// 258 + k - 1 for lag k = 1..max_lag: sum of x_i x_{i+k}
__global__ void __launch_bounds__(kThreads) stats_kernel(const uint8_t* __restrict__ data, uint64_t n,
                                                         uint32_t max_lag, unsigned long long* acc) {
  __shared__ uint32_t hist[kWarps][256];
  const int warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * 256; i += kThreads) (&hist[0][0])[i] = 0u;
  __syncthreads();
  uint64_t s1 = 0, s2 = 0;
  uint64_t lag[LC_STATS_MAX_LAG];
#pragma unroll
  for (int k = 0; k < LC_STATS_MAX_LAG; k++) lag[k] = 0;

  for (uint64_t base = (uint64_t)blockIdx.x * kTile; base < n; base += (uint64_t)gridDim.x * kTile) {
    const uint64_t end = base + kTile < n ? base + kTile : n;
    // each thread takes 16 consecutive bytes at a time
    for (uint64_t i = base + 16ull * threadIdx.x; i < end; i += 16ull * kThreads) {
      uint8_t v[16 + LC_STATS_MAX_LAG];
      const uint64_t cnt = end - i < 16 ? end - i : 16;
      if (cnt == 16 && ((reinterpret_cast<uintptr_t>(data + i) & 15u) == 0)) {
        const uint4 q = *reinterpret_cast<const uint4*>(data + i);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = (uint8_t)(w[j >> 2] >> (8 * (j & 3)));
      } else {
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = j < (int)cnt ? data[i + j] : 0;
      }
      // the bytes after this group, for the lagged products (may cross tiles)
#pragma unroll
      for (int k = 0; k < LC_STATS_MAX_LAG; k++) {
        const uint64_t p = i + 16 + k;
        v[16 + k] = (k < (int)max_lag && p < n) ? data[p] : 0;
      }
#pragma unroll
      for (int j = 0; j < 16; j++) {
        if (j < (int)cnt) {
          const uint32_t x = v[j];
          atomicAdd(&hist[warp][x], 1u);
          s1 += x;
          s2 += x * x;
#pragma unroll
          for (int k = 0; k < LC_STATS_MAX_LAG; k++) {
            // x_{i+j} x_{i+j+k+1}; bytes past the end were read as 0
            lag[k] += (k < (int)max_lag) ? (uint64_t)(x * (uint32_t)v[j + k + 1]) : 0ull;
          }
        }
      }
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += kThreads) {
    uint64_t t = 0;
    for (int w = 0; w < kWarps; w++) t += hist[w][b];
    if (t) atomicAdd(acc + b, (unsigned long long)t);
  }
  // warp-reduce the scalar sums, then one atomic per warp
  for (int off = 16; off; off >>= 1) {
    s1 += __shfl_down_sync(0xFFFFFFFFu, s1, off);
    s2 += __shfl_down_sync(0xFFFFFFFFu, s2, off);
#pragma unroll
    for (int k = 0; k < LC_STATS_MAX_LAG; k++) lag[k] += __shfl_down_sync(0xFFFFFFFFu, lag[k], off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc + 256, (unsigned long long)s1);
    atomicAdd(acc + 257, (unsigned long long)s2);
#pragma unroll
    for (int k = 0; k < LC_STATS_MAX_LAG; k++)
      if (k < (int)max_lag) atomicAdd(acc + 258 + k, (unsigned long long)lag[k]);
  }
}

}  // namespace

cudaError_t launch_stats(const uint8_t* data, uint64_t n, uint32_t max_lag, unsigned long long* acc,
                         int sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc, 0, (258 + LC_STATS_MAX_LAG) * sizeof(unsigned long long), s);
  if (e != cudaSuccess || n == 0) return e;
  uint64_t tiles = (n + kTile - 1) / kTile;
  uint64_t grid = (uint64_t)sms * 4;
  if (tiles < grid) grid = tiles;
  stats_kernel<<<(unsigned)grid, kThreads, 0, s>>>(data, n, max_lag, acc);
  return cudaGetLastError();
}

}  // namespace lc
