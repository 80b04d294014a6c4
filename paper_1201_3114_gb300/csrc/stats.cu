// stats.cu -- byte statistics of a device buffer for the ciphertext
// analysis of Sec. 4: the frequency histogram (Fig. 2), from which the
// Shannon entropy follows, and the lagged products behind the
// auto-correlation of Fig. 3.  Every quantity is an exact integer sum, so
// the result does not depend on the order in which threads add.
//
// One pass over the data.  Each CTA keeps a private histogram in shared
// memory (one copy per warp, against contention on the same bins), reads its
// tile with 16-byte loads, forms the sums of products four bytes at a time
// with the unsigned 4-way byte dot product (__dp4a), and adds its partial
// sums to the global 64-bit totals with one atomic per bin and per sum.
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
    // 32-bit partial sums per tile: a thread adds at most 16 groups of 16
    // bytes per tile, so every partial stays below 256 * 255^2 < 2^32.
    uint32_t t1 = 0, t2 = 0;
    uint32_t tl[LC_STATS_MAX_LAG];
#pragma unroll
    for (int k = 0; k < LC_STATS_MAX_LAG; k++) tl[k] = 0;
    // each thread takes 16 consecutive bytes at a time, as 4 words, plus the
    // next 8 bytes (2 words) for the lagged products; bytes at or past the
    // end of the data read as 0 and add nothing
    for (uint64_t i = base + 16ull * threadIdx.x; i < end; i += 16ull * kThreads) {
      uint32_t w[6];
      const uint64_t cnt = end - i < 16 ? end - i : 16;
      const bool aligned = (reinterpret_cast<uintptr_t>(data + i) & 15u) == 0;
      if (cnt == 16 && aligned) {
        const uint4 q = *reinterpret_cast<const uint4*>(data + i);
        w[0] = q.x;
        w[1] = q.y;
        w[2] = q.z;
        w[3] = q.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; j++) {
          uint32_t v = 0;
#pragma unroll
          for (int b = 0; b < 4; b++)
            if (4 * j + b < (int)cnt) v |= (uint32_t)data[i + 4 * j + b] << (8 * b);
          w[j] = v;
        }
      }
      if (aligned && i + 24 <= n) {
        const uint2 h = *reinterpret_cast<const uint2*>(data + i + 16);
        w[4] = h.x;
        w[5] = h.y;
      } else {
#pragma unroll
        for (int j = 4; j < 6; j++) {
          uint32_t v = 0;
#pragma unroll
          for (int b = 0; b < 4; b++)
            if (i + 4 * j + b < n) v |= (uint32_t)data[i + 4 * j + b] << (8 * b);
          w[j] = v;
        }
      }
#pragma unroll
      for (int j = 0; j < 4; j++) {
        t1 = __dp4a(w[j], 0x01010101u, t1);
        t2 = __dp4a(w[j], w[j], t2);
#pragma unroll
        for (int k = 1; k <= LC_STATS_MAX_LAG; k++) {
          // the word of bytes x_{4j+k} .. x_{4j+k+3}
          const int wi = j + (k >> 2), sh = 8 * (k & 3);
          const uint32_t sw = sh ? __funnelshift_r(w[wi], w[wi + 1], sh) : w[wi];
          tl[k - 1] = __dp4a(w[j], sw, tl[k - 1]);
        }
#pragma unroll
        for (int b = 0; b < 4; b++)
          if (4 * j + b < (int)cnt) atomicAdd(&hist[warp][(w[j] >> (8 * b)) & 255u], 1u);
      }
    }
    s1 += t1;
    s2 += t2;
#pragma unroll
    for (int k = 0; k < LC_STATS_MAX_LAG; k++) lag[k] += tl[k];
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
