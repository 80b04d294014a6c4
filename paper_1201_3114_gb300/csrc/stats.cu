// stats.cu -- byte statistics of a device buffer for the ciphertext
// analysis of Sec. 4: the frequency histogram (Fig. 2), from which the
// Shannon entropy follows, and the lagged products behind the
// auto-correlation of Fig. 3.  Every quantity is an exact integer sum, so
// the result does not depend on the order in which threads add.
//
// One pass over the data.  Each CTA keeps a private histogram in shared
// memory laid out as [bin][lane]: lane l of every warp counts into column l,
// so the 32 atomics of a warp instruction always fall in 32 different banks.
// Threads read 32 consecutive bytes per iteration with 16-byte loads (plus
// the next 8 bytes for the lagged products), form the sums of products four
// bytes at a time with the unsigned 4-way byte dot product (__dp4a), and add
// their partial sums to the global 64-bit totals once per CTA at the end.
// The sum and the sum of squares are not accumulated here: they follow
// exactly from the histogram (the host forms them).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lc.h"

namespace lc {

namespace {

constexpr int kThreads = 256;
constexpr uint32_t kChunk = 32;                          // bytes per thread per iteration
constexpr uint64_t kTile = 8ull * kChunk * kThreads;     // 64 KiB per CTA per tile

// Bytes i .. i + 3 of data as a little-endian word, 0 for bytes at or past
// n (only for the ragged end of the buffer).
__device__ __forceinline__ uint32_t guarded_word(const uint8_t* data, uint64_t i, uint64_t n) {
  uint32_t v = 0;
#pragma unroll
  for (int b = 0; b < 4; b++)
    if (i + b < n) v |= (uint32_t)data[i + b] << (8 * b);
  return v;
}

// acc layout (uint64): [0, 256) histogram, 256 and 257 unused (zero),
// 258 + k - 1 for lag k = 1..max_lag: sum of x_i x_{i+k}.
//
// `data` here is 16-byte aligned; the caller's unaligned head is counted by
// thread 0 of CTA 0 from `head` (h bytes before data).
template <bool kLags>
__global__ void __launch_bounds__(kThreads) stats_kernel(const uint8_t* __restrict__ head, uint32_t h,
                                                         const uint8_t* __restrict__ data, uint64_t m,
                                                         uint32_t max_lag, unsigned long long* acc) {
  __shared__ uint32_t hist[256 * 32];
  for (int i = threadIdx.x; i < 256 * 32; i += kThreads) hist[i] = 0u;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t* const hl = hist + lane;
  uint64_t lag[LC_STATS_MAX_LAG];
#pragma unroll
  for (int k = 0; k < LC_STATS_MAX_LAG; k++) lag[k] = 0;

  // The unaligned head: at most 15 bytes, each with its lagged partners,
  // which may lie in the aligned part.
  if (h && blockIdx.x == 0 && threadIdx.x == 0) {
    for (uint32_t i = 0; i < h; i++) {
      const uint32_t x = head[i];
      atomicAdd(&hl[x * 32u], 1u);
      if (kLags) {
        for (uint32_t k = 1; k <= LC_STATS_MAX_LAG; k++) {
          const uint64_t j = (uint64_t)i + k;  // position in head + data
          uint32_t y = 0;
          if (j < h) y = head[j];
          else if (j - h < m) y = data[j - h];
          lag[k - 1] += (uint64_t)x * y;
        }
      }
    }
  }

  for (uint64_t base = (uint64_t)blockIdx.x * kTile; base < m; base += (uint64_t)gridDim.x * kTile) {
    const uint64_t end = base + kTile < m ? base + kTile : m;
    // 32-bit partial sums per tile: a thread adds 8 chunks of 32 bytes per
    // tile, so every partial stays below 256 * 255^2 < 2^32.
    uint32_t tl[LC_STATS_MAX_LAG];
#pragma unroll
    for (int k = 0; k < LC_STATS_MAX_LAG; k++) tl[k] = 0;
    for (uint64_t i = base + (uint64_t)kChunk * threadIdx.x; i < end; i += (uint64_t)kChunk * kThreads) {
      uint32_t w[10];
      const bool full = i + kChunk <= end;
      if (full) {
        const uint4 a = *reinterpret_cast<const uint4*>(data + i);
        const uint4 b = *reinterpret_cast<const uint4*>(data + i + 16);
        w[0] = a.x, w[1] = a.y, w[2] = a.z, w[3] = a.w;
        w[4] = b.x, w[5] = b.y, w[6] = b.z, w[7] = b.w;
#pragma unroll
        for (int j = 0; j < 8; j++) {
          // address of bin x, column lane: x * 32 + lane words
          atomicAdd(&hl[(w[j] & 255u) << 5], 1u);
          atomicAdd(&hl[((w[j] >> 8) & 255u) << 5], 1u);
          atomicAdd(&hl[((w[j] >> 16) & 255u) << 5], 1u);
          atomicAdd(&hl[(w[j] >> 24) << 5], 1u);
        }
      } else {
        // the ragged end of the buffer: bytes at or past m read as 0 and
        // are not counted
#pragma unroll
        for (int j = 0; j < 8; j++) w[j] = guarded_word(data, i + 4 * j, m);
        for (uint32_t q = 0; q < kChunk && i + q < m; q++)
          atomicAdd(&hl[((w[q >> 2] >> (8 * (q & 3))) & 255u) << 5], 1u);
      }
      if (kLags) {
        if (i + kChunk + 8 <= m) {
          const uint2 c = *reinterpret_cast<const uint2*>(data + i + kChunk);
          w[8] = c.x, w[9] = c.y;
        } else {
          w[8] = guarded_word(data, i + kChunk, m);
          w[9] = guarded_word(data, i + kChunk + 4, m);
        }
        // sh[s][j]: the word of bytes x_{4j+s} .. x_{4j+s+3}, s = 1..3;
        // lag k + 4 reuses the shifted word of index j + 1.
        uint32_t sh1[9], sh2[9], sh3[9];
#pragma unroll
        for (int j = 0; j < 9; j++) {
          sh1[j] = __funnelshift_r(w[j], w[j + 1], 8);
          sh2[j] = __funnelshift_r(w[j], w[j + 1], 16);
          sh3[j] = __funnelshift_r(w[j], w[j + 1], 24);
        }
#pragma unroll
        for (int j = 0; j < 8; j++) {
          tl[0] = __dp4a(w[j], sh1[j], tl[0]);
          tl[1] = __dp4a(w[j], sh2[j], tl[1]);
          tl[2] = __dp4a(w[j], sh3[j], tl[2]);
          tl[3] = __dp4a(w[j], w[j + 1], tl[3]);
          tl[4] = __dp4a(w[j], sh1[j + 1], tl[4]);
          tl[5] = __dp4a(w[j], sh2[j + 1], tl[5]);
          tl[6] = __dp4a(w[j], sh3[j + 1], tl[6]);
          tl[7] = __dp4a(w[j], w[j + 2], tl[7]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < LC_STATS_MAX_LAG; k++) lag[k] += tl[k];
  }
  __syncthreads();
  // bin b: the 32 columns, read starting at a thread-dependent column so the
  // threads of a warp hit different banks
  for (uint32_t b = threadIdx.x; b < 256; b += kThreads) {
    uint64_t t = 0;
    for (uint32_t c = 0; c < 32; c++) t += hist[b * 32u + ((c + b) & 31u)];
    if (t) atomicAdd(acc + b, (unsigned long long)t);
  }
  // warp-reduce the lagged sums, then one atomic per warp and lag
  if (kLags) {
    for (int off = 16; off; off >>= 1) {
#pragma unroll
      for (int k = 0; k < LC_STATS_MAX_LAG; k++) lag[k] += __shfl_down_sync(0xFFFFFFFFu, lag[k], off);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < LC_STATS_MAX_LAG; k++)
        if (k < (int)max_lag) atomicAdd(acc + 258 + k, (unsigned long long)lag[k]);
    }
  }
}

}  // namespace

cudaError_t launch_stats(const uint8_t* data, uint64_t n, uint32_t max_lag, unsigned long long* acc,
                         int sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc, 0, (258 + LC_STATS_MAX_LAG) * sizeof(unsigned long long), s);
  if (e != cudaSuccess || n == 0) return e;
  const uint64_t mis = reinterpret_cast<uintptr_t>(data) & 15u;
  const uint32_t h = (uint32_t)(mis ? (16u - mis < n ? 16u - mis : n) : 0u);
  const uint8_t* body = data + h;
  const uint64_t m = n - h;
  const uint64_t tiles = (m + kTile - 1) / kTile;
  // one wave of resident CTAs: equal shares of tiles, no second wave
  const void* fn = max_lag ? reinterpret_cast<const void*>(&stats_kernel<true>)
                           : reinterpret_cast<const void*>(&stats_kernel<false>);
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0);
  if (e != cudaSuccess) return e;
  uint64_t grid = (uint64_t)sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
  if (tiles < grid) grid = tiles;
  if (grid == 0) grid = 1;
  if (max_lag)
    stats_kernel<true><<<(unsigned)grid, kThreads, 0, s>>>(data, h, body, m, max_lag, acc);
  else
    stats_kernel<false><<<(unsigned)grid, kThreads, 0, s>>>(data, h, body, m, max_lag, acc);
  return cudaGetLastError();
}

}  // namespace lc
