// stats.cu -- byte statistics of a device buffer for the ciphertext
// analysis of Sec. 4: the frequency histogram (Fig. 2), from which the
// Shannon entropy follows, and the lagged products behind the
// auto-correlation of Fig. 3.  Every quantity is an exact integer sum, so
// the result does not depend on the order in which threads add.
//
// One pass over the data, bound by HBM bandwidth in principle and, on
// GB300, by the shared-memory atomics of the histogram (one per byte: the
// SM retires about one warp-wide shared atomic per two cycles) and the
// integer work of the lagged products.  Each CTA keeps a private histogram
// in shared memory laid out as [bin][column], one column per lane and warp
// parity, so the 32 atomics of a warp instruction always fall in 32
// different banks.  Each thread reads 32-byte chunks (and, for the lagged
// products, the 8 bytes after each) straight from global memory with
// 16-byte loads, issuing the next chunk's loads before it counts the
// current one; the lagged sums are formed four bytes at a time with the
// unsigned 4-way byte dot product (__dp4a).  The ragged end of the buffer is
// read with guarded loads.  The sum and the sum of squares are not
// accumulated here: they follow exactly from the histogram (the host forms
// them).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lc.h"

namespace lc {

namespace {

constexpr uint32_t kChunk = 32;  // bytes per thread and count step

// The CTA's histogram, 64 KiB at the start of dynamic shared memory,
// [bin][column] with 64 columns: the counter of bin x in column c sits at
// byte offset (x << 8) | (c << 2), and lane l of warp w counts into column
// l + 32 (w mod 2).  The bin is byte 1 of the offset and the column byte 0,
// so one byte permute of the data word forms each count's offset.  (A
// 32-column layout with a 128-byte bin stride halves the memory but needs a
// shift and an and-or per byte; on GB300 it was 5-6 % slower.)
extern __shared__ __align__(128) uint8_t dyn_smem[];

struct Hist {
  static constexpr uint32_t kCols = 64;
  static constexpr size_t kBytes = (size_t)256 * kCols * 4;

  __device__ __forceinline__ static uint32_t* words() { return reinterpret_cast<uint32_t*>(dyn_smem); }
  // this thread's column, as a byte offset (< 256)
  __device__ __forceinline__ static uint32_t col4() {
    return ((((threadIdx.x >> 5) & 1u) << 5) | (threadIdx.x & 31u)) << 2;
  }
  __device__ __forceinline__ static void count_at(uint32_t off) {
    atomicAdd(reinterpret_cast<uint32_t*>(dyn_smem + off), 1u);
  }
  // one byte x < 256
  __device__ __forceinline__ static void count(uint32_t x, uint32_t col) { count_at((x << 8) | col); }
  // the 32 bytes w[0..7]; col = col4()
  __device__ __forceinline__ static void chunk(uint32_t col, const uint32_t (&w)[10]) {
#pragma unroll
    for (int j = 0; j < 8; j++) {
      // offset byte 0 = the column (byte 0 of col), byte 1 = byte k of w[j],
      // bytes 2-3 = byte 1 of col (zero)
      count_at(__byte_perm(w[j], col, 0x5504u));
      count_at(__byte_perm(w[j], col, 0x5514u));
      count_at(__byte_perm(w[j], col, 0x5524u));
      count_at(__byte_perm(w[j], col, 0x5534u));
    }
  }
  __device__ __forceinline__ static void clear(int nthreads) {
    uint32_t* const h = words();
    for (int i = threadIdx.x; i < (int)(256 * kCols); i += nthreads) h[i] = 0u;
  }
  // after a barrier: add bin b's columns into acc[b], starting at a
  // bin-dependent column so the threads of a warp hit different banks
  __device__ __forceinline__ static void flush(unsigned long long* acc, int nthreads) {
    const uint32_t* const h = words();
    for (uint32_t b = threadIdx.x; b < 256; b += nthreads) {
      uint64_t t = 0;
      for (uint32_t c = 0; c < kCols; c++) t += h[b * kCols + ((c + b) & (kCols - 1u))];
      if (t) atomicAdd(acc + b, (unsigned long long)t);
    }
  }
};

// Launch shapes, chosen by measurement on GB300 (1 GiB, ms): histogram only
// 768 threads x 2 CTAs per SM 0.204 (1024 x 1: 0.205, 512 x 2: 0.216); with
// 8 lags 512 x 2 0.266 (768 x 2: 0.270, 1024 x 1: 0.266-0.278).
constexpr int kHistThreads = 768, kHistMinBlocks = 2;
constexpr int kLagThreads = 512, kLagMinBlocks = 2;

// Bytes i .. i + 3 of data as a little-endian word, 0 for bytes at or past
// n (only for the ragged end of the buffer).
__device__ __forceinline__ uint32_t guarded_word(const uint8_t* data, uint64_t i, uint64_t n) {
  uint32_t v = 0;
#pragma unroll
  for (int b = 0; b < 4; b++)
    if (i + b < n) v |= (uint32_t)data[i + b] << (8 * b);
  return v;
}

// Lagged products x_i x_{i+k}, k = 1..8, of the 32 bytes w[0..7] with their
// 8 successors w[8], w[9], into 32-bit partials.
__device__ __forceinline__ void lags_chunk(const uint32_t (&w)[10], uint32_t (&tl)[LC_STATS_MAX_LAG]) {
  // sh[s][j]: the word of bytes x_{4j+s} .. x_{4j+s+3}, s = 1..3; lag k + 4
  // reuses the shifted word of index j + 1.
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

// acc layout (uint64): [0, 256) histogram, 256 and 257 unused, 258 + k - 1
// for lag k = 1..max_lag: sum of x_i x_{i+k}.
//
// `data` here is 16-byte aligned; the caller's unaligned head is counted by
// thread 0 of CTA 0 from `head` (h bytes before data).  Chunk c reads bytes
// [32c, 32c + 40) of the aligned part: chunks [0, nchunks) lie, with their
// 8 successors, inside it; the rest is counted by the last CTA with guarded
// loads.  The lagged sums stay in 32-bit registers and reach the 64-bit
// totals by global atomics: every 1024 chunks (a chunk adds less than 2^21
// per lag) and at the end, warp-reduced.
template <bool kLags, int kThreads, int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks) stats_kernel(
    const uint8_t* __restrict__ head, uint32_t h, const uint8_t* __restrict__ data, uint64_t m,
    uint64_t nchunks, uint32_t max_lag, unsigned long long* acc) {
  Hist::clear(kThreads);
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t col = Hist::col4();
  uint32_t tl[LC_STATS_MAX_LAG];
#pragma unroll
  for (int k = 0; k < LC_STATS_MAX_LAG; k++) tl[k] = 0;

  if (h && blockIdx.x == 0 && threadIdx.x == 0) {
    // the unaligned head (< 16 bytes), with partners in the aligned part
    for (uint32_t i = 0; i < h; i++) {
      const uint32_t x = head[i];
      Hist::count(x, col);
      if (kLags) {
#pragma unroll
        for (uint32_t k = 1; k <= LC_STATS_MAX_LAG; k++) {
          const uint64_t j = (uint64_t)i + k;
          uint32_t y = 0;
          if (j < h) y = head[j];
          else if (j - h < m) y = data[j - h];
          tl[k - 1] += x * y;
        }
      }
    }
  }

  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  uint64_t c = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
  uint4 a = make_uint4(0, 0, 0, 0), b = a;
  uint2 t8 = make_uint2(0, 0);
  if (c < nchunks) {
    const uint8_t* q = data + c * kChunk;
    a = __ldg(reinterpret_cast<const uint4*>(q));
    b = __ldg(reinterpret_cast<const uint4*>(q + 16));
    t8 = __ldg(reinterpret_cast<const uint2*>(q + 32));
  }
  uint32_t it = 0;
  for (; c < nchunks; c += stride) {
    uint32_t w[10] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, t8.x, t8.y};
    if (c + stride < nchunks) {
      const uint8_t* q = data + (c + stride) * kChunk;
      a = __ldg(reinterpret_cast<const uint4*>(q));
      b = __ldg(reinterpret_cast<const uint4*>(q + 16));
      t8 = __ldg(reinterpret_cast<const uint2*>(q + 32));
    }
    Hist::chunk(col, w);
    if (kLags) {
      lags_chunk(w, tl);
      if ((++it & 1023u) == 0u) {
#pragma unroll
        for (int k = 0; k < LC_STATS_MAX_LAG; k++) {
          if (k < (int)max_lag) atomicAdd(acc + 258 + k, (unsigned long long)tl[k]);
          tl[k] = 0;
        }
      }
    }
  }

  if (blockIdx.x == gridDim.x - 1) {
    for (uint64_t i = nchunks * kChunk + (uint64_t)kChunk * threadIdx.x; i < m; i += (uint64_t)kChunk * kThreads) {
      uint32_t w[10];
#pragma unroll
      for (int j = 0; j < 10; j++) w[j] = guarded_word(data, i + 4 * j, m);
      if (i + kChunk <= m) {
        Hist::chunk(col, w);
      } else {
        for (uint32_t q = 0; i + q < m; q++) Hist::count((w[q >> 2] >> (8 * (q & 3))) & 255u, col);
      }
      if (kLags) lags_chunk(w, tl);
    }
  }
  __syncthreads();
  Hist::flush(acc, kThreads);
  if (kLags) {
#pragma unroll
    for (int k = 0; k < LC_STATS_MAX_LAG; k++) {
      unsigned long long v = tl[k];
      for (int off = 16; off; off >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, off);
      if (lane == 0 && k < (int)max_lag && v) atomicAdd(acc + 258 + k, v);
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
  const uint64_t nchunks = m >= 40 ? (m - 8) / kChunk : 0;
  const void* fn = max_lag ? reinterpret_cast<const void*>(&stats_kernel<true, kLagThreads, kLagMinBlocks>)
                           : reinterpret_cast<const void*>(&stats_kernel<false, kHistThreads, kHistMinBlocks>);
  const int threads = max_lag ? kLagThreads : kHistThreads;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Hist::kBytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, Hist::kBytes);
  if (e != cudaSuccess) return e;
  // one wave of resident CTAs, no more than the chunks need
  uint64_t grid = (uint64_t)sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
  const uint64_t need = (nchunks + threads - 1) / threads;
  if (need < grid) grid = need;
  if (grid == 0) grid = 1;
  if (max_lag)
    stats_kernel<true, kLagThreads, kLagMinBlocks>
        <<<(unsigned)grid, kLagThreads, Hist::kBytes, s>>>(data, h, body, m, nchunks, max_lag, acc);
  else
    stats_kernel<false, kHistThreads, kHistMinBlocks>
        <<<(unsigned)grid, kHistThreads, Hist::kBytes, s>>>(data, h, body, m, nchunks, 0, acc);
  return cudaGetLastError();
}

}  // namespace lc
