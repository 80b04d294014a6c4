// stats.cu -- byte statistics of a device buffer for the ciphertext
// analysis of Sec. 4: the frequency histogram (Fig. 2), from which the
// Shannon entropy follows, and the lagged products behind the
// auto-correlation of Fig. 3.  Every quantity is an exact integer sum, so
// the result does not depend on the order in which threads add.
//
// One pass over the data, bound by HBM bandwidth in principle and, on
// GB300, by the shared-memory atomics of the histogram (one per byte) and
// the integer work of the lagged products.  Each CTA keeps a private
// histogram in shared memory laid out as [bin][lane]: lane l of every warp
// counts into column l, so the 32 atomics of a warp instruction always fall
// in 32 different banks.  Two kernels, each the faster one for its case on
// GB300:
//   - histogram only (max_lag = 0): each thread reads 32-byte chunks
//     straight from global memory with 16-byte loads, the next chunk's loads
//     issued before the current chunk is counted;
//   - with lagged products: the bytes reach the CTA as 16 KiB tiles that one
//     thread copies from global to shared memory with bulk asynchronous
//     copies (cp.async.bulk, completion on an mbarrier), two tiles in flight
//     per CTA.  Each thread counts two 32-byte chunks of a tile (plus the
//     next 8 bytes for the lagged products), forming the sums of products
//     four bytes at a time with the unsigned 4-way byte dot product
//     (__dp4a); the partial sums reach the global 64-bit totals once per CTA
//     at the end.
// The ragged end of the buffer is read with guarded loads.  The sum and the
// sum of squares are not accumulated here: they follow exactly from the
// histogram (the host forms them).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lc.h"

namespace lc {

namespace {

// Chunks per thread in a staged tile, tiles in flight per CTA, and the
// resident CTAs per SM the direct kernel is compiled for (chosen by
// measurement on GB300).
#ifndef LC_STATS_CPT
#define LC_STATS_CPT 2
#endif
#ifndef LC_STATS_STAGES
#define LC_STATS_STAGES 2
#endif
#ifndef LC_STATS_MINB
#define LC_STATS_MINB 5
#endif

constexpr int kThreads = 256;
constexpr uint32_t kChunk = 32;                            // bytes per thread and count step
constexpr int kCpt = LC_STATS_CPT;
constexpr uint32_t kTileBytes = kCpt * kChunk * kThreads;  // bytes per staged tile
constexpr uint32_t kCopyBytes = kTileBytes + 16;           // + the 16 bytes after it (lag partners)
constexpr uint32_t kStageStride = kCopyBytes;              // 16-byte aligned stages
constexpr int kStages = LC_STATS_STAGES;
constexpr size_t kSmemBytes = (size_t)kStages * kStageStride;  // dynamic: the stages

// The CTA's histogram, [bin][lane]: the counter of bin x in lane l's column
// sits at byte offset (x << 7) | (l << 2), so the 32 atomics of a warp
// instruction fall in 32 different banks.  A static array, so that its
// address is a constant and each count needs one shift and one and-or.
__shared__ __align__(128) uint32_t s_hist[256 * 32];
constexpr uint32_t kSpinLimit = 1u << 22;  // bounded mbarrier waits
constexpr int kTimeoutWord = 256;          // acc[256]: set when a wait gave up

// Bytes i .. i + 3 of data as a little-endian word, 0 for bytes at or past
// n (only for the ragged end of the buffer).
__device__ __forceinline__ uint32_t guarded_word(const uint8_t* data, uint64_t i, uint64_t n) {
  uint32_t v = 0;
#pragma unroll
  for (int b = 0; b < 4; b++)
    if (i + b < n) v |= (uint32_t)data[i + b] << (8 * b);
  return v;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Thread 0: announce `bytes` on the barrier and start the bulk copy of
// [src, src + bytes) into shared memory at dst.  16-byte aligned source and
// destination, size a multiple of 16.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Wait for phase `parity` of the barrier to complete; false after
// kSpinLimit polls (each poll may itself suspend the thread for a while).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit; it++) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void count_at(uint32_t off) {
  atomicAdd(reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(s_hist) + off), 1u);
}

// Histogram of the 32 bytes w[0..7] (all counted); lane4 = lane << 2.
__device__ __forceinline__ void hist_chunk(uint32_t lane4, const uint32_t (&w)[10]) {
#pragma unroll
  for (int j = 0; j < 8; j++) {
    count_at(((w[j] << 7) & 0x7F80u) | lane4);
    count_at(((w[j] >> 1) & 0x7F80u) | lane4);
    count_at(((w[j] >> 9) & 0x7F80u) | lane4);
    count_at(((w[j] >> 17) & 0x7F80u) | lane4);
  }
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

// acc layout (uint64): [0, 256) histogram, 256 the timeout flag, 257 unused,
// 258 + k - 1 for lag k = 1..max_lag: sum of x_i x_{i+k}.
//
// `data` here is 16-byte aligned; the caller's unaligned head is counted by
// thread 0 of CTA 0 from `head` (h bytes before data).  Tiles [0, ntiles)
// of kTileBytes are staged (each with the 16 bytes after it, all inside
// the buffer); the rest [ntiles * kTileBytes, m) is counted by the last CTA
// with guarded loads.
template <bool kLags>
__global__ void __launch_bounds__(kThreads) stats_kernel(const uint8_t* __restrict__ head, uint32_t h,
                                                         const uint8_t* __restrict__ data, uint64_t m,
                                                         uint64_t ntiles, uint32_t max_lag,
                                                         unsigned long long* acc) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[kStages];
  uint32_t* const hist = s_hist;
  uint8_t* const stage = smem;
  for (int i = threadIdx.x; i < 256 * 32; i += kThreads) hist[i] = 0u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; s++) mbar_init(smem_addr(&bars[s]), 1u);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lane4 = lane << 2;
  uint64_t lag[LC_STATS_MAX_LAG];
  uint32_t tl[LC_STATS_MAX_LAG];
#pragma unroll
  for (int k = 0; k < LC_STATS_MAX_LAG; k++) lag[k] = 0, tl[k] = 0;

  // The unaligned head: at most 15 bytes, each with its lagged partners,
  // which may lie in the aligned part.
  if (h && blockIdx.x == 0 && threadIdx.x == 0) {
    for (uint32_t i = 0; i < h; i++) {
      const uint32_t x = head[i];
      count_at((x << 7) | lane4);
      if (kLags) {
#pragma unroll
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

  // Staged tiles t = blockIdx.x + i * gridDim.x: a ring of kStages buffers,
  // tile i in stage i mod kStages, its barrier completing phase
  // (i / kStages) mod 2.
  const uint64_t mine = ntiles > blockIdx.x ? (ntiles - blockIdx.x - 1) / gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (uint64_t i = 0; i < (uint64_t)kStages && i < mine; i++)
      bulk_load(smem_addr(stage + i * kStageStride), data + (blockIdx.x + i * gridDim.x) * (uint64_t)kTileBytes,
                kCopyBytes, smem_addr(&bars[i]));
  }
  uint64_t done = 0;
  bool timed_out = false;
  for (uint64_t i = 0; i < mine; i++) {
    const int s = (int)(i % kStages);
    const bool ok = mbar_wait(smem_addr(&bars[s]), (uint32_t)((i / kStages) & 1u));
    if (__syncthreads_or(!ok)) {  // the whole CTA leaves together
      timed_out = true;
      break;
    }
    const uint8_t* st = stage + s * kStageStride;
#pragma unroll
    for (int c = 0; c < kCpt; c++) {
      const uint32_t off = (threadIdx.x + c * kThreads) * kChunk;
      uint32_t w[10];
      const uint4 a = *reinterpret_cast<const uint4*>(st + off);
      const uint4 b = *reinterpret_cast<const uint4*>(st + off + 16);
      const uint2 n8 = *reinterpret_cast<const uint2*>(st + off + 32);
      w[0] = a.x, w[1] = a.y, w[2] = a.z, w[3] = a.w;
      w[4] = b.x, w[5] = b.y, w[6] = b.z, w[7] = b.w;
      w[8] = n8.x, w[9] = n8.y;
      hist_chunk(lane4, w);
      if (kLags) lags_chunk(w, tl);
    }
    // 32-bit partials: one tile adds kCpt x 32 products below 2^16 per lag,
    // so 256 / kCpt tiles stay below 2^32
    static_assert(kCpt == 1 || kCpt == 2 || kCpt == 4, "flush period");
    if ((i & (256u / kCpt - 1u)) == 256u / kCpt - 1u) {
#pragma unroll
      for (int k = 0; k < LC_STATS_MAX_LAG; k++) lag[k] += tl[k], tl[k] = 0;
    }
    done = i + 1;
    __syncthreads();  // every thread is done with stage s
    if (threadIdx.x == 0 && i + kStages < mine) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bulk_load(smem_addr(stage + s * kStageStride),
                data + (blockIdx.x + (i + kStages) * gridDim.x) * (uint64_t)kTileBytes, kCopyBytes,
                smem_addr(&bars[s]));
    }
  }
  if (timed_out) {
    // Record the failure and wait (bounded) for the copies still in flight
    // before the CTA's shared memory is released.
    if (threadIdx.x == 0) {
      atomicOr(acc + kTimeoutWord, 1ull);
      for (uint64_t i = done; i < mine && i < done + kStages; i++)
        mbar_wait(smem_addr(&bars[i % kStages]), (uint32_t)((i / kStages) & 1u));
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < LC_STATS_MAX_LAG; k++) lag[k] += tl[k], tl[k] = 0;

  // The rest of the buffer (< one tile + 32 bytes) on the last CTA, with
  // guarded loads: bytes at or past m read as 0 and are not counted.
  if (blockIdx.x == gridDim.x - 1) {
    for (uint64_t i = ntiles * kTileBytes + (uint64_t)kChunk * threadIdx.x; i < m;
         i += (uint64_t)kChunk * kThreads) {
      uint32_t w[10];
#pragma unroll
      for (int j = 0; j < 10; j++) w[j] = guarded_word(data, i + 4 * j, m);
      if (i + kChunk <= m) {
        hist_chunk(lane4, w);
      } else {
        for (uint32_t q = 0; i + q < m; q++) count_at((((w[q >> 2] >> (8 * (q & 3))) & 255u) << 7) | lane4);
      }
      if (kLags) lags_chunk(w, tl);
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

// Direct variant: each thread reads its 32-byte chunks (and the 8 bytes
// after each) straight from global memory with 16-byte loads, issuing the
// next chunk's loads before it counts the current one, so that no shared
// memory bandwidth goes to staging.  Chunks [0, nchunks) lie, with their 8
// successors, inside the aligned part; the rest is counted by the last CTA
// with guarded loads.  The lagged sums stay in 32-bit registers and reach
// the 64-bit totals by global atomics: every 1024 chunks (a chunk adds less
// than 2^21 per lag) and at the end, warp-reduced.
template <bool kLags>
__global__ void __launch_bounds__(kThreads, LC_STATS_MINB) stats_direct_kernel(
    const uint8_t* __restrict__ head, uint32_t h, const uint8_t* __restrict__ data, uint64_t m,
    uint64_t nchunks, uint32_t max_lag, unsigned long long* acc) {
  uint32_t* const hist = s_hist;
  for (int i = threadIdx.x; i < 256 * 32; i += kThreads) hist[i] = 0u;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t lane4 = lane << 2;
  uint32_t tl[LC_STATS_MAX_LAG];
#pragma unroll
  for (int k = 0; k < LC_STATS_MAX_LAG; k++) tl[k] = 0;

  if (h && blockIdx.x == 0 && threadIdx.x == 0) {
    // the unaligned head (< 16 bytes), with partners in the aligned part
    for (uint32_t i = 0; i < h; i++) {
      const uint32_t x = head[i];
      count_at((x << 7) | lane4);
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
    hist_chunk(lane4, w);
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
        hist_chunk(lane4, w);
      } else {
        for (uint32_t q = 0; i + q < m; q++) count_at((((w[q >> 2] >> (8 * (q & 3))) & 255u) << 7) | lane4);
      }
      if (kLags) lags_chunk(w, tl);
    }
  }
  __syncthreads();
  for (uint32_t bn = threadIdx.x; bn < 256; bn += kThreads) {
    uint64_t t = 0;
    for (uint32_t cl = 0; cl < 32; cl++) t += hist[bn * 32u + ((cl + bn) & 31u)];
    if (t) atomicAdd(acc + bn, (unsigned long long)t);
  }
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

// acc[256] != 0 after the kernel: a bounded wait gave up (LC_ERR_TIMEOUT).
cudaError_t launch_stats(const uint8_t* data, uint64_t n, uint32_t max_lag, unsigned long long* acc,
                         int sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(acc, 0, (258 + LC_STATS_MAX_LAG) * sizeof(unsigned long long), s);
  if (e != cudaSuccess || n == 0) return e;
  const uint64_t mis = reinterpret_cast<uintptr_t>(data) & 15u;
  const uint32_t h = (uint32_t)(mis ? (16u - mis < n ? 16u - mis : n) : 0u);
  const uint8_t* body = data + h;
  const uint64_t m = n - h;
  // staged tiles: tile t and the 16 bytes after it lie inside the first
  // m16 = m rounded down to 16 bytes
  const uint64_t m16 = m & ~(uint64_t)15;
  if (max_lag == 0) {
    // histogram only: the direct kernel; chunk c reads bytes [32c, 32c + 40)
    // of the aligned part
    const uint64_t nchunks = m >= 40 ? (m - 8) / kChunk : 0;
    const void* fnd = reinterpret_cast<const void*>(&stats_direct_kernel<false>);
    int per_sm_d = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_d, fnd, kThreads, 0);
    if (e != cudaSuccess) return e;
    uint64_t grid_d = (uint64_t)sms * (uint64_t)(per_sm_d > 0 ? per_sm_d : 1);
    const uint64_t need = (nchunks + kThreads - 1) / kThreads;
    if (need < grid_d) grid_d = need;
    if (grid_d == 0) grid_d = 1;
    stats_direct_kernel<false><<<(unsigned)grid_d, kThreads, 0, s>>>(data, h, body, m, nchunks, 0, acc);
    return cudaGetLastError();
  }
  // with lagged products: the staged kernel
  const uint64_t ntiles = m16 >= 16 ? (m16 - 16) / kTileBytes : 0;
  const void* fn = reinterpret_cast<const void*>(&stats_kernel<true>);
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, kSmemBytes);
  if (e != cudaSuccess) return e;
  // one wave of resident CTAs, at most one per tile
  uint64_t grid = (uint64_t)sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
  if (ntiles < grid) grid = ntiles;
  if (grid == 0) grid = 1;
  stats_kernel<true><<<(unsigned)grid, kThreads, kSmemBytes, s>>>(data, h, body, m, ntiles, max_lag, acc);
  return cudaGetLastError();
}

}  // namespace lc
