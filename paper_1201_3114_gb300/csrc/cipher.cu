// cipher.cu -- CUDA kernels of the Lorenz-attractor chaotic cipher
// (Marco, Martinez & Bruno, arXiv 1201.3114) for sm_103a.
//
// One thread owns one trajectory: part b of a message in the parallel
// version (Sec. 5) or the whole message in the sequential version (Sec. 3).
// Its Lorenz state (x, y, z) stays in registers for the part's lifetime; the
// part's bytes stream through 16-byte vector loads and stores.  Every
// floating-point operation is an explicit round-to-nearest binary64
// intrinsic (__dadd_rn / __dsub_rn / __dmul_rn) and the file is compiled
// with --fmad=false, so no multiply-add contraction can change a rounding:
// the results are bit-identical to a plain IEEE-754 evaluation in the
// paper's operation order.
//
// Nothing here is a dense contraction, so no tensor-core path exists: the
// kernel is bound by the FP64 issue rate of the SM.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lc_internal.h"

namespace cg = cooperative_groups;

namespace lc {

namespace {

// nu = floor(log10 2^(xi - 6)) = 13 for xi = 52 (Sec. 3.1, Eq. 8).
constexpr double kScale = 1e13;

// ---------------------------------------------------------------------------
// Eq. 1 read as forward Euler of the Lorenz system:
//   x += dt * (sigma (y - x)),  y += dt * ((rho x - y) - x z),
//   z += dt * (x y - beta z),   each operation rounded once.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void euler_step(double& x, double& y, double& z, const DevParams& p) {
  const double dx = __dmul_rn(p.sigma, __dsub_rn(y, x));
  const double dy = __dsub_rn(__dsub_rn(__dmul_rn(p.rho, x), y), __dmul_rn(x, z));
  const double dz = __dsub_rn(__dmul_rn(x, y), __dmul_rn(p.beta, z));
  x = __dadd_rn(x, __dmul_rn(p.dt, dx));
  y = __dadd_rn(y, __dmul_rn(p.dt, dy));
  z = __dadd_rn(z, __dmul_rn(p.dt, dz));
}

__device__ __forceinline__ double pick(uint32_t m, double x, double y, double z) {
  return m == 0 ? x : (m == 1 ? y : z);
}

// floor(RN(alpha * 10^13)) as a two's complement int64: cvt.rmi.s64.f64
// saturates out-of-range values and maps NaN to 0.
__device__ __forceinline__ uint64_t floor_scaled(double alpha) {
  return (uint64_t)__double2ll_rd(__dmul_rn(alpha, kScale));
}

// One trajectory's state between bytes (Sec. 3.2).  V_i caches
// floor(alpha_i 10^13): alpha_i only changes in Step 3, and every R_nu of
// the following byte reads the same V_i.
struct Traj {
  double x, y, z;
  double ax, ay, az;  // a'
  uint64_t V0, V1, V2;
  uint32_t mu0, mu1, mu2;
  uint32_t om0, om1, om2;
};

__device__ __forceinline__ uint32_t rbyte(uint64_t V, uint32_t om) {
  return (uint32_t)(V >> (8u * om)) & 255u;
}

template <bool K4>
__device__ __forceinline__ uint32_t mod_k(uint32_t v, uint32_t k) {
  if (K4) return v & 3u;
  return v % k;
}

// Sec. 3.2, Steps 1-3, for one byte.  dec = 0: x is P_i, returns C_i.
// dec = 1: x is C_i, returns P_i.  The direction is data, not control flow,
// so encrypting and decrypting threads of one warp never diverge.
template <bool K4>
__device__ __forceinline__ uint32_t step_byte(Traj& t, uint32_t x, uint32_t dec, const DevParams& p,
                                              const double* __restrict__ theta) {
  // Step 1 (Eqs. 9, 10): R_nu(alpha_1, Omega_1) + R_nu(alpha_2, Omega_2).
  const uint32_t R1 = rbyte(t.V0, t.om0);
  const uint32_t R2 = rbyte(t.V1, t.om1);
  const uint32_t s = R1 + R2;
  const uint32_t y = (dec ? (x - s) : (x + s)) & 255u;
  const uint32_t P = dec ? y : x;

  // Step 2: Theta = P / 10^(3 + Omega_3) kicks r[mu_3], then F.
  const double th = theta[t.om2 * 256u + P];
  const double kicked = __dadd_rn(pick(t.mu2, t.x, t.y, t.z), th);
  t.x = t.mu2 == 0 ? kicked : t.x;
  t.y = t.mu2 == 1 ? kicked : t.y;
  t.z = t.mu2 == 2 ? kicked : t.z;
  for (uint32_t k = 0; k < p.steps_per_byte; k++) euler_step(t.x, t.y, t.z, p);

  // Step 3: mu from the old alpha and Omega; alpha re-read from r with the
  // new mu (Eq. 6); Omega from the new alpha and the old Omega; r += a'.
  const uint32_t R3 = rbyte(t.V2, t.om2);
  t.mu0 = (t.mu0 + R1) % 3u;
  t.mu1 = (t.mu1 + R2) % 3u;
  t.mu2 = (t.mu2 + R3) % 3u;
  t.V0 = floor_scaled(pick(t.mu0, t.x, t.y, t.z));
  t.V1 = floor_scaled(pick(t.mu1, t.x, t.y, t.z));
  t.V2 = floor_scaled(pick(t.mu2, t.x, t.y, t.z));
  t.om0 = mod_k<K4>(t.om0 + rbyte(t.V0, t.om0), p.k[0]);
  t.om1 = mod_k<K4>(t.om1 + rbyte(t.V1, t.om1), p.k[1]);
  t.om2 = mod_k<K4>(t.om2 + rbyte(t.V2, t.om2), p.k[2]);
  t.x = __dadd_rn(t.x, t.ax);
  t.y = __dadd_rn(t.y, t.ay);
  t.z = __dadd_rn(t.z, t.az);
  return y;
}

template <bool K4>
__device__ __forceinline__ uint32_t step_word(Traj& t, uint32_t w, uint32_t dec, const DevParams& p,
                                              const double* __restrict__ theta) {
  uint32_t o = 0;
#pragma unroll
  for (int j = 0; j < 4; j++) o |= step_byte<K4>(t, (w >> (8 * j)) & 255u, dec, p, theta) << (8 * j);
  return o;
}

// One trajectory: Eq. 5 plus the part offset b * eta, the warm-up, then the
// part's body bytes and its tag.  Returns the tag verdict (always true when
// encrypting).
template <bool K4>
__device__ bool run_row(const DevMsg& M, uint32_t b, const DevParams& p,
                        const double* __restrict__ theta) {
  const bool seq = (M.flags & kFlagSequential) != 0;
  const uint32_t dec = (M.flags & kFlagDecrypt) ? 1u : 0u;
  const uint64_t lo = seq ? 0 : (uint64_t)b * p.block_len;
  const uint64_t len = seq ? M.n : min((uint64_t)p.block_len, M.n - lo);
  const uint64_t tag_off = M.n + (seq ? 0 : (uint64_t)b * p.tag_len);

  Traj t;
  const double off = __dmul_rn((double)b, p.eta);
  t.x = __dadd_rn(M.base[0], off);
  t.y = __dadd_rn(M.base[1], off);
  t.z = __dadd_rn(M.base[2], off);
  t.ax = M.aprime[0];
  t.ay = M.aprime[1];
  t.az = M.aprime[2];
  for (uint32_t s = 0; s < p.n_warm; s++) euler_step(t.x, t.y, t.z, p);
  t.mu0 = M.key_bits & 3u;
  t.mu1 = (M.key_bits >> 2) & 3u;
  t.mu2 = (M.key_bits >> 4) & 3u;
  t.om0 = (M.key_bits >> 8) & 15u;
  t.om1 = (M.key_bits >> 12) & 15u;
  t.om2 = (M.key_bits >> 16) & 15u;
  t.V0 = floor_scaled(pick(t.mu0, t.x, t.y, t.z));
  t.V1 = floor_scaled(pick(t.mu1, t.x, t.y, t.z));
  t.V2 = floor_scaled(pick(t.mu2, t.x, t.y, t.z));

  const uint8_t* src = M.in + lo;
  uint8_t* dst = M.out + lo;
  uint64_t i = 0;
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
    const uint64_t nv = len >> 4;
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    if (nv) {
      uint4 cur = s4[0];
      for (uint64_t c = 0; c < nv; c++) {
        uint4 nxt = cur;
        if (c + 1 < nv) nxt = s4[c + 1];  // read ahead before the store (in-place safe)
        uint4 o;
        o.x = step_word<K4>(t, cur.x, dec, p, theta);
        o.y = step_word<K4>(t, cur.y, dec, p, theta);
        o.z = step_word<K4>(t, cur.z, dec, p, theta);
        o.w = step_word<K4>(t, cur.w, dec, p, theta);
        d4[c] = o;
        cur = nxt;
      }
    }
    i = nv << 4;
  }
  for (; i < len; i++) dst[i] = (uint8_t)step_byte<K4>(t, src[i], dec, p, theta);

  // Tag: T further bytes whose plaintext is the message length, LE64(n).
  bool ok = true;
  for (uint32_t q = 0; q < p.tag_len; q++) {
    const uint32_t Q = (uint32_t)(M.n >> (8 * q)) & 255u;
    if (dec) {
      const uint32_t got = step_byte<K4>(t, M.in[tag_off + q], 1u, p, theta);
      ok = ok && (got == Q);
    } else {
      M.out[tag_off + q] = (uint8_t)step_byte<K4>(t, Q, 0u, p, theta);
    }
  }
  return ok;
}

__device__ __forceinline__ void load_msg(DevMsg& m, const DevMsg* src) {
  const uint4* s = reinterpret_cast<const uint4*>(src);
  uint4* d = reinterpret_cast<uint4*>(&m);
#pragma unroll
  for (int i = 0; i < 5; i++) d[i] = s[i];
}

// Persistent batched kernel: CTAs stay resident and pull rows of the
// flattened part table (sorted longest first) with warp-aggregated atomics.
template <bool K4>
__global__ void __launch_bounds__(256) batch_kernel(const uint8_t* __restrict__ ws,
                                                    uint32_t* __restrict__ scratch,
                                                    DevParams p,
                                                    const double* __restrict__ theta_g) {
  extern __shared__ double s_theta[];
  const int nth = K4 ? 4 * 256 : kThetaEntries;
  for (int i = threadIdx.x; i < nth; i += blockDim.x) s_theta[i] = theta_g[i];
  __syncthreads();

  const DevHeader* H = reinterpret_cast<const DevHeader*>(ws);
  const uint32_t nrows = H->nrows;
  const uint32_t nmsgs = H->nmsgs;
  const DevMsg* msgs = reinterpret_cast<const DevMsg*>(ws + sizeof(DevHeader));
  const DevRow* rows = reinterpret_cast<const DevRow*>(msgs + nmsgs);
  uint32_t* counter = scratch;
  uint32_t* fail = scratch + 4;

  while (true) {
    cg::coalesced_group g = cg::coalesced_threads();
    uint32_t base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, g.size());
    base = g.shfl(base, 0);
    const uint32_t r = base + g.thread_rank();
    if (r >= nrows) break;
    const DevRow row = rows[r];
    DevMsg M;
    load_msg(M, msgs + row.msg);
    const bool ok = run_row<K4>(M, row.b, p, s_theta);
    if (M.flags & kFlagDecrypt) {
      // Segmented vote: threads of the warp holding parts of the same
      // message combine their verdicts; one atomic per message and warp.
      cg::coalesced_group d = cg::coalesced_threads();
      cg::coalesced_group same = cg::labeled_partition(d, row.msg);
      const bool any_bad = same.any(!ok);
      if (same.thread_rank() == 0 && any_bad) atomicOr(fail + row.msg, 1u);
    }
  }
}

// After the batch: per-request status, and fail-closed zeroing of the
// plaintext of every decryption whose verdict failed.
__global__ void finalize_kernel(const uint8_t* __restrict__ ws, const uint32_t* __restrict__ scratch,
                                uint32_t block_len) {
  const DevHeader* H = reinterpret_cast<const DevHeader*>(ws);
  const uint32_t nrows = H->nrows;
  const uint32_t nmsgs = H->nmsgs;
  const DevMsg* msgs = reinterpret_cast<const DevMsg*>(ws + sizeof(DevHeader));
  const DevRow* rows = reinterpret_cast<const DevRow*>(msgs + nmsgs);
  const int32_t* init = reinterpret_cast<const int32_t*>(rows + nrows);
  const uint32_t* fail = scratch + 4;
  const uint32_t total = nrows > nmsgs ? nrows : nmsgs;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    if (i < nmsgs) {
      const int32_t s0 = init[i];
      H->status_out[i] = s0 ? s0 : (fail[i] ? (int32_t)LC_ERR_INTEGRITY : (int32_t)LC_OK);
    }
    if (i < nrows) {
      const DevRow row = rows[i];
      if (fail[row.msg]) {
        const DevMsg& M = msgs[row.msg];
        const bool seq = (M.flags & kFlagSequential) != 0;
        const uint64_t lo = seq ? 0 : (uint64_t)row.b * block_len;
        const uint64_t len = seq ? M.n : min((uint64_t)block_len, M.n - lo);
        for (uint64_t j = 0; j < len; j++) M.out[lo + j] = 0;
      }
    }
  }
}

// Counter-based SplitMix64 byte stream (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t splitmix_word(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void synth_kernel(uint8_t* __restrict__ dst, uint64_t n, uint64_t seed, uint64_t offset) {
  // Thread t writes dst[8t, 8t + 8): stream bytes offset + 8t ...
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t j0 = 8 * t;
  if (j0 >= n) return;
  const uint64_t s = offset + j0;
  const uint64_t w = s >> 3;
  const uint32_t sh = (uint32_t)(s & 7u);
  uint64_t v = splitmix_word(seed, w);
  if (sh) v = (v >> (8 * sh)) | (splitmix_word(seed, w + 1) << (64 - 8 * sh));
  const uint64_t cnt = (n - j0) < 8 ? (n - j0) : 8;
  if (cnt == 8 && (reinterpret_cast<uintptr_t>(dst + j0) & 7u) == 0) {
    *reinterpret_cast<uint64_t*>(dst + j0) = v;
  } else {
    for (uint64_t q = 0; q < cnt; q++) dst[j0 + q] = (uint8_t)(v >> (8 * q));
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host-side launch helpers (called from api.cu)
// ---------------------------------------------------------------------------

size_t batch_kernel_smem(bool k4) { return (k4 ? 4 * 256 : kThetaEntries) * sizeof(double); }

const void* batch_kernel_ptr(bool k4) {
  return k4 ? reinterpret_cast<const void*>(&batch_kernel<true>)
            : reinterpret_cast<const void*>(&batch_kernel<false>);
}

cudaError_t launch_batch(bool k4, int grid, int block, const uint8_t* ws, uint32_t* scratch,
                         const DevParams& p, const double* theta, cudaStream_t s) {
  const size_t smem = batch_kernel_smem(k4);
  if (k4)
    batch_kernel<true><<<grid, block, smem, s>>>(ws, scratch, p, theta);
  else
    batch_kernel<false><<<grid, block, smem, s>>>(ws, scratch, p, theta);
  return cudaGetLastError();
}

cudaError_t launch_finalize(int grid, const uint8_t* ws, const uint32_t* scratch, uint32_t block_len,
                            cudaStream_t s) {
  finalize_kernel<<<grid, 256, 0, s>>>(ws, scratch, block_len);
  return cudaGetLastError();
}

cudaError_t launch_synth(uint8_t* dst, uint64_t n, uint64_t seed, uint64_t offset, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint64_t threads = (n + 7) / 8;
  const uint64_t blocks = (threads + 255) / 256;
  synth_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, n, seed, offset);
  return cudaGetLastError();
}

}  // namespace lc
