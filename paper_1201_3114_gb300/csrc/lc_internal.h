// lc_internal.h -- structures shared by the host side of liblorenzcipher and
// its CUDA kernels.  Nothing here is part of the public ABI (include/lc.h).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "../../include/lc.h"

namespace lc {

// Largest Omega bound supported (Eq. 7 allows k_i <= 4 for xi = 52; the
// library accepts up to 8, i.e. any byte of the int64).
constexpr int kMaxK = 8;
// Theta table: Theta[w][P] = P / 10^(3 + w), w < kMaxK, P < 256 (Sec. 3.2 Step 2).
constexpr int kThetaEntries = kMaxK * 256;

// Cipher kernel variants: any parameters (FP64 pipe only), any parameters
// with k = (4, 4, 4), and the v1 constants sigma = 10, rho = 28, k = 4 whose
// binary64 work is split between the FP64 and integer pipes.
constexpr int kVariantGeneral = 0;
constexpr int kVariantGeneral4 = 1;
constexpr int kVariantV1 = 2;
// The v1 constants with every binary64 operation on the FP64 pipe: shorter
// dependency chains, hence lower latency while the GPU is far from full.
constexpr int kVariantV1Latency = 3;
// kVariantV1 compiled for 4 resident 256-thread CTAs per SM (64 registers).
constexpr int kVariantV1Dense = 4;
// kVariantV1 and kVariantGeneral that also count the digit statistics of
// Fig. 1 (lc_ctx_digit_stats).
constexpr int kVariantV1Digits = 5;
constexpr int kVariantGeneralDigits = 6;
// kVariantV1 and kVariantGeneral that also accumulate the byte statistics
// of every ciphertext they write (lc_ctx_ciphertext_stats), without and with
// the digit statistics.
constexpr int kVariantV1CtStats = 7;
constexpr int kVariantGeneralCtStats = 8;
constexpr int kVariantV1DigitsCtStats = 9;
constexpr int kVariantGeneralDigitsCtStats = 10;
// kVariantV1 for batches that do not fill the persistent grid: the kick
// stays on the FP64 pipe (shorter chains for fewer resident warps).
constexpr int kVariantV1Partial = 11;
// kVariantV1Partial compiled for 4 resident 256-thread CTAs per SM.
constexpr int kVariantV1PartialDense = 12;
// The v1 constants, all binary64 work on the FP64 pipe, each part's three
// coordinates on three warps of a 96-thread CTA (far-from-full batches).
constexpr int kVariantV1Split = 13;
// kVariantV1Dense for batches whose messages carry their own k in {3, 4}^3.
constexpr int kVariantV1MsgK = 14;
constexpr int kNumVariants = 15;
constexpr int kSplitThreads = 96;
constexpr uint32_t kSplitRowsPerCta = 32;
// Below this many parts per SM a v1 batch of the FP64-pipe variant runs split
// (measured crossover on GB300).
constexpr uint32_t kSplitBatchRowsPerSm = 64;

inline bool variant_has_ct_stats(int v) { return v >= kVariantV1CtStats && v <= kVariantGeneralDigitsCtStats; }
inline bool variant_is_general(int v) {
  return v == kVariantGeneral || v == kVariantGeneralDigits || v == kVariantGeneralCtStats ||
         v == kVariantGeneralDigitsCtStats;
}

// Fig. 1 digit statistics: counters per coordinate (128 integer-part bins,
// 3 x 100 digit-pair bins, 1 out-of-range count).
constexpr int kDigBins = 429;

// Fused ciphertext statistics (Sec. 4, Figs. 2-3): 64-bit accumulators
// [0, 256) byte histogram, [256, 256 + LC_STATS_MAX_LAG) sums of x_i x_{i+k}.
constexpr int kCtStatsWords = 256 + LC_STATS_MAX_LAG;
// Threads per CTA of the counting variants (their shared-memory slots are
// sized for it).
constexpr int kCtStatsThreads = 256;
// Shared memory of the counting variants beyond the Theta table: the CTA's
// histogram as [bin][lane] 32-bit counters and one 64-bit accumulator per
// thread and lag.
constexpr size_t kCtStatsSmem = 256 * 32 * sizeof(uint32_t) +
                                (size_t)LC_STATS_MAX_LAG * kCtStatsThreads * sizeof(unsigned long long);

// Below this many parts per SM (1.5 warps per SM sub-partition) a v1 batch
// runs the latency variant (measured crossover on GB300).
constexpr uint32_t kSmallBatchRowsPerSm = 4 * 32 * 3 / 2;

// Constants of the method as the kernels read them.
struct DevParams {
  double sigma, rho, beta, dt, eta;
  uint32_t n_warm;
  uint32_t steps_per_byte;
  uint32_t block_len;
  uint32_t tag_len;
  uint32_t k[3];
  uint32_t k_all4;  // 1 when k = (4, 4, 4): Omega fits in two bits
  uint32_t omega_alpha_shift;  // Step 3's alpha index read with 0-based i
};

// One message of a batch, as the kernels see it (80 bytes).
struct alignas(16) DevMsg {
  const uint8_t* in;   // plaintext (encrypt) or ciphertext (decrypt)
  uint8_t* out;        // ciphertext (encrypt) or plaintext (decrypt)
  uint64_t n;          // plaintext length in bytes
  double base[3];      // RN(a'_j + lambda_j): Eq. 5 without the part offset
  double aprime[3];    // a'_j, added after every byte (Step 3)
  uint32_t key_bits;   // mu_i in bits [2i, 2i+2), Omega_i in bits [8+4i, 12+4i),
                       // with kFlagMsgK: k_i in bits [20+4i, 24+4i)
  uint32_t flags;      // kFlagDecrypt | kFlagSequential | kFlagMsgK
};
static_assert(sizeof(DevMsg) == 80, "DevMsg layout");

constexpr uint32_t kFlagDecrypt = 1u;
constexpr uint32_t kFlagSequential = 2u;
// The message carries its own k (per-request key material, Eq. 7); only the
// general kernel variant reads it.
constexpr uint32_t kFlagMsgK = 4u;

// One trajectory: part `b` of message `msg` (b = 0 in sequential mode).
struct DevRow {
  uint32_t msg;
  uint32_t b;
};

// Batch header, at the start of the uploaded workspace.
struct alignas(16) DevHeader {
  uint32_t nrows;
  uint32_t nmsgs;
  int32_t* status_out;     // caller's status array (device)
  uint32_t rows_per_warp;  // R: rows a warp takes per grab (1..32, see kernel)
  uint32_t reserved0;
  uint64_t reserved1;
};
static_assert(sizeof(DevHeader) == 32, "DevHeader layout");

// R: rows a warp takes per grab.  A warp instruction costs the FP64 pipe
// and the issue slot as much with one active lane as with 32 (measured), so
// rows are packed into full warps (R = 32) and it is the warps that are
// spread over the SMs (see the kernel's first pass).
inline uint32_t rows_per_warp(uint64_t /*nrows*/, uint64_t /*grid_warps*/) { return 32u; }

// Persistent-kernel scratch that lives across launches: the row counter and
// the per-message fail flags.  A memset before each launch of the cipher
// kernel clears both (a memset node at the head of the context's graph; an
// explicit cudaMemsetAsync in the allocation-free path); the finalize kernel
// only reads them.
struct DevScratch {
  uint32_t row_counter;
  uint32_t pad[3];
};

}  // namespace lc
