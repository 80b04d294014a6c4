// noalloc.cu -- lc_run_batch_noalloc: the batched path for callers that
// cannot allocate device memory (see include/lc.h for who they are).
//
// The batched cipher kernel needs scratch memory beyond the caller's inputs
// and outputs: the part table it pulls rows from, the row counter, one
// verdict flag per request and the Theta table.  Here all of it lives in one
// file-scope static device array of fixed size, loaded with the library and
// held by every GPU that loads it until the process exits.  No call below
// allocates: no cudaMalloc / cudaFree / cudaHostAlloc, no CUDA graph, no host
// heap (the host image of the table is a static buffer too).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "keysched.h"
#include "lc_internal.h"

namespace lc {
cudaError_t launch_batch(int variant, int grid, int block, const uint8_t* ws, uint32_t* scratch,
                         const DevParams& p, const double* theta, cudaStream_t s,
                         unsigned long long* dig = nullptr, unsigned long long* ct = nullptr);
cudaError_t launch_finalize(int grid, const uint8_t* ws, const uint32_t* scratch, uint32_t block_len,
                            cudaStream_t s);
const void* batch_kernel_ptr(int variant);
size_t batch_kernel_smem(int variant);
int32_t validate_request(const lc_params& p, const lc_req& r, lc_mode m, size_t* n);
size_t parts_of(const lc_params& p, size_t n, lc_mode m);
void dev_params_from(const lc_params& p, DevParams* d);
int kernel_variant(const DevParams& p);
}  // namespace lc

using namespace lc;

namespace {

// Layout of the static scratch array (offsets are multiples of 256):
//   [0, kFlagsBytes)             row counter (4 words) + one fail flag per request
//   [kThetaOff, +16 KiB)         Theta table, 8 x 256 binary64 values
//   [kWsOff, kScratchBytes)      header | messages | parts | initial statuses
constexpr size_t kScratchBytes = (size_t)2 << 20;
constexpr uint32_t kMaxRequests = LC_NOALLOC_MAX_REQUESTS;
constexpr size_t kFlagsBytes = ((4 + kMaxRequests) * sizeof(uint32_t) + 255) & ~(size_t)255;
constexpr size_t kThetaOff = kFlagsBytes;
constexpr size_t kThetaBytes = kThetaEntries * sizeof(double);
constexpr size_t kWsOff = (kThetaOff + kThetaBytes + 255) & ~(size_t)255;
constexpr size_t kWsBytes = kScratchBytes - kWsOff;
constexpr size_t kMaxParts = LC_NOALLOC_MAX_PARTS;
static_assert(sizeof(DevHeader) + kMaxRequests * (sizeof(DevMsg) + sizeof(int32_t)) +
                      kMaxParts * sizeof(DevRow) <= kWsBytes,
              "LC_NOALLOC_MAX_PARTS does not fit the scratch array");

static __device__ __align__(256) uint8_t g_scratch[kScratchBytes];

// Host image of the uploaded part of the workspace, and the per-device
// address of g_scratch (host code may not use the symbol's name as a device
// address: it names a host-side stand-in).
uint8_t g_host_ws[kWsBytes];
double g_host_theta[kThetaEntries];
constexpr int kMaxDevices = 64;
uint8_t* g_dev_scratch[kMaxDevices];
std::mutex g_mu;

lc_status setup_device(int dev, uint8_t** out) {
  if (dev < 0 || dev >= kMaxDevices) return LC_ERR_CUDA;
  if (g_dev_scratch[dev]) {
    *out = g_dev_scratch[dev];
    return LC_OK;
  }
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || ptr == nullptr) return LC_ERR_CUDA;
  build_theta(g_host_theta);
  uint8_t* base = static_cast<uint8_t*>(ptr);
  if (cudaMemcpy(base + kThetaOff, g_host_theta, kThetaBytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return LC_ERR_CUDA;
  if (cudaMemset(base, 0, kFlagsBytes) != cudaSuccess) return LC_ERR_CUDA;
  g_dev_scratch[dev] = base;
  *out = base;
  return LC_OK;
}

size_t part_len(const lc_params& p, const DevMsg& M, uint32_t b) {
  if (M.flags & kFlagSequential) return (size_t)M.n;
  const size_t lo = (size_t)b * p.block_len;
  return (size_t)M.n - lo < p.block_len ? (size_t)M.n - lo : p.block_len;
}

}  // namespace

extern "C" lc_status lc_run_batch_noalloc(const lc_req* reqs, size_t count, int32_t* status_dev,
                                          lc_mode m, void* stream) {
  if ((!reqs || !status_dev) && count) return LC_ERR_ARG;
  if (m != LC_PARALLEL && m != LC_SEQUENTIAL) return LC_ERR_ARG;
  if (count > kMaxRequests) return LC_ERR_LENGTH;
  if (count == 0) return LC_OK;
  // The part table is uploaded from static pageable memory, which a
  // captured graph would re-read at replay time: capture is refused.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap) != cudaSuccess) return LC_ERR_ARG;
  if (cap != cudaStreamCaptureStatusNone) return LC_ERR_ARG;

  // The default (v1) constants, converted as the context path converts
  // them; they select the v1 kernel variants used below.
  lc_params p;
  lc_params_default(&p);
  DevParams dp;
  dev_params_from(p, &dp);
  if (kernel_variant(dp) != kVariantV1) return LC_ERR_ARG;

  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LC_ERR_CUDA;
  uint8_t* base = nullptr;
  lc_status st = setup_device(dev, &base);
  if (st != LC_OK) return st;

  // Host image: header | messages | parts (full parts first) | statuses.
  DevMsg* msgs = reinterpret_cast<DevMsg*>(g_host_ws + sizeof(DevHeader));
  int32_t init[kMaxRequests];
  size_t nparts = 0;
  for (size_t i = 0; i < count; i++) {
    const lc_req& r = reqs[i];
    DevMsg& M = msgs[i];
    memset(&M, 0, sizeof M);
    size_t n = 0;
    int32_t s = validate_request(p, r, m, &n);
    HostKey key;
    if (s == LC_OK) s = key_schedule(p, r.pw, r.pw_len, &key);
    init[i] = s;
    if (s != LC_OK) continue;
    M.in = r.in;
    M.out = r.out;
    M.n = n;
    for (int j = 0; j < 3; j++) {
      M.base[j] = key.aprime[j] + p.lambda[j];
      M.aprime[j] = key.aprime[j];
    }
    M.key_bits = key.mu[0] | key.mu[1] << 2 | key.mu[2] << 4 | key.omega[0] << 8 |
                 key.omega[1] << 12 | key.omega[2] << 16;
    M.flags = (r.dir == LC_DECRYPT ? kFlagDecrypt : 0u) | (m == LC_SEQUENTIAL ? kFlagSequential : 0u);
    nparts += parts_of(p, n, m);
    if (nparts > kMaxParts) return LC_ERR_LENGTH;
  }
  DevRow* rows = reinterpret_cast<DevRow*>(msgs + count);
  size_t w = 0;
  for (int pass = 0; pass < 2; pass++) {  // full parts, then the shorter ones
    for (size_t i = 0; i < count; i++) {
      if (init[i] != LC_OK) continue;
      const size_t nb = parts_of(p, (size_t)msgs[i].n, m);
      for (size_t b = 0; b < nb; b++) {
        const bool full = (m == LC_PARALLEL) && part_len(p, msgs[i], (uint32_t)b) == p.block_len;
        if (full == (pass == 0)) rows[w++] = DevRow{(uint32_t)i, (uint32_t)b};
      }
    }
  }
  // Longest first among the shorter parts (insertion sort, no heap).
  const size_t first_short = [&] {
    size_t k = 0;
    while (k < w && m == LC_PARALLEL && part_len(p, msgs[rows[k].msg], rows[k].b) == p.block_len) k++;
    return k;
  }();
  for (size_t a = first_short + 1; a < w; a++) {
    const DevRow cur = rows[a];
    const size_t len = part_len(p, msgs[cur.msg], cur.b);
    size_t c = a;
    while (c > first_short && part_len(p, msgs[rows[c - 1].msg], rows[c - 1].b) < len) {
      rows[c] = rows[c - 1];
      c--;
    }
    rows[c] = cur;
  }
  int32_t* init_dev_img = reinterpret_cast<int32_t*>(rows + w);
  memcpy(init_dev_img, init, count * sizeof(int32_t));
  DevHeader hdr;
  memset(&hdr, 0, sizeof hdr);
  hdr.nrows = (uint32_t)w;
  hdr.nmsgs = (uint32_t)count;
  hdr.status_out = status_dev;
  memcpy(g_host_ws, &hdr, sizeof hdr);
  const size_t bytes = sizeof(DevHeader) + count * sizeof(DevMsg) + w * sizeof(DevRow) +
                       count * sizeof(int32_t);

  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LC_ERR_CUDA;
  const int variant = w < (size_t)sms * kSmallBatchRowsPerSm ? kVariantV1Latency : kVariantV1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_ptr(variant), 256,
                                                    batch_kernel_smem(variant)) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  hdr.rows_per_warp = rows_per_warp(w, (uint64_t)sms * per_sm * 8);
  memcpy(g_host_ws, &hdr, sizeof hdr);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* ws = base + kWsOff;
  uint32_t* flags = reinterpret_cast<uint32_t*>(base);
  const double* theta = reinterpret_cast<const double*>(base + kThetaOff);
  // From pageable host memory the copy is staged before the call returns,
  // so the host image may be rebuilt by the next call.
  if (cudaMemcpyAsync(ws, g_host_ws, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return LC_ERR_CUDA;
  if (cudaMemsetAsync(flags, 0, (4 + count) * sizeof(uint32_t), s) != cudaSuccess) return LC_ERR_CUDA;
  if (launch_batch(variant, sms * per_sm, 256, ws, flags, dp, theta, s) != cudaSuccess) return LC_ERR_CUDA;
  if (launch_finalize(256, ws, flags, p.block_len, s) != cudaSuccess) return LC_ERR_CUDA;
  return LC_OK;
}
