// api.cu -- the C ABI of liblorenzcipher (include/lc.h): contexts, the
// flattened part table of the batched path, its CUDA graph, host-buffer
// staging, the launch-shape autotuner and kernel timing.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "keysched.h"
#include "lc_internal.h"

namespace lc {
int kernel_variant(const DevParams& p);
size_t batch_kernel_smem(int variant);
const void* batch_kernel_ptr(int variant);
cudaError_t launch_batch(int variant, int grid, int block, const uint8_t* ws, uint32_t* scratch,
                         const DevParams& p, const double* theta, cudaStream_t s,
                         unsigned long long* dig = nullptr, unsigned long long* ct = nullptr);
cudaError_t launch_finalize(int grid, const uint8_t* ws, const uint32_t* scratch, uint32_t block_len,
                            cudaStream_t s);
cudaError_t launch_synth(uint8_t* dst, uint64_t n, uint64_t seed, uint64_t offset, cudaStream_t s);
cudaError_t launch_ct_stats_fixup(int grid, const uint8_t* ws, uint32_t block_len, uint32_t tag_len,
                                  unsigned long long* ct, cudaStream_t s);
uint32_t emu_mask();
uint32_t warm_mask();
uint32_t partial_mask();
cudaError_t launch_stats(const uint8_t* data, uint64_t n, uint32_t max_lag, unsigned long long* acc,
                         int sms, cudaStream_t s);
}  // namespace lc

using namespace lc;

namespace {

constexpr int kFinalizeGrid = 1024;

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
};

struct Staging {
  uint8_t* host = nullptr;  // pinned
  size_t cap = 0;
  cudaEvent_t done = nullptr;  // the H2D copy out of this slot has finished
  bool used = false;
};

// Device staging of one host-buffer batch in flight.
struct HostSlot {
  uint8_t* io_dev = nullptr;  // the batch's inputs and outputs
  size_t io_cap = 0;
  int32_t* status_dev = nullptr;
  size_t status_cap = 0;
  // Statuses land in pinned memory first (a copy into pageable memory would
  // make the enqueueing call wait for the batch) and reach the caller's
  // array when the batch is retired.
  int32_t* status_pinned = nullptr;
  size_t status_pinned_cap = 0;
  int32_t* status_user = nullptr;
  size_t status_count = 0;
  std::vector<cudaEvent_t> events;  // per chunk: inputs uploaded, chunk computed; + 1
  cudaEvent_t done = nullptr;       // outputs and statuses are in host memory
  uint64_t ticket = 0;              // the batch staged here, 0 if none
};

}  // namespace

struct lc_ctx {
  int device = 0;
  int sm_count = 0;
  lc_params params{};
  DevParams dparams{};
  int variant = kVariantV1;

  double* theta_dev = nullptr;
  uint8_t* ws_dev = nullptr;  // header | msgs | rows | init status
  size_t ws_cap = 0;
  uint32_t* scratch_dev = nullptr;  // counter(4 words) | fail flags
  size_t fail_cap = 0;              // messages covered by the fail flags
  int32_t* status_tmp_dev = nullptr;
  size_t status_tmp_cap = 0;
  unsigned long long* stats_dev = nullptr;  // lc_byte_stats accumulators
  bool digits = false;                      // count the Fig. 1 digit statistics
  unsigned long long* digits_dev = nullptr;  // 3 * kDigBins counters
  bool ct_stats = false;                     // accumulate the ciphertexts' byte statistics
  unsigned long long* ct_stats_dev = nullptr;  // kCtStatsWords counters
  uint64_t ct_stats_bytes = 0;               // ciphertext bytes counted since enabled
  cudaStream_t copy_in = nullptr, copy_out = nullptr;  // host-buffer batch copies
  HostSlot hslots[LC_HOST_INFLIGHT];
  uint64_t next_ticket = 1;
  cudaEvent_t last_batch_done = nullptr;  // the context's latest batch has finished
  cudaStream_t last_batch_stream = nullptr;

  Staging staging[2];
  int slot = 0;

  cudaStream_t cap_stream = nullptr;
  // one captured graph per kernel variant
  struct GraphSlot {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t ev_node_a = nullptr, ev_node_b = nullptr;
    cudaGraphNode_t kernel_node = nullptr;  // the cipher kernel
    cudaKernelNodeParams kparams{};         // its launch parameters as captured
    bool valid = false;
    int grid = 0;      // CTAs of the full persistent grid
    int cur_grid = 0;  // CTAs the executable graph launches now
  } graphs[kNumVariants];

  lc_launch launch{256, 0, 0, 0, 0, 0, 0, 0};
  std::vector<lc_tune_entry> tune_report;  // the last lc_tune's candidates

  std::unordered_map<std::string, HostKey> keys;

  bool timing = false;
  std::vector<EventPair> ev_free, ev_pending;
  double total_ms = 0.0;
  uint64_t timed_launches = 0;
  uint64_t launches = 0;

  std::vector<DevMsg> h_msgs;
  std::vector<DevRow> h_rows;
  std::vector<int32_t> h_init;
};

namespace {

thread_local char g_last_error[256] = "";

lc_status cuda_fail(cudaError_t e, const char* what = nullptr, int line = 0) {
  if (e == cudaSuccess) return LC_OK;
  snprintf(g_last_error, sizeof g_last_error, "%s (%d) at api.cu:%d: %s", cudaGetErrorName(e), (int)e,
           line, what ? what : "");
  if (e == cudaErrorMemoryAllocation) return LC_ERR_NOMEM;
  return LC_ERR_CUDA;
}

#define LC_CUDA(expr)                                            \
  do {                                                           \
    cudaError_t _e = (expr);                                     \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr, __LINE__); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void to_dev_params(const lc_params& p, DevParams* d) {
  d->sigma = p.sigma;
  d->rho = p.rho;
  d->beta = p.beta;
  d->dt = p.dt;
  d->eta = p.eta;
  d->n_warm = p.n_warm;
  d->steps_per_byte = p.steps_per_byte;
  d->block_len = p.block_len;
  d->tag_len = p.tag_len;
  for (int i = 0; i < 3; i++) d->k[i] = p.k[i];
  d->k_all4 = (p.k[0] == 4 && p.k[1] == 4 && p.k[2] == 4) ? 1u : 0u;
  d->omega_alpha_shift = p.omega_alpha_shift;
}

size_t nblocks_of(const lc_params& p, size_t n, lc_mode m) {
  if (m == LC_SEQUENTIAL || n == 0) return 1;
  return (n + p.block_len - 1) / p.block_len;
}

size_t ct_len(const lc_params& p, size_t n, lc_mode m) {
  return n + (size_t)p.tag_len * nblocks_of(p, n, m);
}

bool pt_len(const lc_params& p, size_t c, lc_mode m, size_t* n) {
  if (c < p.tag_len) return false;
  if (m == LC_SEQUENTIAL) {
    *n = c - p.tag_len;
    return true;
  }
  const size_t per = (size_t)p.block_len + p.tag_len;
  const size_t guess = c / per;
  for (size_t nb = std::max<size_t>(guess, 1); nb <= guess + 1; nb++) {
    if ((size_t)p.tag_len * nb > c) break;
    const size_t cand = c - (size_t)p.tag_len * nb;
    if (nblocks_of(p, cand, LC_PARALLEL) == nb) {
      *n = cand;
      return true;
    }
  }
  return false;
}

bool ranges_conflict(const void* a, size_t alen, const void* b, size_t blen) {
  if (a == b) return false;  // exact in-place is allowed
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return alen && blen && x < y + blen && y < x + alen;
}

lc_status get_key(lc_ctx* ctx, const uint8_t* pw, size_t n, const HostKey** out) {
  if (pw == nullptr || n < 1 || n > 32) return LC_ERR_PASSWORD;
  std::string k(reinterpret_cast<const char*>(pw), n);
  auto it = ctx->keys.find(k);
  if (it == ctx->keys.end()) {
    HostKey hk;
    lc_status st = key_schedule(ctx->params, pw, n, &hk);
    if (st != LC_OK) return st;
    if (ctx->keys.size() > 65536) ctx->keys.clear();
    it = ctx->keys.emplace(std::move(k), hk).first;
  }
  *out = &it->second;
  return LC_OK;
}

template <typename T>
lc_status grow_device(T** ptr, size_t* cap, size_t need_elems, bool* changed) {
  if (need_elems <= *cap) return LC_OK;
  size_t n = std::max<size_t>(need_elems, *cap + *cap / 2);
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  LC_CUDA(cudaMalloc(reinterpret_cast<void**>(ptr), n * sizeof(T)));
  *cap = n;
  if (changed) *changed = true;
  return LC_OK;
}

void release_graph(lc_ctx* ctx) {
  for (auto& g : ctx->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g.exec = nullptr;
    g.graph = nullptr;
    g.ev_node_a = g.ev_node_b = nullptr;
    g.kernel_node = nullptr;
    g.valid = false;
  }
}

void invalidate_graphs(lc_ctx* ctx) {
  for (auto& g : ctx->graphs) g.valid = false;
}

lc_status event_pair(lc_ctx* ctx, EventPair* ep) {
  if (!ctx->ev_free.empty()) {
    *ep = ctx->ev_free.back();
    ctx->ev_free.pop_back();
    return LC_OK;
  }
  LC_CUDA(cudaEventCreate(&ep->a));
  LC_CUDA(cudaEventCreate(&ep->b));
  return LC_OK;
}

lc_status drain_timing(lc_ctx* ctx) {
  for (auto& ep : ctx->ev_pending) {
    LC_CUDA(cudaEventSynchronize(ep.b));
    float ms = 0.f;
    LC_CUDA(cudaEventElapsedTime(&ms, ep.a, ep.b));
    ctx->total_ms += ms;
    ctx->timed_launches++;
    ctx->ev_free.push_back(ep);
  }
  ctx->ev_pending.clear();
  return LC_OK;
}

int resident_ctas(int variant, int threads) {
  int per_sm = 0;
  const void* fn = batch_kernel_ptr(variant);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads,
                                                    batch_kernel_smem(variant)) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm;
}

// Graph of variant v: clear the counter and fail flags -> event A ->
// persistent cipher kernel -> event B -> finalize.  Kernel arguments are
// fixed workspace pointers; the per-batch sizes live in the uploaded header,
// so replays need no re-capture until the workspace moves or the shape
// changes.
lc_status build_graph(lc_ctx* ctx, int v) {
  auto& G = ctx->graphs[v];
  if (G.exec) cudaGraphExecDestroy(G.exec);
  if (G.graph) cudaGraphDestroy(G.graph);
  G.exec = nullptr;
  G.graph = nullptr;
  G.valid = false;
  // the counting and split variants have CTA shapes of their own
  const int threads = v == kVariantV1Split       ? kSplitThreads
                      : variant_has_ct_stats(v) ? kCtStatsThreads
                                                : (int)ctx->launch.threads_per_cta;
  int per_sm = resident_ctas(v, threads);
  if (ctx->launch.ctas_per_sm) per_sm = std::min<int>(per_sm, (int)ctx->launch.ctas_per_sm);
  G.grid = ctx->sm_count * per_sm;

  EventPair ep;
  lc_status st = event_pair(ctx, &ep);
  if (st != LC_OK) return st;
  ctx->ev_free.push_back(ep);

  cudaStream_t s = ctx->cap_stream;
  LC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemsetAsync(ctx->scratch_dev, 0, (4 + ctx->fail_cap) * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaEventRecordWithFlags(ep.a, s, cudaEventRecordExternal);
  if (e == cudaSuccess)
    e = launch_batch(v, G.grid, threads, ctx->ws_dev, ctx->scratch_dev, ctx->dparams, ctx->theta_dev, s,
                     ctx->digits_dev, ctx->ct_stats_dev);
  if (e == cudaSuccess) e = cudaEventRecordWithFlags(ep.b, s, cudaEventRecordExternal);
  if (e == cudaSuccess)
    e = launch_finalize(kFinalizeGrid, ctx->ws_dev, ctx->scratch_dev, ctx->params.block_len, s);
  if (e == cudaSuccess && variant_has_ct_stats(v))
    e = launch_ct_stats_fixup(kFinalizeGrid, ctx->ws_dev, ctx->params.block_len, ctx->params.tag_len,
                              ctx->ct_stats_dev, s);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e != cudaSuccess ? e : e2);
  }
  G.graph = g;
  size_t nn = 0;
  LC_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  LC_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
  G.kernel_node = nullptr;
  for (auto nd : nodes) {
    cudaGraphNodeType ty;
    LC_CUDA(cudaGraphNodeGetType(nd, &ty));
    if (ty == cudaGraphNodeTypeEventRecord) {
      cudaEvent_t ev;
      LC_CUDA(cudaGraphEventRecordNodeGetEvent(nd, &ev));
      if (ev == ep.a) G.ev_node_a = nd;
      if (ev == ep.b) G.ev_node_b = nd;
    } else if (ty == cudaGraphNodeTypeKernel) {
      cudaKernelNodeParams kp{};
      LC_CUDA(cudaGraphKernelNodeGetParams(nd, &kp));
      if (kp.func == batch_kernel_ptr(v)) {
        G.kernel_node = nd;
        G.kparams = kp;
      }
    }
  }
  if (!G.kernel_node) return LC_ERR_CUDA;
  LC_CUDA(cudaGraphInstantiate(&G.exec, g, 0));
  G.cur_grid = G.grid;
  G.valid = true;
  return LC_OK;
}

// Kernel variant for a batch of nrows parts: v1 batches that cannot fill
// the GPU run the latency variant.
int batch_variant(const lc_ctx* ctx, size_t nrows, bool msg_k = false) {
  // a request with its own k other than (4, 4, 4) needs a build that reads
  // k per message
  const bool v1 = !msg_k && ctx->variant == kVariantV1;
  if (ctx->ct_stats) {
    if (ctx->digits) return v1 ? kVariantV1DigitsCtStats : kVariantGeneralDigitsCtStats;
    return v1 ? kVariantV1CtStats : kVariantGeneralCtStats;
  }
  const uint64_t thr = ctx->launch.small_batch_rows ? ctx->launch.small_batch_rows
                                                    : (uint64_t)ctx->sm_count * kSmallBatchRowsPerSm;
  if (msg_k) {
    // k in {3, 4}^3 per message: the v1 build that reads k per message for
    // batches that fill the GPU, the general path for the rest
    if (ctx->digits) return kVariantGeneralDigits;
    return ctx->variant == kVariantV1 && nrows >= thr ? kVariantV1MsgK : kVariantGeneral;
  }
  if (ctx->digits) return ctx->variant == kVariantV1 ? kVariantV1Digits : kVariantGeneralDigits;
  if (ctx->variant != kVariantV1) return ctx->variant;
  if (nrows < thr) {
    // auto: one Euler step per byte only (with more, the exchanges outweigh the gain)
    const uint64_t split = ctx->launch.split_rows ? ctx->launch.split_rows
                           : ctx->params.steps_per_byte == 1 ? (uint64_t)ctx->sm_count * kSplitBatchRowsPerSm
                                                             : 0;
    return nrows < split ? kVariantV1Split : kVariantV1Latency;
  }
  const int full = ctx->launch.dense_build ? kVariantV1Dense : kVariantV1;
  // a batch that does not fill the persistent grid runs on fewer CTAs per SM
  uint64_t fill = ctx->launch.full_grid_rows;
  if (!fill) {
    const int threads = (int)ctx->launch.threads_per_cta;
    int per_sm = resident_ctas(full, threads);
    if (ctx->launch.ctas_per_sm) per_sm = std::min<int>(per_sm, (int)ctx->launch.ctas_per_sm);
    fill = (uint64_t)ctx->sm_count * (uint64_t)per_sm * (uint64_t)threads;
  }
  if (nrows >= fill) return full;
  return ctx->launch.dense_build ? kVariantV1PartialDense : kVariantV1Partial;
}

// Host validation of one request; LC_OK or the request's status code.
int32_t validate_req(const lc_params& p, const lc_req& r, lc_mode m, size_t* n_out) {
  size_t n = 0;
  int32_t st = LC_OK;
  if (r.dir > 1) {
    st = LC_ERR_ARG;
  } else if (r.dir == LC_ENCRYPT) {
    n = r.in_len;
    if ((n && !r.in) || !r.out) st = LC_ERR_ARG;
    else if (r.out_cap < ct_len(p, n, m)) st = LC_ERR_LENGTH;
    else if (ranges_conflict(r.in, n, r.out, ct_len(p, n, m))) st = LC_ERR_ARG;
  } else {
    if (!r.in) st = LC_ERR_ARG;
    else if (!pt_len(p, r.in_len, m, &n)) st = LC_ERR_LENGTH;
    else if (n && !r.out) st = LC_ERR_ARG;
    else if (r.out_cap < n) st = LC_ERR_LENGTH;
    else if (ranges_conflict(r.in, r.in_len, r.out, n)) st = LC_ERR_ARG;
  }
  if (st == LC_OK && (!r.pw || r.pw_len < 1 || r.pw_len > 32)) st = LC_ERR_PASSWORD;
  *n_out = n;
  return st;
}


// Per-request key material (lc_req_ex): lambda inside the ranges Sec. 3.1
// gives for Eq. 5, k with 2 < k_i <= floor((52 - 14) / 8) = 4 (Eq. 7).
int32_t validate_key_ex(const lc_req_ex& e) {
  if (e.key_flags & ~(uint32_t)(LC_KEY_LAMBDA | LC_KEY_K)) return LC_ERR_ARG;
  if (e.key_flags & LC_KEY_LAMBDA) {
    const double lo[3] = {-15.67, -11.28, 0.090}, hi[3] = {16.01, 16.01, 62.0};
    for (int j = 0; j < 3; j++)
      if (!(e.lambda[j] > lo[j] && e.lambda[j] < hi[j])) return LC_ERR_ARG;
  }
  if (e.key_flags & LC_KEY_K)
    for (int j = 0; j < 3; j++)
      if (e.k[j] < 3 || e.k[j] > 4) return LC_ERR_ARG;
  return LC_OK;
}

// Validate the requests, build the message and part tables (parts sorted
// longest first so warps hold parts of equal length), upload them and
// replay the graph on `s`.  ex (optional) gives each request's own key
// material; then reqs is ignored.
lc_status run_batch_impl(lc_ctx* ctx, const lc_req* reqs, size_t count, int32_t* status_dev,
                         lc_mode m, cudaStream_t s, const lc_req_ex* ex = nullptr) {
  const lc_params& p = ctx->params;
  ctx->h_msgs.resize(count);
  ctx->h_init.resize(count);
  ctx->h_rows.clear();
  size_t full_rows = 0;
  std::vector<DevRow> partial;
  bool msg_k = false;  // some request's k differs from (4, 4, 4)

  for (size_t i = 0; i < count; i++) {
    const lc_req& r = ex ? ex[i].req : reqs[i];
    DevMsg& M = ctx->h_msgs[i];
    memset(&M, 0, sizeof M);
    size_t n = 0;
    const HostKey* key = nullptr;
    int32_t init = validate_req(p, r, m, &n);
    if (init == LC_OK && ex) init = validate_key_ex(ex[i]);
    if (init == LC_OK) {
      lc_status ks = get_key(ctx, r.pw, r.pw_len, &key);
      if (ks != LC_OK) init = ks;
    }
    ctx->h_init[i] = init;
    if (init != LC_OK) continue;
    M.in = r.in;
    M.out = r.out;
    M.n = n;
    const bool own_lam = ex && (ex[i].key_flags & LC_KEY_LAMBDA);
    const bool own_k = ex && (ex[i].key_flags & LC_KEY_K);
    for (int j = 0; j < 3; j++) {
      const double lam = own_lam ? ex[i].lambda[j] : p.lambda[j];
      M.base[j] = key->aprime[j] + lam;  // one rounding, Eq. 5
      M.aprime[j] = key->aprime[j];
    }
    uint32_t om[3];
    for (int j = 0; j < 3; j++) om[j] = own_k ? key->omega_mod[j][ex[i].k[j]] : key->omega[j];
    M.key_bits = key->mu[0] | key->mu[1] << 2 | key->mu[2] << 4 | om[0] << 8 | om[1] << 12 | om[2] << 16;
    M.flags = (r.dir == LC_DECRYPT ? kFlagDecrypt : 0u) | (m == LC_SEQUENTIAL ? kFlagSequential : 0u);
    if (own_k) {
      M.key_bits |= ex[i].k[0] << 20 | ex[i].k[1] << 24 | ex[i].k[2] << 28;
      M.flags |= kFlagMsgK;
      if (ex[i].k[0] != 4 || ex[i].k[1] != 4 || ex[i].k[2] != 4) msg_k = true;
    }
    const size_t nb = nblocks_of(p, n, m);
    if (nb > 0xFFFFFFFFull) return LC_ERR_ARG;
    for (size_t b = 0; b < nb; b++) {
      const size_t len = (m == LC_SEQUENTIAL) ? n : std::min<size_t>(p.block_len, n - b * p.block_len);
      DevRow row{(uint32_t)i, (uint32_t)b};
      if (m == LC_PARALLEL && len == p.block_len) {
        ctx->h_rows.push_back(row);
        full_rows++;
      } else {
        partial.push_back(row);
      }
    }
  }
  // Longest first: full parts, then the rest by decreasing length.
  auto row_len = [&](const DevRow& r) -> size_t {
    const DevMsg& M = ctx->h_msgs[r.msg];
    if (M.flags & kFlagSequential) return M.n;
    return std::min<size_t>(p.block_len, M.n - (size_t)r.b * p.block_len);
  };
  std::stable_sort(partial.begin(), partial.end(),
                   [&](const DevRow& a, const DevRow& b) { return row_len(a) > row_len(b); });
  ctx->h_rows.insert(ctx->h_rows.end(), partial.begin(), partial.end());
  if (ctx->h_rows.size() > 0xFFFFFFF0ull || count > 0xFFFFFFF0ull) return LC_ERR_ARG;

  const size_t nrows = ctx->h_rows.size();
  const size_t bytes = sizeof(DevHeader) + count * sizeof(DevMsg) + nrows * sizeof(DevRow) +
                       count * sizeof(int32_t);
  // Ciphertext bytes this batch adds to the fused statistics: the CTAs'
  // 32-bit histogram columns stay exact below 2^32 bytes per batch.
  uint64_t ct_bytes = 0;
  if (ctx->ct_stats) {
    for (size_t i = 0; i < count; i++)
      if (ctx->h_init[i] == LC_OK && !(ctx->h_msgs[i].flags & kFlagDecrypt))
        ct_bytes += ct_len(p, (size_t)ctx->h_msgs[i].n, m);
    if (ct_bytes > 0xFFFFFFFFull) return LC_ERR_ARG;
  }

  // Device workspace (graphs are rebuilt whenever a buffer moves).
  const int v = batch_variant(ctx, nrows, msg_k);
  bool changed = false;
  lc_status st = grow_device(&ctx->ws_dev, &ctx->ws_cap, bytes, &changed);
  if (st != LC_OK) return st;
  size_t fail_need = std::max<size_t>(count, 1024);
  if (fail_need > ctx->fail_cap) {
    size_t cap_words = 4 + std::max(fail_need, ctx->fail_cap + ctx->fail_cap / 2);
    if (ctx->scratch_dev) cudaFree(ctx->scratch_dev);
    ctx->scratch_dev = nullptr;
    ctx->fail_cap = 0;
    LC_CUDA(cudaMalloc(&ctx->scratch_dev, cap_words * sizeof(uint32_t)));
    LC_CUDA(cudaMemset(ctx->scratch_dev, 0, cap_words * sizeof(uint32_t)));
    ctx->fail_cap = cap_words - 4;
    changed = true;
  }
  if (changed) invalidate_graphs(ctx);
  if (!ctx->graphs[v].valid) {
    st = build_graph(ctx, v);
    if (st != LC_OK) return st;
  }
  auto& G = ctx->graphs[v];

  // Pinned staging, double-buffered: wait until the copy that last used
  // this slot has left it.
  Staging& sg = ctx->staging[ctx->slot];
  ctx->slot ^= 1;
  if (sg.used) LC_CUDA(cudaEventSynchronize(sg.done));
  if (sg.cap < bytes) {
    if (sg.host) cudaFreeHost(sg.host);
    sg.host = nullptr;
    sg.cap = 0;
    size_t cap = std::max(bytes, (size_t)1 << 20);
    LC_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&sg.host), cap, cudaHostAllocDefault));
    sg.cap = cap;
  }
  if (!sg.done) LC_CUDA(cudaEventCreateWithFlags(&sg.done, cudaEventDisableTiming));
  DevHeader hdr;
  memset(&hdr, 0, sizeof hdr);
  hdr.nrows = (uint32_t)nrows;
  hdr.nmsgs = (uint32_t)count;
  hdr.status_out = status_dev;
  // Grid of this launch: whole CTAs per SM, as few as give every row a
  // thread in the first pass (the per-SM load stays the same), so that a
  // batch smaller than the GPU leaves CTA slots for other streams' batches.
  const uint64_t threads = variant_has_ct_stats(v) ? (uint64_t)kCtStatsThreads : ctx->launch.threads_per_cta;
  const int full_per_sm = std::max(1, G.grid / std::max(1, ctx->sm_count));
  const uint64_t need = (nrows + (uint64_t)ctx->sm_count * threads - 1) / ((uint64_t)ctx->sm_count * threads);
  int grid = ctx->sm_count * (int)std::min<uint64_t>(std::max<uint64_t>(need, 1), (uint64_t)full_per_sm);
  // the split kernel: one CTA per 32 parts (not persistent)
  if (v == kVariantV1Split)
    grid = (int)std::max<uint64_t>(1, (nrows + kSplitRowsPerCta - 1) / kSplitRowsPerCta);
  hdr.rows_per_warp = rows_per_warp(nrows, (uint64_t)grid * (threads / 32));
  uint8_t* w = sg.host;
  memcpy(w, &hdr, sizeof hdr);
  w += sizeof hdr;
  if (count) memcpy(w, ctx->h_msgs.data(), count * sizeof(DevMsg));
  w += count * sizeof(DevMsg);
  if (nrows) memcpy(w, ctx->h_rows.data(), nrows * sizeof(DevRow));
  w += nrows * sizeof(DevRow);
  if (count) memcpy(w, ctx->h_init.data(), count * sizeof(int32_t));

  // Every batch of a context uses the same workspace: when the caller
  // switches streams, this batch's upload waits on the GPU for the previous
  // batch (its kernels read the workspace until they finish).
  if (ctx->last_batch_done && ctx->last_batch_stream != s)
    LC_CUDA(cudaStreamWaitEvent(s, ctx->last_batch_done, 0));
  LC_CUDA(cudaMemcpyAsync(ctx->ws_dev, sg.host, bytes, cudaMemcpyHostToDevice, s));
  LC_CUDA(cudaEventRecord(sg.done, s));
  sg.used = true;

  if (ctx->timing) {
    EventPair ep;
    st = event_pair(ctx, &ep);
    if (st != LC_OK) return st;
    LC_CUDA(cudaGraphExecEventRecordNodeSetEvent(G.exec, G.ev_node_a, ep.a));
    LC_CUDA(cudaGraphExecEventRecordNodeSetEvent(G.exec, G.ev_node_b, ep.b));
    ctx->ev_pending.push_back(ep);
    if (ctx->ev_pending.size() > 4096) {
      st = drain_timing(ctx);
      if (st != LC_OK) return st;
    }
  }
  if (grid != G.cur_grid) {
    cudaKernelNodeParams kp = G.kparams;
    kp.gridDim = dim3((unsigned)grid, 1, 1);
    LC_CUDA(cudaGraphExecKernelNodeSetParams(G.exec, G.kernel_node, &kp));
    G.cur_grid = grid;
  }
  LC_CUDA(cudaGraphLaunch(G.exec, s));
  ctx->launches += variant_has_ct_stats(v) ? 3 : 2;  // cipher kernel + finalize (+ statistics fix-up)
  ctx->ct_stats_bytes += ct_bytes;
#ifdef LC_CHECKED
  {
    // Checked build: wait for the batch and report a table index or part
    // range the kernel found invalid (it skipped them).
    uint32_t chk[2] = {0, 0};
    LC_CUDA(cudaMemcpyAsync(chk, ctx->scratch_dev + 1, sizeof chk, cudaMemcpyDeviceToHost, s));
    LC_CUDA(cudaStreamSynchronize(s));
    if (chk[0]) {
      snprintf(g_last_error, sizeof g_last_error, "checked build: invalid part table entry %u (flags %u)",
               chk[1] ? chk[1] - 1u : 0u, chk[0]);
      return LC_ERR_CUDA;
    }
  }
#endif
  if (!ctx->last_batch_done)
    LC_CUDA(cudaEventCreateWithFlags(&ctx->last_batch_done, cudaEventDisableTiming));
  LC_CUDA(cudaEventRecord(ctx->last_batch_done, s));
  ctx->last_batch_stream = s;
  return LC_OK;
}

lc_status ensure_status_tmp(lc_ctx* ctx, size_t count) {
  return grow_device(&ctx->status_tmp_dev, &ctx->status_tmp_cap, std::max<size_t>(count, 1), nullptr);
}

}  // namespace

namespace lc {
// Request validation, framing lengths and kernel parameters, shared with
// other entry points.
int32_t validate_request(const lc_params& p, const lc_req& r, lc_mode m, size_t* n) {
  return validate_req(p, r, m, n);
}
void dev_params_from(const lc_params& p, DevParams* d) { to_dev_params(p, d); }
size_t parts_of(const lc_params& p, size_t n, lc_mode m) { return nblocks_of(p, n, m); }
}  // namespace lc

// ===========================================================================
// Public ABI
// ===========================================================================

extern "C" {

uint32_t lc_version(void) { return LC_PARAMS_VERSION; }

uint32_t lc_build_flags(void) {
#ifdef LC_CHECKED
  return LC_BUILD_CHECKED;
#else
  return 0u;
#endif
}

const char* lc_last_cuda_error(void) { return g_last_error; }

const char* lc_status_string(lc_status s) {
  switch (s) {
    case LC_OK: return "ok";
    case LC_ERR_ARG: return "invalid argument";
    case LC_ERR_PASSWORD: return "password length outside 1..32 bytes";
    case LC_ERR_LENGTH: return "invalid length or buffer too small";
    case LC_ERR_INTEGRITY: return "integrity check failed";
    case LC_ERR_CUDA: return "CUDA error";
    case LC_ERR_TIMEOUT: return "device wait timed out";
    case LC_ERR_NOMEM: return "out of device memory";
  }
  return "unknown status";
}

lc_status lc_params_default(lc_params* out) {
  if (!out) return LC_ERR_ARG;
  out->sigma = 10.0;
  out->rho = 28.0;
  out->beta = 8.0 / 3.0;
  out->dt = 0.01;
  out->n_warm = 3000;
  out->steps_per_byte = 1;
  out->lambda[0] = 1.0;
  out->lambda[1] = 1.0;
  out->lambda[2] = 20.0;
  out->k[0] = out->k[1] = out->k[2] = 4;
  out->block_len = 4096;
  out->tag_len = 8;
  out->eta = 1.0 / 16777216.0;
  out->omega_alpha_shift = 0;
  out->reserved = 0;
  return LC_OK;
}

lc_status lc_ctx_create(int device, lc_ctx** out) {
  if (!out) return LC_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LC_ERR_CUDA;
  lc_ctx* ctx = new (std::nothrow) lc_ctx();
  if (!ctx) return LC_ERR_NOMEM;
  ctx->device = device;
  DeviceGuard g(device);
  lc_params_default(&ctx->params);
  to_dev_params(ctx->params, &ctx->dparams);
  ctx->variant = kernel_variant(ctx->dparams);
  lc_status st = LC_OK;
  cudaError_t e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->theta_dev, kThetaEntries * sizeof(double));
  if (e == cudaSuccess) {
    std::vector<double> th(kThetaEntries);
    build_theta(th.data());
    e = cudaMemcpy(ctx->theta_dev, th.data(), kThetaEntries * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    for (int v = 0; v < kNumVariants; v++) {
      e = cudaFuncSetAttribute(batch_kernel_ptr(v), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)batch_kernel_smem(v));
      if (e != cudaSuccess) break;
    }
  }
  if (e != cudaSuccess) st = cuda_fail(e);
  if (st != LC_OK) {
    lc_ctx_destroy(ctx);
    return st;
  }
  *out = ctx;
  return LC_OK;
}

void lc_ctx_destroy(lc_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  release_graph(ctx);
  for (auto& ep : ctx->ev_free) {
    cudaEventDestroy(ep.a);
    cudaEventDestroy(ep.b);
  }
  for (auto& ep : ctx->ev_pending) {
    cudaEventDestroy(ep.a);
    cudaEventDestroy(ep.b);
  }
  for (auto& sg : ctx->staging) {
    if (sg.host) cudaFreeHost(sg.host);
    if (sg.done) cudaEventDestroy(sg.done);
  }
  if (ctx->theta_dev) cudaFree(ctx->theta_dev);
  if (ctx->ws_dev) cudaFree(ctx->ws_dev);
  if (ctx->scratch_dev) cudaFree(ctx->scratch_dev);
  if (ctx->status_tmp_dev) cudaFree(ctx->status_tmp_dev);
  for (auto& h : ctx->hslots) {
    if (h.io_dev) cudaFree(h.io_dev);
    if (h.status_dev) cudaFree(h.status_dev);
    if (h.status_pinned) cudaFreeHost(h.status_pinned);
    for (auto ev : h.events) cudaEventDestroy(ev);
    if (h.done) cudaEventDestroy(h.done);
  }
  if (ctx->stats_dev) cudaFree(ctx->stats_dev);
  if (ctx->digits_dev) cudaFree(ctx->digits_dev);
  if (ctx->ct_stats_dev) cudaFree(ctx->ct_stats_dev);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->copy_in) cudaStreamDestroy(ctx->copy_in);
  if (ctx->copy_out) cudaStreamDestroy(ctx->copy_out);
  if (ctx->last_batch_done) cudaEventDestroy(ctx->last_batch_done);
  delete ctx;
}

lc_status lc_ctx_set_params(lc_ctx* ctx, const lc_params* p) {
  if (!ctx || !p || !params_valid(*p)) return LC_ERR_ARG;
  ctx->params = *p;
  to_dev_params(*p, &ctx->dparams);
  ctx->variant = kernel_variant(ctx->dparams);
  ctx->keys.clear();
  invalidate_graphs(ctx);
  return LC_OK;
}

lc_status lc_ctx_get_params(const lc_ctx* ctx, lc_params* p) {
  if (!ctx || !p) return LC_ERR_ARG;
  *p = ctx->params;
  return LC_OK;
}

size_t lc_ciphertext_len(const lc_ctx* ctx, size_t n, lc_mode m) {
  lc_params p;
  if (ctx) p = ctx->params; else lc_params_default(&p);
  return ct_len(p, n, m);
}

lc_status lc_plaintext_len(const lc_ctx* ctx, size_t c_len, lc_mode m, size_t* n) {
  if (!n) return LC_ERR_ARG;
  lc_params p;
  if (ctx) p = ctx->params; else lc_params_default(&p);
  return pt_len(p, c_len, m, n) ? LC_OK : LC_ERR_LENGTH;
}

lc_status lc_run_batch(lc_ctx* ctx, const lc_req* reqs, size_t count, int32_t* status_dev, lc_mode m,
                       void* stream) {
  if (!ctx || (!reqs && count) || (!status_dev && count)) return LC_ERR_ARG;
  if (m != LC_PARALLEL && m != LC_SEQUENTIAL) return LC_ERR_ARG;
  if (count == 0) return LC_OK;
  DeviceGuard g(ctx->device);
  return run_batch_impl(ctx, reqs, count, status_dev, m, static_cast<cudaStream_t>(stream));
}

lc_status lc_run_batch_ex(lc_ctx* ctx, const lc_req_ex* reqs, size_t count, int32_t* status_dev,
                          lc_mode m, void* stream) {
  if (!ctx || (!reqs && count) || (!status_dev && count)) return LC_ERR_ARG;
  if (m != LC_PARALLEL && m != LC_SEQUENTIAL) return LC_ERR_ARG;
  if (count == 0) return LC_OK;
  DeviceGuard g(ctx->device);
  return run_batch_impl(ctx, nullptr, count, status_dev, m, static_cast<cudaStream_t>(stream), reqs);
}

lc_status lc_encrypt(lc_ctx* ctx, const uint8_t* pw, size_t pw_len, const uint8_t* P_dev, size_t n,
                     uint8_t* C_dev, size_t c_cap, lc_mode m, void* stream) {
  if (!ctx || (n && !P_dev) || !C_dev) return LC_ERR_ARG;
  if (m != LC_PARALLEL && m != LC_SEQUENTIAL) return LC_ERR_ARG;
  if (pw_len < 1 || pw_len > 32 || !pw) return LC_ERR_PASSWORD;
  if (c_cap < ct_len(ctx->params, n, m)) return LC_ERR_LENGTH;
  if (ranges_conflict(P_dev, n, C_dev, ct_len(ctx->params, n, m))) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  lc_status st = ensure_status_tmp(ctx, 1);
  if (st != LC_OK) return st;
  lc_req r{pw, (uint32_t)pw_len, LC_ENCRYPT, P_dev, n, C_dev, c_cap};
  return run_batch_impl(ctx, &r, 1, ctx->status_tmp_dev, m, static_cast<cudaStream_t>(stream));
}

lc_status lc_decrypt(lc_ctx* ctx, const uint8_t* pw, size_t pw_len, const uint8_t* C_dev, size_t c_len,
                     uint8_t* P_dev, size_t p_cap, lc_mode m, void* stream) {
  if (!ctx || !C_dev) return LC_ERR_ARG;
  if (m != LC_PARALLEL && m != LC_SEQUENTIAL) return LC_ERR_ARG;
  size_t n = 0;
  if (!pt_len(ctx->params, c_len, m, &n)) return LC_ERR_LENGTH;
  if (n && !P_dev) return LC_ERR_ARG;
  if (pw_len < 1 || pw_len > 32 || !pw) return LC_ERR_PASSWORD;
  if (p_cap < n) return LC_ERR_LENGTH;
  if (ranges_conflict(C_dev, c_len, P_dev, n)) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  lc_status st = ensure_status_tmp(ctx, 1);
  if (st != LC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lc_req r{pw, (uint32_t)pw_len, LC_DECRYPT, C_dev, c_len, P_dev, p_cap};
  st = run_batch_impl(ctx, &r, 1, ctx->status_tmp_dev, m, s);
  if (st != LC_OK) return st;
  int32_t verdict = LC_ERR_CUDA;
  LC_CUDA(cudaMemcpyAsync(&verdict, ctx->status_tmp_dev, sizeof verdict, cudaMemcpyDeviceToHost, s));
  LC_CUDA(cudaStreamSynchronize(s));
  return (lc_status)verdict;
}

// ---------------------------------------------------------------------------
// Host-buffer batches: inputs are copied into a staging slot on the device,
// the batch runs there, and outputs and statuses are copied back.  Each
// batch in flight owns one of LC_HOST_INFLIGHT slots, so the copies of one
// batch overlap the kernel of another.
// ---------------------------------------------------------------------------

// Wait for the batch staged in h, if any, hand its statuses over and free
// the slot.
static lc_status retire_slot(HostSlot& h) {
  if (!h.ticket) return LC_OK;
  h.ticket = 0;
  LC_CUDA(cudaEventSynchronize(h.done));
  memcpy(h.status_user, h.status_pinned, h.status_count * sizeof(int32_t));
  return LC_OK;
}

// Enqueue one host-buffer batch into slot h.  after_stream: the input copies
// also wait for the work already on s (the synchronous entry point's stream
// semantics).
static lc_status enqueue_host(lc_ctx* ctx, HostSlot& h, const lc_req* reqs, size_t count,
                              int32_t* status_host, lc_mode m, cudaStream_t s, bool after_stream) {
  const lc_params& p = ctx->params;

  // Bytes each request will write: its full result, clipped to out_cap.
  std::vector<size_t> out_len(count);
  for (size_t i = 0; i < count; i++) {
    const lc_req& r = reqs[i];
    size_t n = 0, olen = 0;
    if (r.dir == LC_ENCRYPT) olen = ct_len(p, r.in_len, m);
    else if (pt_len(p, r.in_len, m, &n)) olen = n;
    out_len[i] = r.out ? std::min(olen, r.out_cap) : 0;
  }

  // Requests whose host buffers follow each other are copied as one run.
  // Each run lands in the device staging area at the same address modulo
  // 256 as on the host, so the kernel's 16-byte vector path applies
  // whenever it would for the host buffers.
  struct Run {
    size_t first, last;
    const uint8_t* h;
    size_t span, dev_off;
  };
  size_t cursor = 0;
  auto plan = [&](bool input, std::vector<Run>& runs) {
    for (size_t i = 0; i < count;) {
      const uint8_t* hp = input ? reqs[i].in : reqs[i].out;
      size_t span = input ? reqs[i].in_len : out_len[i];
      size_t j = i + 1;
      while (hp && j < count) {
        const uint8_t* hj = input ? reqs[j].in : reqs[j].out;
        if (hj != hp + span) break;
        span += input ? reqs[j].in_len : out_len[j];
        j++;
      }
      cursor = (cursor + 255) & ~(size_t)255;
      const size_t off = cursor + (reinterpret_cast<uintptr_t>(hp) & 255u);
      runs.push_back(Run{i, j, hp, span, off});
      cursor = off + span;
      i = j;
    }
  };
  std::vector<Run> in_runs, out_runs;
  plan(true, in_runs);
  plan(false, out_runs);
  lc_status st = grow_device(&h.io_dev, &h.io_cap, std::max<size_t>(cursor, 256), nullptr);
  if (st != LC_OK) return st;
  st = grow_device(&h.status_dev, &h.status_cap, count, nullptr);
  if (st != LC_OK) return st;
  if (h.status_pinned_cap < count) {
    if (h.status_pinned) cudaFreeHost(h.status_pinned);
    h.status_pinned = nullptr;
    h.status_pinned_cap = 0;
    const size_t cap = std::max<size_t>(count, 4096);
    LC_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&h.status_pinned), cap * sizeof(int32_t),
                          cudaHostAllocDefault));
    h.status_pinned_cap = cap;
  }
  h.status_user = status_host;
  h.status_count = count;

  std::vector<lc_req> dreq(reqs, reqs + count);
  for (const Run& r : in_runs)
    for (size_t k = r.first; k < r.last; k++)
      dreq[k].in = r.h ? h.io_dev + r.dev_off + (reqs[k].in - r.h) : nullptr;
  for (const Run& r : out_runs)
    for (size_t k = r.first; k < r.last; k++) {
      dreq[k].out = r.h ? h.io_dev + r.dev_off + (reqs[k].out - r.h) : nullptr;
      dreq[k].out_cap = out_len[k] < reqs[k].out_cap ? out_len[k] : reqs[k].out_cap;
    }

  // Software pipeline over chunks of whole requests: chunk c+1's inputs
  // upload on one copy stream while chunk c computes on `s`, and chunk c's
  // outputs download on a second copy stream while chunk c+1 computes.
  // Each chunk is one kernel launch, and a launch whose parts barely exceed
  // the resident grid runs a nearly empty second wave as long as a full
  // one, so chunks are only cut for batches of several grid waves (>= 4 GiB
  // per chunk); a 2 GB batch split in four ran 17.6 GB/s end to end against
  // 22 GB/s as one launch.  Overlap between batches comes from the slots.
  size_t total_in = 0;
  for (size_t i = 0; i < count; i++) total_in += reqs[i].in_len;
  const size_t chunk = (size_t)(ctx->launch.host_chunk_mib ? ctx->launch.host_chunk_mib : 4096) << 20;
  const size_t K = std::max<size_t>(1, std::min<size_t>(4, total_in / chunk));
  std::vector<size_t> bound{0};
  {
    size_t acc = 0, next = 1;
    for (size_t i = 0; i < count && next < K; i++) {
      acc += reqs[i].in_len;
      if (acc * K >= total_in * next) {
        bound.push_back(i + 1);
        next++;
      }
    }
    if (bound.back() != count) bound.push_back(count);
  }
  // the copies of the requests [a, b) that fall in each run
  auto copy_span = [&](const std::vector<Run>& runs, bool input, size_t a, size_t b,
                       cudaStream_t cs) -> cudaError_t {
    for (const Run& r : runs) {
      const size_t lo = std::max(r.first, a), hi = std::min(r.last, b);
      if (lo >= hi || !r.h) continue;
      const uint8_t* h0 = input ? reqs[lo].in : reqs[lo].out;
      const uint8_t* h1 = input ? reqs[hi - 1].in + reqs[hi - 1].in_len : reqs[hi - 1].out + out_len[hi - 1];
      const size_t len = (size_t)(h1 - h0);
      if (!len) continue;
      uint8_t* d = h.io_dev + r.dev_off + (h0 - r.h);
      cudaError_t e = input ? cudaMemcpyAsync(d, h0, len, cudaMemcpyHostToDevice, cs)
                            : cudaMemcpyAsync(const_cast<uint8_t*>(h0), d, len, cudaMemcpyDeviceToHost, cs);
      if (e == cudaErrorInvalidValue) {
        // Buffers that are adjacent in address space but belong to
        // different page-locked allocations cannot be copied as one range:
        // copy them one request at a time.
        cudaGetLastError();
        e = cudaSuccess;
        for (size_t k = lo; k < hi && e == cudaSuccess; k++) {
          const uint8_t* hk = input ? reqs[k].in : reqs[k].out;
          const size_t lk = input ? reqs[k].in_len : out_len[k];
          if (!lk) continue;
          uint8_t* dk = h.io_dev + r.dev_off + (hk - r.h);
          e = input ? cudaMemcpyAsync(dk, hk, lk, cudaMemcpyHostToDevice, cs)
                    : cudaMemcpyAsync(const_cast<uint8_t*>(hk), dk, lk, cudaMemcpyDeviceToHost, cs);
        }
      }
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  if (!ctx->copy_in) LC_CUDA(cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking));
  if (!ctx->copy_out) LC_CUDA(cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking));
  while (h.events.size() < 2 * K + 1) {
    cudaEvent_t ev;
    LC_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    h.events.push_back(ev);
  }
  if (!h.done) LC_CUDA(cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming));
  cudaEvent_t* evs = h.events.data();
  if (after_stream) {
    LC_CUDA(cudaEventRecord(evs[2 * K], s));
    LC_CUDA(cudaStreamWaitEvent(ctx->copy_in, evs[2 * K], 0));
  }
  for (size_t c = 0; c + 1 < bound.size(); c++) {
    const size_t a = bound[c], b = bound[c + 1];
    LC_CUDA(copy_span(in_runs, true, a, b, ctx->copy_in));
    LC_CUDA(cudaEventRecord(evs[2 * c], ctx->copy_in));
    LC_CUDA(cudaStreamWaitEvent(s, evs[2 * c], 0));
    st = run_batch_impl(ctx, dreq.data() + a, b - a, h.status_dev + a, m, s);
    if (st != LC_OK) return st;
    LC_CUDA(cudaEventRecord(evs[2 * c + 1], s));
    LC_CUDA(cudaStreamWaitEvent(ctx->copy_out, evs[2 * c + 1], 0));
    LC_CUDA(copy_span(out_runs, false, a, b, ctx->copy_out));
  }
  LC_CUDA(cudaMemcpyAsync(h.status_pinned, h.status_dev, count * sizeof(int32_t), cudaMemcpyDeviceToHost,
                          ctx->copy_out));
  LC_CUDA(cudaEventRecord(h.done, ctx->copy_out));
  return LC_OK;
}

// Take a slot (waiting for the oldest batch if all are in use), enqueue the
// batch and hand out its ticket.
static lc_status submit_host(lc_ctx* ctx, const lc_req* reqs, size_t count, int32_t* status_host,
                             lc_mode m, cudaStream_t s, bool after_stream, uint64_t* ticket) {
  const uint64_t t = ctx->next_ticket++;
  *ticket = t;
  if (count == 0) return LC_OK;
  HostSlot* h = &ctx->hslots[0];
  for (auto& c : ctx->hslots)
    if (c.ticket < h->ticket) h = &c;  // a free slot (ticket 0) or the oldest batch
  lc_status st = retire_slot(*h);
  if (st != LC_OK) return st;
  st = enqueue_host(ctx, *h, reqs, count, status_host, m, s, after_stream);
  if (st != LC_OK) {
    // leave nothing of this batch in flight
    cudaStreamSynchronize(ctx->copy_in);
    cudaStreamSynchronize(s);
    cudaStreamSynchronize(ctx->copy_out);
    return st;
  }
  h->ticket = t;
  return LC_OK;
}

static lc_status wait_host(lc_ctx* ctx, uint64_t ticket) {
  lc_status st = LC_OK;
  for (auto& h : ctx->hslots)
    if (h.ticket && h.ticket <= ticket) {
      lc_status r = retire_slot(h);
      if (st == LC_OK) st = r;
    }
  return st;
}

lc_status lc_run_batch_host(lc_ctx* ctx, const lc_req* reqs, size_t count, int32_t* status_host,
                            lc_mode m, void* stream) {
  if (!ctx || (!reqs && count) || (!status_host && count)) return LC_ERR_ARG;
  if (m != LC_PARALLEL && m != LC_SEQUENTIAL) return LC_ERR_ARG;
  if (count == 0) return LC_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint64_t t = 0;
  lc_status st = submit_host(ctx, reqs, count, status_host, m, s, true, &t);
  if (st != LC_OK) return st;
  st = wait_host(ctx, t);
  if (st != LC_OK) return st;
  LC_CUDA(cudaStreamSynchronize(s));
  return LC_OK;
}

lc_status lc_submit_batch_host(lc_ctx* ctx, const lc_req* reqs, size_t count, int32_t* status_host,
                               lc_mode m, void* stream, uint64_t* ticket) {
  if (!ctx || !ticket || (!reqs && count) || (!status_host && count)) return LC_ERR_ARG;
  if (m != LC_PARALLEL && m != LC_SEQUENTIAL) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  return submit_host(ctx, reqs, count, status_host, m, static_cast<cudaStream_t>(stream), false, ticket);
}

lc_status lc_wait_batch_host(lc_ctx* ctx, uint64_t ticket) {
  if (!ctx || ticket == 0 || ticket >= ctx->next_ticket) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  return wait_host(ctx, ticket);
}

lc_status lc_ctx_get_launch(const lc_ctx* ctx, lc_launch* out) {
  if (!ctx || !out) return LC_ERR_ARG;
  *out = ctx->launch;
  return LC_OK;
}

lc_status lc_ctx_set_launch(lc_ctx* ctx, const lc_launch* l) {
  if (!ctx || !l) return LC_ERR_ARG;
  if (l->threads_per_cta < 32 || l->threads_per_cta > 256 || l->threads_per_cta % 32) return LC_ERR_ARG;
  if (l->ctas_per_sm > 64 || l->smem_staging != 0 || l->dense_build > 1) return LC_ERR_ARG;
  ctx->launch = *l;
  invalidate_graphs(ctx);
  return LC_OK;
}

lc_status lc_tune(lc_ctx* ctx, size_t probe_bytes, void* stream, lc_launch* best) {
  if (!ctx) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const lc_params& p = ctx->params;
  const bool v1 = ctx->variant == kVariantV1;
  if (probe_bytes == 0) {
    // four waves, in parts, of the largest persistent grid among the
    // candidates, so that no candidate is timed on a partly filled wave
    int most = 0;
    for (int v : {ctx->variant, v1 ? kVariantV1Dense : ctx->variant})
      for (int tpc : {64, 128, 256}) most = std::max(most, resident_ctas(v, tpc) * tpc);
    probe_bytes = (size_t)4 * ctx->sm_count * most * p.block_len;
  }

  // Probe messages: log-uniform sizes in [1 KiB, 4 MiB] from a SplitMix64
  // counter stream, until probe_bytes are covered.
  auto mix = [](uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  std::vector<size_t> sizes;
  size_t total = 0, out_total = 0;
  const double lo = std::log(1024.0), hi = std::log(4194304.0);
  for (uint64_t i = 0; total < probe_bytes; i++) {
    const double u = (double)(mix(0x7E57ull + (i + 1) * 0x9E3779B97F4A7C15ull) >> 11) * 0x1p-53;
    size_t n = (size_t)std::floor(std::exp(lo + u * (hi - lo)));
    n = std::min<size_t>(std::max<size_t>(n, 1024), 4194304);
    sizes.push_back(n);
    total += n;
    out_total += ct_len(p, n, LC_PARALLEL);
  }
  const size_t count = sizes.size();
  uint8_t* buf = nullptr;
  const size_t status_off = (total + out_total + 255) & ~(size_t)255;
  LC_CUDA(cudaMalloc(&buf, status_off + count * sizeof(int32_t)));
  uint8_t* in = buf;
  uint8_t* out = buf + total;
  int32_t* stat = reinterpret_cast<int32_t*>(buf + status_off);
  lc_status st = cuda_fail(launch_synth(in, total, 0x7E57ull, 0, s));
  std::vector<std::string> pws(count);
  std::vector<lc_req> reqs(count);
  for (size_t i = 0, a = 0, b = 0; i < count; i++) {
    char tmp[32];
    snprintf(tmp, sizeof tmp, "tune-probe-%08zx", i);
    pws[i] = tmp;
    const size_t c = ct_len(p, sizes[i], LC_PARALLEL);
    reqs[i] = lc_req{reinterpret_cast<const uint8_t*>(pws[i].data()), (uint32_t)pws[i].size(), LC_ENCRYPT,
                     in + a, sizes[i], out + b, c};
    a += sizes[i];
    b += c;
  }

  const lc_launch saved = ctx->launch;
  lc_launch bestl = saved;
  double best_ms = 1e300;
  ctx->tune_report.clear();
  // the probe times the plain throughput variant and adds nothing to the
  // digit or ciphertext statistics being counted
  const bool saved_digits = ctx->digits, saved_ct = ctx->ct_stats;
  ctx->digits = false;
  ctx->ct_stats = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == LC_OK) st = cuda_fail(cudaEventCreate(&e0));
  if (st == LC_OK) st = cuda_fail(cudaEventCreate(&e1));
  for (uint32_t dense = 0; dense <= (v1 ? 1u : 0u) && st == LC_OK; dense++) {
    for (uint32_t tpc : {64u, 128u, 256u}) {
      if (st != LC_OK) break;
      const int v = v1 ? (dense ? kVariantV1Dense : kVariantV1) : ctx->variant;
      const int maxc = resident_ctas(v, (int)tpc);
      std::vector<uint32_t> cands = {0};  // as many as fit
      if (maxc > 1) cands.push_back((uint32_t)(maxc - 1));
      for (uint32_t c : cands) {
        // small_batch_rows = 1: the probe runs the throughput variant
        ctx->launch = lc_launch{tpc, c, 0, 1, saved.host_chunk_mib, dense, saved.full_grid_rows, saved.split_rows};
        invalidate_graphs(ctx);
        st = run_batch_impl(ctx, reqs.data(), count, stat, LC_PARALLEL, s);  // graph build, warm-up
        if (st != LC_OK) break;
        std::vector<double> ms3;
        for (int rep = 0; rep < 3 && st == LC_OK; rep++) {
          st = cuda_fail(cudaEventRecord(e0, s));
          if (st == LC_OK) st = run_batch_impl(ctx, reqs.data(), count, stat, LC_PARALLEL, s);
          if (st == LC_OK) st = cuda_fail(cudaEventRecord(e1, s));
          if (st == LC_OK) st = cuda_fail(cudaEventSynchronize(e1));
          float ms = 0.f;
          if (st == LC_OK) st = cuda_fail(cudaEventElapsedTime(&ms, e0, e1));
          ms3.push_back(ms);
        }
        if (st != LC_OK) break;
        std::sort(ms3.begin(), ms3.end());
        const double med = ms3[1];
        lc_launch rec{tpc, c, 0, saved.small_batch_rows, saved.host_chunk_mib, dense, saved.full_grid_rows,
                      saved.split_rows};
        ctx->tune_report.push_back(lc_tune_entry{rec, med});
        if (med < best_ms) {
          best_ms = med;
          bestl = rec;
        }
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(buf);
  ctx->launch = (st == LC_OK) ? bestl : saved;
  ctx->digits = saved_digits;
  ctx->ct_stats = saved_ct;
  invalidate_graphs(ctx);
  if (best) *best = ctx->launch;
  return st;
}

lc_status lc_tune_report(const lc_ctx* ctx, lc_tune_entry* out, size_t cap, size_t* n) {
  if (!ctx || !n) return LC_ERR_ARG;
  *n = ctx->tune_report.size();
  for (size_t i = 0; i < cap && i < ctx->tune_report.size() && out; i++) out[i] = ctx->tune_report[i];
  return LC_OK;
}

lc_status lc_ctx_timing(lc_ctx* ctx, int enable) {
  if (!ctx) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  lc_status st = drain_timing(ctx);
  ctx->timing = enable != 0;
  ctx->total_ms = 0.0;
  ctx->timed_launches = 0;
  return st;
}

lc_status lc_ctx_kernel_time(lc_ctx* ctx, double* total_ms, uint64_t* launches) {
  if (!ctx) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  lc_status st = drain_timing(ctx);
  if (total_ms) *total_ms = ctx->total_ms;
  if (launches) *launches = ctx->timed_launches;
  return st;
}

uint64_t lc_ctx_launch_count(const lc_ctx* ctx) { return ctx ? ctx->launches : 0; }

uint32_t lc_emu_mask(void) { return emu_mask(); }
uint32_t lc_warm_mask(void) { return warm_mask(); }
uint32_t lc_partial_mask(void) { return partial_mask(); }

lc_status lc_byte_stats(lc_ctx* ctx, const uint8_t* data_dev, size_t n, uint32_t max_lag,
                        lc_byte_stats_t* out, void* stream) {
  if (!ctx || !out || (n && !data_dev) || max_lag > LC_STATS_MAX_LAG) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  constexpr size_t kWords = 258 + LC_STATS_MAX_LAG;
  if (!ctx->stats_dev) LC_CUDA(cudaMalloc(&ctx->stats_dev, kWords * sizeof(unsigned long long)));
  LC_CUDA(launch_stats(data_dev, n, max_lag, ctx->stats_dev, ctx->sm_count, s));
  unsigned long long acc[kWords];
  LC_CUDA(cudaMemcpyAsync(acc, ctx->stats_dev, sizeof acc, cudaMemcpyDeviceToHost, s));
  LC_CUDA(cudaStreamSynchronize(s));
  ctx->launches += 1;
  out->n = n;
  // the sums follow exactly from the histogram: sum b * count, sum b^2 * count
  out->sum = 0;
  out->sum_sq = 0;
  for (int b = 0; b < 256; b++) {
    out->hist[b] = acc[b];
    out->sum += (uint64_t)b * acc[b];
    out->sum_sq += (uint64_t)b * (uint64_t)b * acc[b];
  }
  for (int k = 0; k < LC_STATS_MAX_LAG; k++) out->lag_sum[k] = (uint32_t)k < max_lag ? acc[258 + k] : 0;
  return LC_OK;
}

lc_status lc_ctx_digit_stats(lc_ctx* ctx, int enable) {
  if (!ctx) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  if (enable) {
    const size_t bytes = 3 * kDigBins * sizeof(unsigned long long);
    if (!ctx->digits_dev) {
      LC_CUDA(cudaDeviceSynchronize());
      LC_CUDA(cudaMalloc(&ctx->digits_dev, bytes));
      invalidate_graphs(ctx);  // the counting variants take this pointer
    }
    LC_CUDA(cudaDeviceSynchronize());
    LC_CUDA(cudaMemset(ctx->digits_dev, 0, bytes));
  }
  ctx->digits = enable != 0;
  return LC_OK;
}

lc_status lc_ctx_get_digit_stats(lc_ctx* ctx, lc_digit_stats_t* out) {
  if (!ctx || !out) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  memset(out, 0, sizeof *out);
  if (!ctx->digits_dev) return LC_OK;
  unsigned long long h[3 * kDigBins];
  LC_CUDA(cudaDeviceSynchronize());
  LC_CUDA(cudaMemcpy(h, ctx->digits_dev, sizeof h, cudaMemcpyDeviceToHost));
  for (int c = 0; c < 3; c++) {
    const unsigned long long* hc = h + c * kDigBins;
    for (int b = 0; b < 128; b++) out->int_part[c][b] = hc[b];
    for (int j = 0; j < 3; j++)
      for (int d = 0; d < 100; d++) out->digits[c][j][d] = hc[128 + 100 * j + d];
    out->out_of_range[c] = hc[428];
  }
  for (int b = 0; b < 128; b++) out->states += out->int_part[0][b];
  out->states += out->out_of_range[0];
  return LC_OK;
}

lc_status lc_ctx_ciphertext_stats(lc_ctx* ctx, int enable) {
  if (!ctx) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  if (enable) {
    const size_t bytes = kCtStatsWords * sizeof(unsigned long long);
    if (!ctx->ct_stats_dev) {
      LC_CUDA(cudaDeviceSynchronize());
      LC_CUDA(cudaMalloc(&ctx->ct_stats_dev, bytes));
      invalidate_graphs(ctx);  // the counting variants take this pointer
    }
    LC_CUDA(cudaDeviceSynchronize());
    LC_CUDA(cudaMemset(ctx->ct_stats_dev, 0, bytes));
    ctx->ct_stats_bytes = 0;
  }
  ctx->ct_stats = enable != 0;
  return LC_OK;
}

lc_status lc_ctx_get_ciphertext_stats(lc_ctx* ctx, lc_byte_stats_t* out) {
  if (!ctx || !out) return LC_ERR_ARG;
  DeviceGuard g(ctx->device);
  memset(out, 0, sizeof *out);
  if (!ctx->ct_stats_dev) return LC_OK;
  unsigned long long h[kCtStatsWords];
  LC_CUDA(cudaDeviceSynchronize());
  LC_CUDA(cudaMemcpy(h, ctx->ct_stats_dev, sizeof h, cudaMemcpyDeviceToHost));
  out->n = ctx->ct_stats_bytes;
  for (int b = 0; b < 256; b++) {
    out->hist[b] = h[b];
    out->sum += (uint64_t)b * h[b];
    out->sum_sq += (uint64_t)b * (uint64_t)b * h[b];
  }
  for (int k = 0; k < LC_STATS_MAX_LAG; k++) out->lag_sum[k] = h[256 + k];
  return LC_OK;
}

lc_status lc_key_info(const lc_params* p, const uint8_t* pw, size_t pw_len, lc_key_info_t* out) {
  if (!out) return LC_ERR_ARG;
  lc_params prm;
  if (p) prm = *p; else lc_params_default(&prm);
  if (!params_valid(prm)) return LC_ERR_ARG;
  HostKey k;
  lc_status st = key_schedule(prm, pw, pw_len, &k);
  if (st != LC_OK) return st;
  for (int i = 0; i < 3; i++) {
    out->aprime[i] = k.aprime[i];
    out->mu[i] = k.mu[i];
    out->omega[i] = k.omega[i];
  }
  out->L = k.L;
  out->D = k.D;
  return LC_OK;
}

lc_status lc_plan_batch_ex(const lc_params* p, const lc_req_ex* reqs, size_t count, lc_mode m,
                           int32_t* init_status, uint64_t* nrows) {
  if ((!reqs || !init_status) && count) return LC_ERR_ARG;
  if (m != LC_PARALLEL && m != LC_SEQUENTIAL) return LC_ERR_ARG;
  lc_params prm;
  if (p) prm = *p; else lc_params_default(&prm);
  if (!params_valid(prm)) return LC_ERR_ARG;
  uint64_t rows = 0;
  for (size_t i = 0; i < count; i++) {
    size_t n = 0;
    init_status[i] = validate_req(prm, reqs[i].req, m, &n);
    if (init_status[i] == LC_OK) init_status[i] = validate_key_ex(reqs[i]);
    if (init_status[i] == LC_OK) rows += nblocks_of(prm, n, m);
  }
  if (nrows) *nrows = rows;
  return LC_OK;
}

lc_status lc_plan_batch(const lc_params* p, const lc_req* reqs, size_t count, lc_mode m,
                        int32_t* init_status, uint64_t* nrows) {
  if ((!reqs || !init_status) && count) return LC_ERR_ARG;
  if (m != LC_PARALLEL && m != LC_SEQUENTIAL) return LC_ERR_ARG;
  lc_params prm;
  if (p) prm = *p; else lc_params_default(&prm);
  if (!params_valid(prm)) return LC_ERR_ARG;
  uint64_t rows = 0;
  for (size_t i = 0; i < count; i++) {
    size_t n = 0;
    init_status[i] = validate_req(prm, reqs[i], m, &n);
    if (init_status[i] == LC_OK) rows += nblocks_of(prm, n, m);
  }
  if (nrows) *nrows = rows;
  return LC_OK;
}

lc_status lc_synth_uniform(uint8_t* dst_dev, size_t n, uint64_t seed, uint64_t offset, void* stream) {
  if (n && !dst_dev) return LC_ERR_ARG;
  return cuda_fail(launch_synth(dst_dev, n, seed, offset, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
