/*
 * lc.h -- C ABI of liblorenzcipher, a CUDA (sm_103a) implementation of the
 * parallel Lorenz-attractor chaotic cipher of Marco, Martinez & Bruno,
 * "Fast, parallel and secure cryptography algorithm using Lorenz's
 * attractor" (arXiv 1201.3114).
 *
 * The problem statement is that of Sec. 1: a plaintext P of n_p bytes and a
 * password pi give a ciphertext C = E_pi(P), and P = D_pi(C).  Sec. 2 adds
 * that a changed ciphertext is detected (integrity); Sec. 5 splits the
 * message into parts with their own initial conditions (parallel version).
 *
 * Conventions for every call below:
 *   - Buffers named *_dev are device pointers (cudaMalloc / PyTorch CUDA
 *     tensors) on the context's device; *_host are host pointers.  The caller
 *     owns every buffer it passes; the library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; calls documented as "asynchronous"
 *     return before the GPU has finished.
 *   - Passwords are host bytes, 1..32 long (reading of the length limit of
 *     Sec. 3.1); other lengths give LC_ERR_PASSWORD.
 *   - Errors are returned as lc_status, never thrown.  There is no CPU
 *     fallback: without a usable CUDA device every compute call returns
 *     LC_ERR_CUDA.
 *   - One lc_ctx must not be used by two host threads at once.  One thread
 *     may pass different streams to one context: a context's batches share
 *     its workspace, so each waits on the GPU for the context's previous
 *     batch when the stream changes.  Independent streams that should run
 *     concurrently need a context each.
 *   - In-place operation (input == output) is allowed: every byte is read by
 *     the same thread before it is written.  Partly overlapping input and
 *     output ranges give LC_ERR_ARG.
 */
#ifndef LC_H
#define LC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LC_PARAMS_VERSION 1u

typedef enum {
  LC_OK = 0,
  LC_ERR_ARG = 1,       /* null pointer, bad size, overlap, bad params */
  LC_ERR_PASSWORD = 2,  /* password length outside 1..32 */
  LC_ERR_LENGTH = 3,    /* ciphertext length no plaintext length maps to,
                           or an output buffer that is too small */
  LC_ERR_INTEGRITY = 4, /* decryption: a part's tag did not verify */
  LC_ERR_CUDA = 5,      /* CUDA runtime error or no device */
  LC_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up (reserved: no call
                           of this version waits on the device) */
  LC_ERR_NOMEM = 7      /* device workspace could not be allocated */
} lc_status;

typedef enum {
  LC_PARALLEL = 0,  /* Sec. 5: independent parts of block_len bytes */
  LC_SEQUENTIAL = 1 /* Sec. 3: one trajectory over the whole message */
} lc_mode;

typedef enum { LC_ENCRYPT = 0, LC_DECRYPT = 1 } lc_dir;

/* Constants of the method.  Sec. 3.1 fixes sigma, rho, beta, bounds dt and
 * lambda, gives n_it = 3000 and bounds k; the values left open are fixed by
 * lc_params_default() (dt = 0.01, lambda = (1, 1, 20), k = (4, 4, 4),
 * block_len = 4096, tag_len = 8, eta = 2^-24, one Euler step per byte,
 * n_it read as the warm-up length).  Layout mirrors the oracle's. */
typedef struct {
  double sigma, rho, beta; /* Lorenz parameters, Sec. 3.1 */
  double dt;               /* Euler step; Sec. 3.1 bounds it by 0 < dt <= 0.027, the
                              library takes any non-NaN value (0 freezes r) */
  uint32_t n_warm;         /* Euler steps before the first byte */
  uint32_t steps_per_byte; /* applications of F per byte (1..4096) */
  double lambda[3];        /* offset of r_0, Eq. 5 */
  uint32_t k[3];           /* Omega_i in [0, k_i), Eq. 7; 1 <= k_i <= 8 */
  uint32_t block_len;      /* bytes per part (Sec. 5), 16..2^24, multiple of 16 */
  uint32_t tag_len;        /* integrity bytes per part, 1..8 */
  double eta;              /* offset between consecutive parts' r_0 */
  uint32_t omega_alpha_shift; /* Sec. 3.2 Step 3 moves Omega_i with alpha_j,
                                 j = [(i+2) mod 3]+1: 0 reads i as 1-based
                                 (j = i, the default), 1 as 0-based (a
                                 cyclic shift); 1 runs the FP64-pipe kernel */
  uint32_t reserved;       /* must be 0 */
} lc_params;

typedef struct lc_ctx lc_ctx;

/* LC_PARAMS_VERSION of the arithmetic this library implements. */
uint32_t lc_version(void);

/* How this library was built: LC_BUILD_CHECKED is set in the checked build
 * (compiled with -DLC_CHECKED), whose kernels validate every part-table
 * index and part range before use, skip and record any invalid entry, and
 * whose batch calls then wait for the batch and return LC_ERR_CUDA with the
 * entry named in lc_last_cuda_error().  A debugging aid standing in for a
 * memory checker; the paper has no counterpart. */
#define LC_BUILD_CHECKED 1u
uint32_t lc_build_flags(void);

/* Static English text for a status code (never NULL). */
const char* lc_status_string(lc_status s);

/* Text of the last CUDA failure a call of this thread turned into
 * LC_ERR_CUDA / LC_ERR_NOMEM: the CUDA error, the failing call and its
 * place ("" if none).  Valid until the thread's next failing call. */
const char* lc_last_cuda_error(void);

/* The default ("v1") constants described above. */
lc_status lc_params_default(lc_params* out);

/* Create a context on CUDA device `device`.  The context owns its device
 * workspace (tables of parts and keys, verdict flags, the Theta table), a
 * key cache and the captured CUDA graph of the batched path.  *out is NULL
 * on failure.  Errors: LC_ERR_ARG (out NULL), LC_ERR_CUDA (no such device),
 * LC_ERR_NOMEM. */
lc_status lc_ctx_create(int device, lc_ctx** out);

/* Wait for the context's work and release everything it owns. NULL is a no-op. */
void lc_ctx_destroy(lc_ctx* ctx);

/* Replace / read the constants used by later calls (default: v1).
 * LC_ERR_ARG if a field is out of the documented range. */
lc_status lc_ctx_set_params(lc_ctx* ctx, const lc_params* p);
lc_status lc_ctx_get_params(const lc_ctx* ctx, lc_params* p);

/* Ciphertext length for an n-byte message: n + tag_len * nblocks with
 * nblocks = max(1, ceil(n / block_len)) in parallel mode, 1 in sequential
 * mode (the empty message still carries one tag). */
size_t lc_ciphertext_len(const lc_ctx* ctx, size_t n, lc_mode m);

/* Inverse of lc_ciphertext_len; LC_ERR_LENGTH if no n maps to c_len. */
lc_status lc_plaintext_len(const lc_ctx* ctx, size_t c_len, lc_mode m, size_t* n);

/* Sec. 3.2 Steps 1-3 over every part of P (Sec. 5), C = E_pi(P).
 * P_dev: n bytes (may be NULL when n == 0).  C_dev: c_cap >=
 * lc_ciphertext_len(n, m) bytes; bytes [0, n) hold the coded message at the
 * plaintext's offsets and the tags follow.  Asynchronous on `stream`.
 * Errors: LC_ERR_ARG, LC_ERR_PASSWORD, LC_ERR_LENGTH (c_cap too small),
 * LC_ERR_CUDA, LC_ERR_NOMEM. */
lc_status lc_encrypt(lc_ctx* ctx, const uint8_t* pw, size_t pw_len,
                     const uint8_t* P_dev, size_t n, uint8_t* C_dev, size_t c_cap,
                     lc_mode m, void* stream);

/* P = D_pi(C) and the integrity verdict of Sec. 2.  C_dev holds c_len bytes;
 * P_dev receives n bytes (p_cap >= n).  Synchronises `stream`.  Returns
 * LC_ERR_INTEGRITY if any part's tag failed, and then P is all zeros
 * (fail-closed).  Other errors as lc_encrypt, LC_ERR_LENGTH for a c_len no
 * plaintext length maps to. */
lc_status lc_decrypt(lc_ctx* ctx, const uint8_t* pw, size_t pw_len,
                     const uint8_t* C_dev, size_t c_len, uint8_t* P_dev, size_t p_cap,
                     lc_mode m, void* stream);

/* One request of a batch.  dir = LC_ENCRYPT: `in` holds in_len plaintext
 * bytes and `out` receives lc_ciphertext_len(in_len) bytes.  dir =
 * LC_DECRYPT: `in` holds an in_len-byte ciphertext and `out` receives the
 * plaintext.  out_cap is the capacity of `out`. */
typedef struct {
  const uint8_t* pw;
  uint32_t pw_len;
  uint32_t dir;
  const uint8_t* in;
  size_t in_len;
  uint8_t* out;
  size_t out_cap;
} lc_req;

/* Batched path: every part of every request runs in one persistent kernel
 * over a flattened table of parts, replayed from a CUDA graph.  Requests are
 * independent and may mix directions and passwords; `in`/`out` are device
 * pointers.  status_dev (device, `count` int32) receives each request's
 * lc_status: LC_OK, LC_ERR_INTEGRITY (its output then zeroed), or the host
 * validation error of that request (LC_ERR_PASSWORD / LC_ERR_LENGTH /
 * LC_ERR_ARG; nothing is computed for it).  Asynchronous on `stream`.  The
 * call itself fails (LC_ERR_ARG) only for a NULL ctx/reqs/status_dev or an
 * unusable stream, LC_ERR_NOMEM / LC_ERR_CUDA for workspace or launch
 * failures.  The request array and the passwords may be reused as soon as
 * the call returns; the device buffers must stay valid until the stream
 * reaches this point. */
lc_status lc_run_batch(lc_ctx* ctx, const lc_req* reqs, size_t count, int32_t* status_dev,
                       lc_mode m, void* stream);

/* Key material beyond the password (Sec. 3.1): lambda, the offset of the
 * starting point r_0 = a' + lambda (Eq. 5), and k, the range of Omega_i
 * (Eq. 7).  The paper leaves both to be chosen within stated ranges, so they
 * belong to the secret like the password.  A request of lc_run_batch_ex
 * carries them when key_flags has LC_KEY_LAMBDA / LC_KEY_K; otherwise the
 * context's parameters apply.  Valid values are those of Sec. 3.1:
 * -15.67 < lambda_1 < 16.01, -11.28 < lambda_2 < 16.01,
 * 0.090 < lambda_3 < 62.000, and 2 < k_i <= floor((52 - 14) / 8) = 4;
 * anything else gives the request LC_ERR_ARG. */
#define LC_KEY_LAMBDA 1u
#define LC_KEY_K 2u
typedef struct {
  lc_req req;
  uint32_t key_flags; /* LC_KEY_LAMBDA | LC_KEY_K */
  uint32_t k[3];
  double lambda[3];
} lc_req_ex;

/* lc_run_batch with per-request key material: the same call, results and
 * errors, for lc_req_ex requests.  Requests of one batch may mix lambda and
 * k values.  A batch in which some request's k is not (4, 4, 4) runs, with
 * the context's v1 constants and at least the small-batch threshold of
 * parts (lc_launch.small_batch_rows), the v1 build that reads k per message;
 * otherwise the kernel variant that keeps all binary64 work on the FP64
 * pipe. */
lc_status lc_run_batch_ex(lc_ctx* ctx, const lc_req_ex* reqs, size_t count, int32_t* status_dev,
                          lc_mode m, void* stream);

/* lc_run_batch with HOST buffers: `in` / `out` are host pointers (pinned
 * memory gives the best copy rate) and status_host is host memory.  The
 * library copies the inputs to its own device staging area (one copy per
 * run of requests whose host buffers are contiguous), runs the batch and
 * copies the outputs and statuses back; returns after the stream has
 * synchronised.  The call's return value is LC_OK unless the call itself
 * failed; per-request results are in status_host. */
lc_status lc_run_batch_host(lc_ctx* ctx, const lc_req* reqs, size_t count,
                            int32_t* status_host, lc_mode m, void* stream);

/* Host-buffer batches a context can hold in flight (one device staging area
 * each). */
#define LC_HOST_INFLIGHT 3u

/* lc_run_batch_host without the wait, so that consecutive batches overlap:
 * batch k+1's input copies run while batch k computes, and batch k's output
 * copies while batch k+1 computes.  The paper has no counterpart; this is a
 * pipelining aid of the library.
 *
 * The call validates and plans the batch, enqueues the input copies (on a
 * copy stream of the context), the batch (on `stream`) and the output and
 * status copies (on a second copy stream of the context), and returns with
 * *ticket set to a number > 0 that increases per context.  Buffers: the
 * request array and the passwords may be reused when the call returns; the
 * host inputs must stay unchanged, and the host outputs and status_host
 * hold undefined bytes, until lc_wait_batch_host returns for this ticket or
 * a later one.  The inputs are read after the call returns, with no
 * ordering against earlier work on `stream`: host buffers filled by
 * asynchronous copies must be complete before the call.  Pinned host
 * buffers keep every copy asynchronous; with pageable output buffers the
 * call waits for the batch.  With LC_HOST_INFLIGHT batches already in
 * flight, the call first waits for the oldest (which completes its ticket).
 * count == 0 gives a ticket that is already complete.  Errors: LC_ERR_ARG
 * (NULL ctx or ticket, NULL reqs or status_host with count > 0, a bad
 * mode), otherwise as lc_run_batch_host; after an error nothing of this
 * batch is in flight and *ticket must not be waited for. */
lc_status lc_submit_batch_host(lc_ctx* ctx, const lc_req* reqs, size_t count,
                               int32_t* status_host, lc_mode m, void* stream, uint64_t* ticket);

/* Wait until the batch of `ticket`, and every batch submitted before it, has
 * finished and its outputs and statuses are in host memory.  LC_OK if they
 * already were; LC_ERR_ARG for ticket 0 or a ticket not yet issued;
 * LC_ERR_CUDA if a copy or kernel of those batches failed. */
lc_status lc_wait_batch_host(lc_ctx* ctx, uint64_t ticket);

/* Launch shape of the batched kernel: threads per CTA (32..256, multiple of
 * 32), resident CTAs per SM for the persistent grid (0 = as many as fit),
 * smem_staging (reserved, must be 0), and small_batch_rows: with the
 * default constants, a batch of fewer parts than this runs the kernel
 * variant that keeps all binary64 work on the FP64 pipe (lower latency
 * while the GPU is far from full); larger batches run the variant that
 * moves the multiplies to the integer pipes (higher throughput).  0 = auto
 * (192 parts per SM).  host_chunk_mib: a host-buffer batch whose inputs
 * exceed this many MiB is cut into up to 4 chunks of whole requests, so
 * that one chunk's copies overlap another's kernel (0 = 4096 MiB).
 * dense_build: 1 = the throughput variant's builds compiled for 4 resident
 * 256-thread CTAs per SM (at most 64 registers per thread) instead of the
 * default builds for 3 (0).  full_grid_rows: a throughput-variant batch of
 * at least this many parts fills the persistent grid and runs the build
 * that also moves the kick of Step 2 to the integer pipes (lc_emu_mask);
 * a smaller batch, whose grid is cut to fewer CTAs per SM, runs the build
 * that keeps it on the FP64 pipe (lc_partial_mask), whose shorter
 * dependency chains suit fewer resident warps (0 = auto: the threads of
 * the full persistent grid).  split_rows: a batch of the FP64-pipe variant
 * with fewer parts than this runs its split build, in which each part's
 * three coordinates are computed by three warps of a 96-thread CTA that
 * exchange them through shared memory every Euler step (a warp issues at
 * most one binary64 instruction per 64 cycles, so this shortens one part's
 * latency while the GPU is far from full; 0 = auto: 64 parts per SM with
 * one Euler step per byte, never with more).  None of these changes
 * results. */
typedef struct {
  uint32_t threads_per_cta;
  uint32_t ctas_per_sm;
  uint32_t smem_staging;
  uint32_t small_batch_rows;
  uint32_t host_chunk_mib;
  uint32_t dense_build;
  uint32_t full_grid_rows;
  uint32_t split_rows;
} lc_launch;

lc_status lc_ctx_get_launch(const lc_ctx* ctx, lc_launch* out);
lc_status lc_ctx_set_launch(lc_ctx* ctx, const lc_launch* l);

/* Autotuner: times candidate launch shapes of the throughput variant on a
 * synthetic batch and keeps the fastest in the context; *best (may be NULL)
 * receives it.  The probe batch has the shape of a batched workload:
 * messages of log-uniform sizes between 1 KiB and 4 MiB (seeded, device-
 * generated bytes, distinct passwords, all encrypted in parallel mode)
 * totalling `probe_bytes` (0 = enough parts to fill the largest candidate
 * persistent grid four times; pass the size of a typical batch to tune for
 * it).  Candidates: threads per CTA in {64, 128, 256},
 * all resident CTAs per SM or one fewer, each with the default and the
 * dense build (lc_launch.dense_build); each candidate runs once untimed and
 * three times timed with CUDA events on `stream`, and the median counts.
 * The other lc_launch fields keep their values.  Synchronises `stream`;
 * allocates the probe's buffers for the duration of the call.  Never
 * changes results. */
lc_status lc_tune(lc_ctx* ctx, size_t probe_bytes, void* stream, lc_launch* best);

/* Timings of the last lc_tune call on this context: up to `cap` candidates
 * (launch shape and median milliseconds) in the order tried; *n receives how
 * many there were.  LC_ERR_ARG for a NULL ctx or n. */
typedef struct {
  lc_launch launch;
  double median_ms;
} lc_tune_entry;
lc_status lc_tune_report(const lc_ctx* ctx, lc_tune_entry* out, size_t cap, size_t* n);

/* Accumulated device time of the context's main cipher kernel since the
 * last reset, measured with CUDA events on the launching stream (enabled by
 * lc_ctx_timing(ctx, 1); reading synchronises those events). */
lc_status lc_ctx_timing(lc_ctx* ctx, int enable);
lc_status lc_ctx_kernel_time(lc_ctx* ctx, double* total_ms, uint64_t* launches);

/* Number of kernels the library has launched through this context. */
uint64_t lc_ctx_launch_count(const lc_ctx* ctx);

/* Host-only inspection of the key schedule of Sec. 3.1 (Eqs. 2-7): a' = g(a),
 * the initial mu and Omega for password pw under parameters p (NULL =
 * defaults).  Needs no GPU.  LC_ERR_PASSWORD for a length outside 1..32,
 * LC_ERR_ARG for a NULL out or invalid p. */
typedef struct {
  double aprime[3];
  uint32_t mu[3];
  uint32_t omega[3];
  uint32_t L, D;
} lc_key_info_t;
lc_status lc_key_info(const lc_params* p, const uint8_t* pw, size_t pw_len, lc_key_info_t* out);

/* Host-only validation of a batch, exactly as lc_run_batch performs it:
 * init_status (host, `count` int32) receives LC_OK or the request's
 * validation error, *nrows the number of trajectories (parts) the valid
 * requests need.  Needs no GPU. */
lc_status lc_plan_batch(const lc_params* p, const lc_req* reqs, size_t count, lc_mode m,
                        int32_t* init_status, uint64_t* nrows);
/* The same for lc_req_ex requests (their key material is checked too). */
lc_status lc_plan_batch_ex(const lc_params* p, const lc_req_ex* reqs, size_t count, lc_mode m,
                           int32_t* init_status, uint64_t* nrows);

/* Measured issue rates (results per second / 1e9) of the SM pipes the cipher
 * uses, from throughput microbenchmarks on `device` (not part of the paper's
 * method; the roofline denominators of the FP64-bound kernel).  ialu counts
 * 32-bit integer add/logic results, imad 32-bit integer multiply-adds, ffma
 * fp32 fused multiply-adds.  Synchronises the device. */
typedef struct {
  double dadd_gops, dmul_gops, cvt_gops;
  double imad_gops, ialu_gops, ffma_gops;
  double sm_clock_mhz;
  uint32_t sm_count, reserved;
} lc_pipe_rates;
lc_status lc_probe_pipes(int device, lc_pipe_rates* out);

/* Issue interval of binary64 adds for few warps (not part of the paper's
 * method; it explains the latency of one trajectory): one CTA of `warps`
 * warps (1..32) on `device`, the first `lanes` lanes (1..32) of each warp
 * running `chains` (1, 2, 4 or 8) independent chains of dependent DADDs.
 * *cycles receives the SM clock cycles per DADD warp instruction of the
 * slowest warp.  Synchronises the device. */
lc_status lc_probe_fp64_warp(int device, uint32_t warps, uint32_t chains, uint32_t lanes,
                             double* cycles);

/* Allocation-free batched path.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they
 * encrypt or decrypt -- for example code whose device memory is entirely
 * owned by another allocator or memory pool (a cudaMalloc would fail or
 * fragment that pool), code running inside an allocator's own callback or
 * while holding its lock (a nested allocation would recurse or deadlock),
 * and latency-critical threads that must not hit the device-wide
 * synchronisation that cudaMalloc / cudaFree can imply.
 *
 * It runs the same persistent cipher kernel as lc_run_batch, with requests
 * and results as there (device buffers, per-request status in status_dev),
 * but without an lc_ctx and always with the default (v1) parameters.  All
 * scratch memory the kernel needs beyond the caller's buffers -- the part
 * table, the row counter, the per-request verdict flags and the Theta
 * table -- sits in one fixed 2 MiB static device array inside the library,
 * which every GPU that loads the library holds until the process exits.  No
 * call allocates (no cudaMalloc, cudaFree, pinned host memory, graph or
 * host heap).
 *
 * Limits: at most LC_NOALLOC_MAX_REQUESTS requests and LC_NOALLOC_MAX_PARTS
 * parts (4096-byte parts in parallel mode, one per message in sequential
 * mode; about 983 MB of parallel-mode data) per call; larger batches are
 * rejected with LC_ERR_LENGTH before any GPU work.
 *
 * The first call on a device sets that device up (looks up the array's
 * device address and copies the Theta table into it, synchronously).  Every
 * call uses the same array and leaves its contents behind; each call clears
 * the counter and flags it needs.  Calls whose GPU work overlaps (for
 * example on two streams without ordering between them) race on the array:
 * issue them on one stream, or synchronise between them.  The part table is
 * copied to the device from static pageable host memory, so the call may
 * wait on the host until earlier work on `stream` has drained; the call
 * must not be captured into a CUDA graph, and a capturing `stream` gives
 * LC_ERR_ARG.  Otherwise asynchronous on `stream`; uses the current device.
 * Errors: LC_ERR_ARG, LC_ERR_LENGTH, LC_ERR_CUDA. */
#define LC_NOALLOC_MAX_REQUESTS 1024u
#define LC_NOALLOC_MAX_PARTS 240000u
lc_status lc_run_batch_noalloc(const lc_req* reqs, size_t count, int32_t* status_dev, lc_mode m,
                               void* stream);

/* Exactness check of the integer-pipe binary64 routines (not part of the
 * paper's method).  GB300 issues binary64 add/multiply at about 1/38 of its
 * 32-bit integer rate, so the v1 kernel computes part of its binary64 work
 * with integer instructions that reproduce IEEE-754 round-to-nearest-even
 * bit for bit.  This call evaluates routine `op` on n operand bit patterns
 * (a_dev, and b_dev for the two-operand routines) and writes the routine's
 * result bits to sw_dev and the hardware instruction's to hw_dev (device
 * arrays of n uint64).  LC_SFP_FLOOR13 gives the low 32 bits of
 * floor(RN(a * 10^13)) as cvt.rmi.s64.f64 computes it.  Asynchronous. */
enum {
  LC_SFP_ADD = 0,     /* a + b */
  LC_SFP_SUB = 1,     /* a - b */
  LC_SFP_MUL = 2,     /* a * b */
  LC_SFP_MUL10 = 3,   /* 10 * a */
  LC_SFP_MUL28 = 4,   /* 28 * a */
  LC_SFP_FLOOR13 = 5, /* low 32 bits of floor(RN(a * 10^13)) */
  LC_SFP_MULDT = 6,   /* 0.01 * a (the compile-time constant multiply) */
  LC_SFP_MULBETA = 7, /* RN(8/3) * a (the same) */
  LC_SFP_ADD_KICK = 8, /* a + b by the known-order adder for a larger than
                          b >= 0 (the kick of Step 2) */
  LC_SFP_ADD_Z = 9     /* a + b by the known-order adder for a > 0 larger than
                          b (the Euler step's z update) */
};
lc_status lc_softfp_eval(uint32_t op, const uint64_t* a_dev, const uint64_t* b_dev, uint64_t* sw_dev,
                         uint64_t* hw_dev, size_t n, void* stream);

/* The binary64 operations the v1 kernel computes on the integer pipe, as
 * bit masks fixed at build time (diagnostic): lc_emu_mask for the byte
 * steps of full-grid batches, lc_partial_mask for those of smaller batches
 * of the throughput variant, lc_warm_mask for the Euler steps of the
 * warm-up. */
uint32_t lc_emu_mask(void);
uint32_t lc_partial_mask(void);
uint32_t lc_warm_mask(void);

/* Byte statistics of a device buffer, for the ciphertext analysis of
 * Sec. 4: the frequency histogram (Fig. 2; the Shannon entropy
 * S = -sum p_i log2 p_i follows from it) and the sums behind the
 * auto-correlation of Fig. 3, all exact integers: sum x_i, sum x_i^2 and,
 * for k = 1..max_lag (max_lag <= LC_STATS_MAX_LAG), sum_{i < n-k} x_i x_{i+k}.
 * Uses the context's workspace; synchronises `stream`. */
#define LC_STATS_MAX_LAG 8
typedef struct {
  uint64_t n;
  uint64_t hist[256];
  uint64_t sum, sum_sq;
  uint64_t lag_sum[LC_STATS_MAX_LAG];
} lc_byte_stats_t;
lc_status lc_byte_stats(lc_ctx* ctx, const uint8_t* data_dev, size_t n, uint32_t max_lag,
                        lc_byte_stats_t* out, void* stream);

/* Digit statistics of the trajectory coordinates, Fig. 1 (Sec. 3.1): after
 * the Euler step(s) of every byte step (body and tag bytes, both
 * directions) of every trajectory a batch runs, each coordinate v of r is
 * counted by its sign-magnitude decimal expansion:
 *   int_part[c][trunc(v) + 64]   (trunc toward zero, clamped to 0..127),
 *   digits[c][j][floor(RN(|v| 10^(2j+2))) mod 100]   for the decimal digit
 *                                pairs 1-2 (j = 0), 3-4 (j = 1), 5-6 (j = 2),
 * or, when |v| >= 2^31 or v is NaN, in out_of_range[c] only; c = 0, 1, 2 for
 * x, y, z.  states = the byte steps counted.
 *
 * lc_ctx_digit_stats(ctx, 1) zeroes the counters and makes the context's
 * later batches count (they then run a counting build of the FP64-pipe or
 * v1 kernel, with identical outputs); 0 stops counting.  Synchronises the
 * device.  lc_ctx_get_digit_stats synchronises the device and reads the
 * counts accumulated since the last enable (all zero if never enabled). */
typedef struct {
  uint64_t states;
  uint64_t int_part[3][128];
  uint64_t digits[3][3][100];
  uint64_t out_of_range[3];
} lc_digit_stats_t;
lc_status lc_ctx_digit_stats(lc_ctx* ctx, int enable);
lc_status lc_ctx_get_digit_stats(lc_ctx* ctx, lc_digit_stats_t* out);

/* Byte statistics of every ciphertext the context writes, fused into the
 * cipher kernel (Sec. 4: the histogram of Fig. 2 and the lagged products
 * behind the auto-correlation of Fig. 3), so that no second pass reads the
 * ciphertexts.  lc_ctx_ciphertext_stats(ctx, 1) zeroes the accumulators and
 * makes the context's later encryptions (lc_encrypt, lc_run_batch,
 * lc_run_batch_ex and the host-buffer batches; decryptions are not counted)
 * run a counting build of the cipher kernel with identical outputs, 256
 * threads per CTA; 0 stops counting.  Synchronises the device.
 * lc_ctx_get_ciphertext_stats synchronises the device and returns the sum,
 * over those ciphertexts C, of what lc_byte_stats(C, |C|, LC_STATS_MAX_LAG)
 * gives: n = the ciphertext bytes, the histogram, sum, sum_sq, and lag_sum[k]
 * = the sum of x_i x_{i+k+1} over pairs inside one ciphertext.  All zero if
 * never enabled.  While counting, a batch whose encryptions write 2^32 or
 * more ciphertext bytes gives LC_ERR_ARG (the kernel's per-CTA counters are
 * 32-bit). */
lc_status lc_ctx_ciphertext_stats(lc_ctx* ctx, int enable);
lc_status lc_ctx_get_ciphertext_stats(lc_ctx* ctx, lc_byte_stats_t* out);

/* Seeded input generator (not part of the paper's method): writes bytes
 * [offset, offset + n) of the counter-based SplitMix64 byte stream `seed`
 * (Steele, Lea & Flood 2014; byte j = byte j mod 8, little-endian, of word
 * j / 8, word i = mix(seed + (i + 1) * 0x9E3779B97F4A7C15)) to dst_dev.
 * Asynchronous on `stream`. */
lc_status lc_synth_uniform(uint8_t* dst_dev, size_t n, uint64_t seed, uint64_t offset,
                           void* stream);

#ifdef __cplusplus
}
#endif
#endif
