// probe.cu -- issue-rate microbenchmarks of the SM pipes the cipher uses:
// binary64 add and multiply, binary64 -> int64 floor conversion, 32-bit
// integer multiply-add and logic/add, and fp32 fused multiply-add.  They
// give the measured denominators of the roofline (the cipher's hot loop is
// bound by the FP64 issue rate, which GB300 provides at a small fraction of
// its fp32 rate).
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lc.h"

namespace {

constexpr int kChains = 8;

__global__ void probe_dadd(double* out, int iters, double c) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) a[j] = threadIdx.x * 1e-3 + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = __dadd_rn(a[j], c);
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < kChains; j++) s += a[j];
  if (s == 12345.678) out[0] = s;
}

__global__ void probe_dmul(double* out, int iters, double c) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) a[j] = 1.0 + threadIdx.x * 1e-6 + j * 1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = __dmul_rn(a[j], c);
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < kChains; j++) s += a[j];
  if (s == 12345.678) out[0] = s;
}

// One cvt.rmi.s64.f64 per link; the OR only re-biases the exponent so the
// next input is again a normal number (one integer op on the high word).
__global__ void probe_cvt(double* out, int iters) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) a[j] = 1.5 + threadIdx.x + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < kChains; j++) {
      long long v = __double2ll_rd(a[j]);
      a[j] = __longlong_as_double(v | 0x4330000000000000ll);
    }
  }
  double s = 0;
#pragma unroll
  for (int j = 0; j < kChains; j++) s += a[j];
  if (s == 12345.678) out[0] = s;
}

__global__ void probe_imad(uint32_t* out, int iters, uint32_t m, uint32_t c) {
  uint32_t a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) a[j] = threadIdx.x + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = a[j] * m + c;
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kChains; j++) s ^= a[j];
  if (s == 0x12345678u) out[0] = s;
}

// Two integer ops per link: an add and an xor with a shifted copy folded by
// the compiler into IADD3 / LOP3 / SHF forms.
__global__ void probe_ialu(uint32_t* out, int iters, uint32_t c) {
  uint32_t a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) a[j] = threadIdx.x * 7u + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = (a[j] + c) ^ (a[j] >> 7);
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < kChains; j++) s ^= a[j];
  if (s == 0x12345678u) out[0] = s;
}

__global__ void probe_ffma(float* out, int iters, float m, float c) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; j++) a[j] = threadIdx.x * 1e-3f + j;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < kChains; j++) a[j] = __fmaf_rn(a[j], m, c);
  }
  float s = 0;
#pragma unroll
  for (int j = 0; j < kChains; j++) s += a[j];
  if (s == 12345.678f) out[0] = s;
}

template <typename F>
double time_ms(F launch, cudaStream_t s) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  launch();  // warm-up
  cudaEventRecord(a, s);
  launch();
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

// One CTA of `warps` warps; in each warp the first `lanes` lanes run K
// independent chains of n dependent DADDs.  Each warp records its cycle
// count (clock64) for the loop.
template <int K>
__global__ void probe_fp64_warp(double* out, long long* cyc, int n, int lanes, double c) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double a[K];
#pragma unroll
  for (int k = 0; k < K; k++) a[k] = threadIdx.x * 1e-3 + k;
  __syncthreads();
  const long long t0 = clock64();
  if (lane < lanes) {
    for (int i = 0; i < n; i++) {
#pragma unroll
      for (int k = 0; k < K; k++) a[k] = __dadd_rn(a[k], c);
    }
  }
  const long long t1 = clock64();
  double s = 0;
#pragma unroll
  for (int k = 0; k < K; k++) s += a[k];
  if (s == 12345.678) out[0] = s;
  if (lane == 0) cyc[warp] = t1 - t0;
}

}  // namespace

extern "C" lc_status lc_probe_fp64_warp(int device, uint32_t warps, uint32_t chains, uint32_t lanes,
                                        double* cycles) {
  if (!cycles || warps < 1 || warps > 32 || lanes < 1 || lanes > 32 ||
      (chains != 1 && chains != 2 && chains != 4 && chains != 8))
    return LC_ERR_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return LC_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return LC_ERR_CUDA;
  void* buf = nullptr;
  if (cudaMalloc(&buf, 64 + 32 * sizeof(long long)) != cudaSuccess) {
    cudaSetDevice(prev);
    return LC_ERR_CUDA;
  }
  double* d = static_cast<double*>(buf);
  long long* cyc = reinterpret_cast<long long*>(static_cast<char*>(buf) + 64);
  const int n = 20000, threads = 32 * (int)warps;
  for (int rep = 0; rep < 2; rep++) {  // the first run warms up
    switch (chains) {
      case 1: probe_fp64_warp<1><<<1, threads>>>(d, cyc, n, (int)lanes, 1e-9); break;
      case 2: probe_fp64_warp<2><<<1, threads>>>(d, cyc, n, (int)lanes, 1e-9); break;
      case 4: probe_fp64_warp<4><<<1, threads>>>(d, cyc, n, (int)lanes, 1e-9); break;
      default: probe_fp64_warp<8><<<1, threads>>>(d, cyc, n, (int)lanes, 1e-9); break;
    }
  }
  long long h[32];
  cudaError_t e = cudaMemcpy(h, cyc, warps * sizeof(long long), cudaMemcpyDeviceToHost);
  cudaFree(buf);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return LC_ERR_CUDA;
  long long mx = 0;
  for (uint32_t w = 0; w < warps; w++) mx = h[w] > mx ? h[w] : mx;
  *cycles = (double)mx / ((double)n * chains);
  return LC_OK;
}

extern "C" lc_status lc_probe_pipes(int device, lc_pipe_rates* out) {
  if (!out) return LC_ERR_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return LC_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return LC_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  void* buf = nullptr;
  if (cudaMalloc(&buf, 64) != cudaSuccess) {
    cudaSetDevice(prev);
    return LC_ERR_CUDA;
  }
  cudaStream_t s = 0;
  const int threads = 256, blocks = sms * 8;
  const double links = (double)blocks * threads * kChains;
  const int it_fp64 = 2000, it_fast = 20000;
  double* d = static_cast<double*>(buf);
  uint32_t* u = static_cast<uint32_t*>(buf);
  float* f = static_cast<float*>(buf);
  double ms;
  ms = time_ms([&] { probe_dadd<<<blocks, threads, 0, s>>>(d, it_fp64, 1e-9); }, s);
  out->dadd_gops = links * it_fp64 / (ms * 1e6);
  ms = time_ms([&] { probe_dmul<<<blocks, threads, 0, s>>>(d, it_fp64, 0.9999999999); }, s);
  out->dmul_gops = links * it_fp64 / (ms * 1e6);
  ms = time_ms([&] { probe_cvt<<<blocks, threads, 0, s>>>(d, it_fp64); }, s);
  out->cvt_gops = links * it_fp64 / (ms * 1e6);
  ms = time_ms([&] { probe_imad<<<blocks, threads, 0, s>>>(u, it_fast, 1664525u, 1013904223u); }, s);
  out->imad_gops = links * it_fast / (ms * 1e6);
  ms = time_ms([&] { probe_ialu<<<blocks, threads, 0, s>>>(u, it_fast, 0x9E3779B9u); }, s);
  out->ialu_gops = 2.0 * links * it_fast / (ms * 1e6);
  ms = time_ms([&] { probe_ffma<<<blocks, threads, 0, s>>>(f, it_fast, 0.999f, 1e-3f); }, s);
  out->ffma_gops = links * it_fast / (ms * 1e6);
  out->sm_count = (uint32_t)sms;
  int clk_khz = 0;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, device);
  out->sm_clock_mhz = clk_khz / 1000.0;
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(buf);
  cudaSetDevice(prev);
  return e == cudaSuccess ? LC_OK : LC_ERR_CUDA;
}
