// softfp_eval.cu -- lc_softfp_eval: runs each integer-pipe binary64 routine
// of softfp64.cuh next to the hardware instruction on caller-supplied bit
// patterns, so a test can check that the two agree bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lc.h"
#include "softfp64.cuh"

namespace {

__global__ void eval_kernel(uint32_t op, const uint64_t* __restrict__ a, const uint64_t* __restrict__ b,
                            uint64_t* __restrict__ sw, uint64_t* __restrict__ hw, size_t n) {
  namespace S = lc::sfp;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double x = S::from_bits(a[i]);
    const double y = b ? S::from_bits(b[i]) : 0.0;
    uint64_t s = 0, h = 0;
    switch (op) {
      case LC_SFP_ADD: s = S::bits(S::dadd(x, y)); h = S::bits(__dadd_rn(x, y)); break;
      case LC_SFP_SUB: s = S::bits(S::dsub(x, y)); h = S::bits(__dsub_rn(x, y)); break;
      case LC_SFP_MUL: s = S::bits(S::dmul(x, y)); h = S::bits(__dmul_rn(x, y)); break;
      case LC_SFP_MUL10: s = S::bits(S::mul_small<5, 1>(x)); h = S::bits(__dmul_rn(10.0, x)); break;
      case LC_SFP_MUL28: s = S::bits(S::mul_small<7, 2>(x)); h = S::bits(__dmul_rn(28.0, x)); break;
      case LC_SFP_FLOOR13:
        s = S::floor_scaled_lo32(x);
        h = (uint32_t)(uint64_t)__double2ll_rd(__dmul_rn(x, 1e13));
        break;
      case LC_SFP_MULDT:
        s = S::bits(S::dmul_const<0x3F847AE147AE147Bull>(x));
        h = S::bits(__dmul_rn(x, 0.01));
        break;
      case LC_SFP_MULBETA:
        s = S::bits(S::dmul_const<0x4005555555555555ull>(x));
        h = S::bits(__dmul_rn(x, 8.0 / 3.0));
        break;
      case LC_SFP_ADD_KICK: s = S::bits(S::dadd_small<false, true>(x, y)); h = S::bits(__dadd_rn(x, y)); break;
      case LC_SFP_ADD_Z: s = S::bits(S::dadd_small<true, false>(x, y)); h = S::bits(__dadd_rn(x, y)); break;
      default: break;
    }
    sw[i] = s;
    hw[i] = h;
  }
}

}  // namespace

extern "C" lc_status lc_softfp_eval(uint32_t op, const uint64_t* a_dev, const uint64_t* b_dev,
                                    uint64_t* sw_dev, uint64_t* hw_dev, size_t n, void* stream) {
  if (op > LC_SFP_ADD_Z) return LC_ERR_ARG;
  if (n && (!a_dev || !sw_dev || !hw_dev)) return LC_ERR_ARG;
  if (n && !b_dev && (op <= LC_SFP_MUL || op >= LC_SFP_ADD_KICK)) return LC_ERR_ARG;
  if (n == 0) return LC_OK;
  eval_kernel<<<1024, 256, 0, static_cast<cudaStream_t>(stream)>>>(op, a_dev, b_dev, sw_dev, hw_dev, n);
  return cudaGetLastError() == cudaSuccess ? LC_OK : LC_ERR_CUDA;
}
