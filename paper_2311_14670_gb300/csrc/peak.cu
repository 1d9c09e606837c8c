// Measured arithmetic peaks of the float64 and float32 FMA pipes (s2gb_fma_chain).
//
// Every thread runs kChains independent FMA chains x <- x * a + b for `iters` steps and writes the
// sum of its chains, so that nothing can be folded away.  With a = 1 - 2^-20 and b = 2^-30 the
// chains converge to b / (1 - a) = 2^-10 and never overflow or go subnormal.  The caller times the
// launch with CUDA events: the launch performs blocks * threads * kChains * iters FMAs.
#include <cuda_runtime.h>

#include "s2gb_internal.h"

namespace s2gb {
namespace {

constexpr int kChains = 8;

template <typename F>
__global__ void __launch_bounds__(256) fma_chain_kernel(F* __restrict__ out, long long iters, F a, F b) {
  F x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (F)(threadIdx.x + c);
  for (long long k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  F s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace s2gb

extern "C" int s2gb_fma_chain(int precision, int blocks, int threads, long long iters, void* out,
                              void* stream) {
  if (blocks < 1 || threads < 32 || threads > 256 || (threads & 31) || iters < 1 || !out)
    return S2GB_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (precision == S2GB_FP64) {
    s2gb::fma_chain_kernel<double><<<blocks, threads, 0, st>>>(
        reinterpret_cast<double*>(out), iters, 1.0 - 0x1p-20, 0x1p-30);
  } else if (precision == S2GB_FP32) {
    s2gb::fma_chain_kernel<float><<<blocks, threads, 0, st>>>(
        reinterpret_cast<float*>(out), iters, 1.0f - 0x1p-20f, 0x1p-30f);
  } else {
    return S2GB_EINVAL;
  }
  return s2gb::launched() == cudaSuccess ? S2GB_OK : S2GB_ECUDA;
}

extern "C" int s2gb_fma_chain_lanes(void) { return s2gb::kChains; }
