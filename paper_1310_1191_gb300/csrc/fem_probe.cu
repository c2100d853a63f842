// Throughput probe of the FP64 and FP32 FMA pipes: the denominators of the
// rooflines of the CUDA-core kernels are measured with it rather than taken
// from unit counts and clocks.  Every thread runs kChains independent
// multiply-add chains a <- a * x + y (x slightly below 1, so the values stay
// bounded and normal), kChains * iters multiply-adds per thread in all.
#include <cuda_runtime.h>

#include <string>

#include "fem_internal.h"

namespace fem {

constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, T x, T y, T *out, int64_t *clk) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t c0 = 0, t0 = 0;
  if (clk && threadIdx.x == 0) {
    c0 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = (T)(1 + (tid + k) % 7) * (T)0.125;
  for (int64_t i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = fma(a[k], x, y);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  out[tid] = s;
  if (clk && threadIdx.x == 0) {  // this CTA's SM clock cycles and nanoseconds
    int64_t t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    clk[2 * blockIdx.x] = clock64() - c0;
    clk[2 * blockIdx.x + 1] = t1 - t0;
  }
}

}  // namespace fem

using namespace fem;

extern "C" int fem_probe_fma(int fp64, int64_t iters, int64_t n_threads, void *out, int64_t *clk, void *stream) {
  if (iters < 1 || n_threads < 256 || n_threads % 256 != 0 || n_threads / 256 > 0x7fffffffLL || !out ||
      ((uintptr_t)out & 7) || ((uintptr_t)clk & 7)) {
    set_error("fem_probe_fma: iters >= 1, n_threads a positive multiple of 256 and 8-byte aligned out, clk");
    return FEM_EINVAL;
  }
  const unsigned grid = (unsigned)(n_threads / 256);
  cudaStream_t s = (cudaStream_t)stream;
  if (fp64)
    fma_probe_kernel<double><<<grid, 256, 0, s>>>(iters, 0.99999, 1e-5, static_cast<double *>(out), clk);
  else
    fma_probe_kernel<float><<<grid, 256, 0, s>>>(iters, 0.99999f, 1e-5f, static_cast<float *>(out), clk);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("fem_probe_fma: ") + cudaGetErrorString(e));
    return FEM_ECUDA;
  }
  return FEM_OK;
}
