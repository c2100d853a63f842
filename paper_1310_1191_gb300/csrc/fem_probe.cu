// Throughput probe of the FP64 and FP32 FMA pipes: the denominators of the
// rooflines of the CUDA-core kernels are measured with it rather than taken
// from unit counts and clocks.  The loop is the contraction kernels' inner
// loop: each thread keeps a TM x TN register tile of accumulators and, per
// step, loads a TM-vector and a TN-vector from shared memory and adds their
// outer product (TM TN multiply-adds).  A plain chain a <- a x + y per
// register reaches only about 85 % of the FP64 pipe on this GPU; the
// outer-product loop, like the contraction, reaches it.
#include <cuda_runtime.h>

#include <string>

#include "fem_fma.cuh"
#include "fem_internal.h"

namespace fem {

template <class T> struct ProbeTile;
template <> struct ProbeTile<double> { static constexpr int TM = 4, TN = 4; };
template <> struct ProbeTile<float> { static constexpr int TM = 8, TN = 8; };

// every access stays in bounds: shared indexes < 32 TM and 32 TN, out[tid]
// with tid < gridDim.x * 256 = n_threads, clk[2 blockIdx.x + 1] < 2 gridDim.x
template <class T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, T *out, int64_t *clk) {
  constexpr int TM = ProbeTile<T>::TM, TN = ProbeTile<T>::TN;
  __shared__ __align__(16) T sa[32 * TM];
  __shared__ __align__(16) T sb[32 * TN];
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t c0 = 0, t0 = 0;
  if (clk && threadIdx.x == 0) {
    c0 = clock64();
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  }
  for (int i = threadIdx.x; i < 32 * TM; i += blockDim.x) sa[i] = (T)1 + (T)1e-3 * (T)(i % 11);
  for (int i = threadIdx.x; i < 32 * TN; i += blockDim.x) sb[i] = (T)1e-7 * (T)(1 + i % 13);
  __syncthreads();
  T acc[TM][TN];
#pragma unroll
  for (int m = 0; m < TM; m++)
#pragma unroll
    for (int n = 0; n < TN; n++) acc[m][n] = (T)0;
  for (int64_t it = 0; it < iters; it++) {
#pragma unroll 4
    for (int k = 0; k < 32; k++) {
      T av[TM], bv[TN];
      lds_vec<T, TM, TM>(sa + k * TM, av);
      lds_vec<T, TN, TN>(sb + k * TN, bv);
#pragma unroll
      for (int m = 0; m < TM; m++)
#pragma unroll
        for (int n = 0; n < TN; n++) acc[m][n] = fma(av[m], bv[n], acc[m][n]);
    }
  }
  T s = 0;
#pragma unroll
  for (int m = 0; m < TM; m++)
#pragma unroll
    for (int n = 0; n < TN; n++) s += acc[m][n];
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
    fma_probe_kernel<double><<<grid, 256, 0, s>>>(iters, static_cast<double *>(out), clk);
  else
    fma_probe_kernel<float><<<grid, 256, 0, s>>>(iters, static_cast<float *>(out), clk);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("fem_probe_fma: ") + cudaGetErrorString(e));
    return FEM_ECUDA;
  }
  return FEM_OK;
}
