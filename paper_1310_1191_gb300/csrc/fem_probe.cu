// Throughput probe of the FP64 and FP32 FMA pipes: the denominators of the
// rooflines of the CUDA-core kernels are measured with it rather than taken
// from unit counts and clocks.  Two loop forms: (0) independent chains
// a <- a x + y, 8 per thread; (1) the contraction kernels' inner loop, a
// TM x TN register tile of accumulators plus, per step, the outer product of
// a TM-vector and a TN-vector loaded from shared memory.  On this GPU the
// chains reach about 85 % of the FP64 pipe and the outer products all of it,
// while in FP32 the chains come closer to the pipe than the outer products
// (whose shared loads and registers limit them); the caller takes the better
// form per type.
#include <cuda_runtime.h>

#include <string>

#include "fem_fma.cuh"
#include "fem_internal.h"

namespace fem {

template <class T> struct ProbeTile;
template <> struct ProbeTile<double> { static constexpr int TM = 4, TN = 4; };
template <> struct ProbeTile<float> { static constexpr int TM = 8, TN = 8; };

__device__ __forceinline__ void probe_clock(int64_t *c, int64_t *t) {
  *c = clock64();
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(*t));
}

// form 0: 8 independent multiply-add chains per thread, iters steps each
template <class T>
__global__ void __launch_bounds__(256) fma_probe_chains(int64_t iters, T x, T y, T *out, int64_t *clk) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t c0 = 0, t0 = 0;
  if (clk && threadIdx.x == 0) probe_clock(&c0, &t0);
  T a[8];
#pragma unroll
  for (int k = 0; k < 8; k++) a[k] = (T)(1 + (tid + k) % 7) * (T)0.125;
  for (int64_t i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = fma(a[k], x, y);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) s += a[k];
  out[tid] = s;
  if (clk && threadIdx.x == 0) {  // this CTA's SM clock cycles and nanoseconds
    int64_t c1, t1;
    probe_clock(&c1, &t1);
    clk[2 * blockIdx.x] = c1 - c0;
    clk[2 * blockIdx.x + 1] = t1 - t0;
  }
}

// form 1: register-tile outer products from shared memory.  Every access
// stays in bounds: shared indexes < 32 TM and 32 TN, out[tid] with
// tid < gridDim.x * 256 = n_threads, clk[2 blockIdx.x + 1] < 2 gridDim.x
template <class T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, T *out, int64_t *clk) {
  constexpr int TM = ProbeTile<T>::TM, TN = ProbeTile<T>::TN;
  __shared__ __align__(16) T sa[32 * TM];
  __shared__ __align__(16) T sb[32 * TN];
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t c0 = 0, t0 = 0;
  if (clk && threadIdx.x == 0) probe_clock(&c0, &t0);
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

extern "C" int fem_probe_fma(int fp64, int form, int64_t iters, int64_t n_threads, void *out, int64_t *clk,
                             void *stream) {
  if (iters < 1 || n_threads < 256 || n_threads % 256 != 0 || n_threads / 256 > 0x7fffffffLL || !out ||
      ((uintptr_t)out & 7) || ((uintptr_t)clk & 7) || (form != 0 && form != 1)) {
    set_error("fem_probe_fma: form 0 or 1, iters >= 1, n_threads a positive multiple of 256, "
              "8-byte aligned out and clk");
    return FEM_EINVAL;
  }
  const unsigned grid = (unsigned)(n_threads / 256);
  cudaStream_t s = (cudaStream_t)stream;
  if (form == 0) {
    if (fp64)
      fma_probe_chains<double><<<grid, 256, 0, s>>>(iters, 0.99999, 1e-5, static_cast<double *>(out), clk);
    else
      fma_probe_chains<float><<<grid, 256, 0, s>>>(iters, 0.99999f, 1e-5f, static_cast<float *>(out), clk);
  } else if (fp64) {
    fma_probe_kernel<double><<<grid, 256, 0, s>>>(iters, static_cast<double *>(out), clk);
  } else {
    fma_probe_kernel<float><<<grid, 256, 0, s>>>(iters, static_cast<float *>(out), clk);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("fem_probe_fma: ") + cudaGetErrorString(e));
    return FEM_ECUDA;
  }
  return FEM_OK;
}
