// FP32 instantiations of the CUDA-core contraction kernels (geometry in FP64,
// point matrices rounded to FP32, FP32 FMA contraction and outputs).
#include "fem_fma.cuh"

namespace fem {
int launch_fma_f32(int elem, int p, const FmaArgs &a, void *stream) {
  return launch_fma_any<float>(elem, p, a, stream);
}
int launch_fma_elastic_f32(int p, const FmaArgs &a, void *stream) {
  return launch_fma_elastic<float>(p, a, stream);
}
}  // namespace fem
