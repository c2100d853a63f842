// FP64 instantiations of the CUDA-core contraction kernels.
#include "fem_fma.cuh"

namespace fem {
int launch_fma_f64(int elem, int p, const FmaArgs &a, void *stream) {
  return launch_fma_any<double>(elem, p, a, stream);
}
int launch_fma_elastic_f64(int p, const FmaArgs &a, void *stream) {
  return launch_fma_elastic<double>(p, a, stream);
}
}  // namespace fem
