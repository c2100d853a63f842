// Instantiations of the CUDA-core contraction kernels for linear
// elastostatics on prisms with the paper's quadrature rule (Table 1's point
// counts), FP64 and FP32.
#include "fem_fma.cuh"

namespace fem {
int launch_fma_t1_elastic_f64(int p, const FmaArgs &a, void *stream) {
  return launch_fma_elastic_table1<double>(p, a, stream);
}
int launch_fma_t1_elastic_f32(int p, const FmaArgs &a, void *stream) {
  return launch_fma_elastic_table1<float>(p, a, stream);
}
}  // namespace fem
