// Instantiations of the CUDA-core contraction kernels that read stored
// Jacobian terms (split geometry, the paper's NOJAC variants) instead of
// computing J from the vertex coordinates.
#include "fem_fma.cuh"

namespace fem {
int launch_fma_terms(int elem, int p, int prec, const FmaArgs &a, void *stream) {
  return prec == FEM_F64 ? launch_fma_any<double, 0, true>(elem, p, a, stream)
                         : launch_fma_any<float, 0, true>(elem, p, a, stream);
}
int launch_fma_elastic_terms(int p, int prec, const FmaArgs &a, void *stream) {
  return prec == FEM_F64 ? launch_fma_elastic<double, true>(p, a, stream)
                         : launch_fma_elastic<float, true>(p, a, stream);
}
}  // namespace fem
