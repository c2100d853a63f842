// FP32 kernels with a per-point nonlinear coefficient law (exact or network).
#include "fem_fma.cuh"

namespace fem {
int launch_fma_law_f32(int elem, int p, int law, const FmaArgs &a, void *stream) {
  if (law == 1) return launch_fma_any<float, 1>(elem, p, a, stream);
  if (law == 2) return launch_fma_any<float, 2>(elem, p, a, stream);
  return FEM_EINVAL;
}
}  // namespace fem
