// Instantiations of the tensor-core kernel: nonlinear coefficient law, exact (1) or network (2), BF16x3, collapsed rule.
#include "fem_tc.cuh"

namespace fem {
int launch_tc_law(int p, int law, const TcArgs &a, void *stream) {
  return law == 1 ? launch_tc_any<false, false, 1>(p, a, stream) : launch_tc_any<false, false, 2>(p, a, stream);
}
}  // namespace fem
