// Instantiations of the tensor-core kernel: linear elastostatics (BF16x3 and FP16x3), collapsed rule.
#include "fem_tc.cuh"

namespace fem {
int launch_tc_elastic(int p, bool f16, const TcArgs &a, void *stream) {
  return f16 ? launch_tc_any<true, true>(p, a, stream) : launch_tc_any<false, true>(p, a, stream);
}
}  // namespace fem
