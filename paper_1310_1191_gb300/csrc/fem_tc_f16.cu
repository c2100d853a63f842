// Instantiations of the tensor-core kernel: FP16x3 scalar form, collapsed rule.
#include "fem_tc.cuh"

namespace fem {
int launch_tc_scalar_f16(int p, const TcArgs &a, void *stream) { return launch_tc_any<true, false>(p, a, stream); }
}  // namespace fem
