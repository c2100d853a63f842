// Instantiations of the tensor-core kernel: BF16x3 scalar form, collapsed rule.
#include "fem_tc.cuh"

namespace fem {
int launch_tc_scalar_bf16(int p, const TcArgs &a, void *stream) { return launch_tc_any<false, false>(p, a, stream); }
}  // namespace fem
