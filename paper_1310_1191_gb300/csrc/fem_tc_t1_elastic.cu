// Instantiations of the tensor-core kernel: linear elastostatics (BF16x3 and
// FP16x3) with the paper's rule (Table 1's point counts).
#include "fem_tc.cuh"

namespace fem {
int launch_tc_elastic_t1(int p, bool f16, const TcArgs &a, void *stream) {
  return f16 ? launch_tc_any<true, true, 0, FEM_RULE_TABLE1>(p, a, stream)
             : launch_tc_any<false, true, 0, FEM_RULE_TABLE1>(p, a, stream);
}
}  // namespace fem
