// Tensor-core bound pass (placeholder until the tcgen05 kernel lands).
#include "fused_tc.cuh"

namespace bcrown {

bool tc_supported(const bcrown_net*) { return false; }
size_t tc_workspace_bytes(const bcrown_net*, int, bool) { return 0; }
int tc_bound(bcrown_net*, const bcrown_domain*, const bcrown_batch*, const Tables&, char*, size_t, bool,
             const float*, const float*, float*, float*, float*, cudaStream_t) {
  return fail(BCROWN_ERR_UNIMPLEMENTED, "tensor-core path not built");
}

}  // namespace bcrown
