// Tensor-core (tcgen05, BF16 operands, FP32 accumulation in TMEM) bound pass for fully
// connected networks.  Declarations used by the C-ABI layer.
#pragma once

#include "kernels_simt.cuh"

namespace bcrown {

bool tc_supported(const bcrown_net* net);
size_t tc_workspace_bytes(const bcrown_net* net, int R, bool grad);
int tc_bound(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* bt, const Tables& tb, char* ws,
             size_t ws_bytes, bool grad, const float* alpha, const float* beta, float* lb, float* dalpha,
             float* dbeta, cudaStream_t s);

void tc_release(const bcrown_net* net);

}  // namespace bcrown
