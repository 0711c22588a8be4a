// Tensor-core (tcgen05, BF16 operands, FP32 accumulation in TMEM) bound pass for fully
// connected networks.  Declarations used by the C-ABI layer.
#pragma once

#include <cuda_bf16.h>

#include "kernels_simt.cuh"

namespace bcrown {

bool tc_supported(const bcrown_net* net);
// Device workspace of the fused path for B subdomains of P properties: the row plan and, with
// the gradient, the stash of A^(i).
size_t tc_workspace_bytes(const bcrown_net* net, int B, int P, bool grad);
// plan = true (re)builds the grouping of the batch's rows into property-uniform tiles in the
// workspace; a later call on the same batch and workspace may pass false to reuse it.  With
// dalpha16 set (and grad), dlb/dalpha is written there in BF16 instead of to dalpha.
int tc_bound(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* bt, const Tables& tb, char* ws,
             size_t ws_bytes, bool grad, bool plan, const float* alpha, const float* beta, float* lb, float* dalpha,
             float* dbeta, cudaStream_t s, __nv_bfloat16* dalpha16 = nullptr);

void tc_release(const bcrown_net* net);

}  // namespace bcrown
