// BF16 layer-by-layer bound pass for networks the fused kernel does not take (conv layers, wide
// fully connected layers): every contraction a tcgen05 GEMM whose epilogue applies the next step
// of the recursion (relaxation, beta shift and bias sums; concretisation; the adjoint).
// Declarations used by the C-ABI layer.
#pragma once

#include "kernels_simt.cuh"

namespace bcrown {

bool lt_supported(const bcrown_net* net);
// Device workspace for R rows of P properties (grad: with the stash of A at the unstable
// neurons, n_alpha long).
size_t lt_workspace_bytes(const bcrown_net* net, int R, int P, int64_t n_alpha, bool grad);
// Bound (and with grad, dlb/dalpha and dlb/dbeta) of the batch's rows on the BF16 layer path.
int lt_bound(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* bt, const Tables& tb, char* ws,
             size_t ws_bytes, bool grad, const float* alpha, const float* beta, float* lb, float* dalpha,
             float* dbeta, cudaStream_t s);
void lt_release(const bcrown_net* net);

}  // namespace bcrown
