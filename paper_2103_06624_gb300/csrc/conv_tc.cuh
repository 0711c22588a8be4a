// Conv layers on the tensor cores (BF16 operands, FP32 accumulation) for the layer-by-layer
// path of the BF16 precision.  Declarations used by the C-ABI layer.
#pragma once

#include "kernels_simt.cuh"

namespace bcrown {

bool tcg_supported(const bcrown_net* net);
// Bytes of im2col operand per row of the largest pass (gather: conv operands built in shared
// memory, only fully connected layers use the buffer).
size_t tcg_col_bytes_per_row(const bcrown_net* net, bool gather);
// Contraction of conv layer i for R rows: im2col of the operand into `col` (col_bytes long),
// then tcgen05 GEMMs.  fwd = false: dst = A^(i-1) = the transposed convolution of src =
// Lambda^(i) (one GEMM per stride phase); fwd = true: dst = W^(i) h + b^(i) from src = h.
int tcg_conv(bcrown_net* net, int i, bool fwd, int R, const float* src, float* dst, const float* bias, char* col,
             size_t col_bytes, cudaStream_t s);
void tcg_release(const bcrown_net* net);

}  // namespace bcrown
