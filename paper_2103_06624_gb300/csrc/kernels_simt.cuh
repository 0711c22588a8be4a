// SIMT (CUDA-core) kernels of the bound pass, its adjoint and the optimiser.
//
// Paper references: relaxation Lemma 2.1 / Eq. definition_D, definition_lowerb;
// recursion Eq. definition_A; concretisation Eq. beta_crown_lp (box form);
// optimiser Eq. opt_alpha_beta with Adam (Appendix C.1).
#pragma once

#include "bcrown_internal.cuh"

namespace bcrown {

// ----------------------------------------------------------------------------------------
// Per-row context
// ----------------------------------------------------------------------------------------
struct RowsCtx {
  int r0;      // first global row of this chunk
  int R;       // rows in this chunk
  int K;       // specs
  int P;       // properties
  BatchView bt;
  Tables tb;
  const float* x_lo;
  const float* x_hi;
  const float* l;
  const float* u;
  int* status;
};

__device__ __forceinline__ void flag(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Split entries of one row that fall in hidden layer `layer`, staged in shared memory.
struct SplitSlot {
  int idx;
  int sign;
  int t;  // position in the subdomain's split list (beta slot)
};

// Loads the row's split list filtered to `layer`; returns the count (block-uniform).
// Invalid entries (layer/index/sign out of range, list too long) are skipped and flagged.
__device__ __forceinline__ int stage_splits(const RowsCtx& c, int b, int layer, int d_layer,
                                            SplitSlot* slots, int* n_slots) {
  if (threadIdx.x == 0) *n_slots = 0;
  __syncthreads();
  int cnt = c.bt.split_cnt[b];
  int off = c.bt.split_off[b];
  if (cnt < 0 || cnt > BCROWN_MAX_SPLITS) {
    if (threadIdx.x == 0) flag(c.status, BCROWN_ERR_ARG);
    cnt = 0;
  }
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    int ly = c.bt.split_layer[off + t];
    int j = (int)c.bt.split_idx[off + t];
    int s = c.bt.split_sign[off + t];
    if (s != -1 && s != 1) {
      flag(c.status, BCROWN_ERR_ARG);
      continue;
    }
    if (ly != layer) continue;
    if (j < 0 || j >= d_layer) {
      flag(c.status, BCROWN_ERR_ARG);
      continue;
    }
    int q = atomicAdd(n_slots, 1);
    slots[q] = SplitSlot{j, s, t};
  }
  __syncthreads();
  return *n_slots;
}

// Per-row bitmask of the layer's split neurons (bit j of mask[j / 32]), so that the per-neuron
// test is one shared-memory load instead of a scan of the split list; the list is scanned only
// for neurons whose bit is set.  Block-wide: words [0, ceil(d / 32)) are written.
constexpr int SPLIT_MASK_WORDS = 8192;  // layers of up to 262144 neurons; wider ones scan the list
__device__ __forceinline__ void split_mask_block(const SplitSlot* slots, int ns, int d, uint32_t* mask) {
  for (int w = threadIdx.x; w < (d + 31) / 32; w += blockDim.x) mask[w] = 0u;
  __syncthreads();
  for (int q = threadIdx.x; q < ns; q += blockDim.x) atomicOr(&mask[slots[q].idx >> 5], 1u << (slots[q].idx & 31));
  __syncthreads();
}
__device__ __forceinline__ bool split_bit(const uint32_t* mask, int j) { return (mask[j >> 5] >> (j & 31)) & 1u; }

// Valid-layer check for splits across all layers (done once per row by the init kernel).
__device__ __forceinline__ bool row_prop(const RowsCtx& c, int rl, int* b, int* k, int* p) {
  int r = c.r0 + rl;
  *b = r / c.K;
  *k = r - *b * c.K;
  *p = c.bt.prop_of[*b];
  return (*p >= 0 && *p < c.P);
}

// ----------------------------------------------------------------------------------------
// Block reductions
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int MODE>  // 0 nearest, 1 toward -inf, 2 toward +inf
__device__ __forceinline__ double dadd(double a, double b) {
  if (MODE == 1) return __dadd_rd(a, b);
  if (MODE == 2) return __dadd_ru(a, b);
  return a + b;
}

template <int MODE>
__device__ __forceinline__ double warp_dsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v = dadd<MODE>(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// FP32 sums with a rounding direction: MODE 0 nearest, 1 down (toward -inf), 2 up.  Directed
// rounding at every step makes the result a lower (1) or upper (2) bound of the exact sum.
template <int MODE>
__device__ __forceinline__ float fadd(float a, float b) {
  if (MODE == 1) return __fadd_rd(a, b);
  if (MODE == 2) return __fadd_ru(a, b);
  return a + b;
}
template <int MODE>
__device__ __forceinline__ float block_fsum(float v, float* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fadd<MODE>(v, __shfl_xor_sync(0xffffffffu, v, o));
  int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  float s = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.f;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) s = fadd<MODE>(s, __shfl_xor_sync(0xffffffffu, s, o));
  if (threadIdx.x == 0) sh[0] = s;
  __syncthreads();
  return sh[0];
}

// Sum over the block (result valid in every thread).  `sh` needs 32 entries.
__device__ __forceinline__ float block_sum(float v, float* sh) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  float s = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.f;
  if (w == 0) s = warp_sum(s);
  if (threadIdx.x == 0) sh[0] = s;
  __syncthreads();
  return sh[0];
}

template <int MODE>
__device__ __forceinline__ double block_dsum(double v, double* sh) {
  v = warp_dsum<MODE>(v);
  int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  double s = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) s = warp_dsum<MODE>(s);
  if (threadIdx.x == 0) sh[0] = s;
  __syncthreads();
  return sh[0];
}

}  // namespace bcrown
