// CUDA-core kernels: per-property tables, the relaxation epilogue, FP32 contractions
// (dense and convolution), concretisation, the adjoint epilogue, projected Adam,
// batch_split and the rigorous (CERTIFY) variants.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "kernels_simt.cuh"
#include "simt.cuh"

namespace bcrown {

std::atomic<long long> g_launches{0};

// ----------------------------------------------------------------------------------------
// Per-property tables from l, u: code, unstable rank, upper chord (Lemma 2.1)
// ----------------------------------------------------------------------------------------
// Property p's neurons in segments of TAB_SEG, one block per (property, segment).  With more
// than one segment the unstable ranks need each segment's offset: k_tables_count counts a
// segment's unstable neurons into the first rank slot of the segment, k_tables_scan turns
// those counts into exclusive offsets in place (and U[p] = the total), and k_tables starts
// from the offset in its first slot, which only its own block reads and overwrites.
constexpr int TAB_SEG = 4096;

__device__ __forceinline__ bool is_unstable(float lv, float uv) { return lv < 0.f && uv > 0.f; }

__global__ void __launch_bounds__(1024) k_tables_count(int H, const float* __restrict__ l,
                                                       const float* __restrict__ u, int32_t* rank) {
  __shared__ int tot;
  const int p = blockIdx.x, seg = blockIdx.y;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  int c = 0;
  const int end = min(H, (seg + 1) * TAB_SEG);
  for (int n = seg * TAB_SEG + threadIdx.x; n < end; n += blockDim.x)
    c += is_unstable(l[(size_t)p * H + n], u[(size_t)p * H + n]) ? 1 : 0;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) atomicAdd(&tot, c);
  __syncthreads();
  if (threadIdx.x == 0) rank[(size_t)p * H + (size_t)seg * TAB_SEG] = tot;
}

__global__ void k_tables_scan(int H, int nseg, int32_t* rank, int32_t* U) {
  const int p = blockIdx.x;
  if (threadIdx.x != 0) return;
  int run = 0;
  for (int q = 0; q < nseg; ++q) {
    int32_t* slot = rank + (size_t)p * H + (size_t)q * TAB_SEG;
    const int c = *slot;
    *slot = run;
    run += c;
  }
  U[p] = run;
}

__global__ void __launch_bounds__(1024) k_tables(int H, int nseg, const float* __restrict__ l,
                                                 const float* __restrict__ u, uint8_t* code,
                                                 int32_t* rank, float* slope, float* icpt,
                                                 int32_t* U) {
  __shared__ int warp_tot[32];
  __shared__ int running;
  const int p = blockIdx.x, seg = blockIdx.y;
  const float* lp = l + (size_t)p * H;
  const float* up = u + (size_t)p * H;
  if (threadIdx.x == 0) running = nseg > 1 ? rank[(size_t)p * H + (size_t)seg * TAB_SEG] : 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int end = min(H, (seg + 1) * TAB_SEG);
  for (int base = seg * TAB_SEG; base < end; base += blockDim.x) {
    int n = base + threadIdx.x;
    float lv = 0.f, uv = 0.f;
    bool un = false;
    if (n < end) {
      lv = lp[n];
      uv = up[n];
      un = is_unstable(lv, uv);
    }
    unsigned m = __ballot_sync(0xffffffffu, un);
    int pre = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[w] = __popc(m);
    __syncthreads();
    int woff = 0, tot = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      if (q < w) woff += warp_tot[q];
      tot += warp_tot[q];
    }
    if (n < end) {
      size_t g = (size_t)p * H + n;
      uint8_t c = un ? CODE_UNSTABLE : (lv >= 0.f ? CODE_ACTIVE : CODE_INACTIVE);
      code[g] = c;
      rank[g] = un ? running + woff + pre : -1;
      float sl = 0.f, ic = 0.f;
      if (un) {
        // upper chord u (z - l) / (u - l) with its slope and intercept rounded up: still an
        // upper bound of ReLU on [l, u] (z - l >= 0 there), so every precision may use it
        sl = __fdiv_ru(uv, __fsub_rd(uv, lv));
        ic = __fmul_ru(sl, -lv);
      }
      slope[g] = sl;
      icpt[g] = ic;
    }
    __syncthreads();
    if (threadIdx.x == 0) running += tot;
    __syncthreads();
  }
  if (nseg == 1 && threadIdx.x == 0) U[p] = running;
}

// Loads issued where they are written (volatile asm keeps a batch of independent loads ahead
// of the code that uses them instead of letting the compiler sink each to its first use);
// 0 when pred is false.
__device__ __forceinline__ float ld_f32(const float* p, bool pred) {
  float v;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.f32 %0, 0f00000000;\n\t@q ld.global.f32 %0, [%1];\n\t}"
               : "=f"(v)
               : "l"(p), "r"((uint32_t)pred)
               : "memory");
  return v;
}
__device__ __forceinline__ int32_t ld_s32(const int32_t* p, bool pred) {
  int32_t v;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.s32 %0, 0;\n\t@q ld.global.s32 %0, [%1];\n\t}"
               : "=r"(v)
               : "l"(p), "r"((uint32_t)pred)
               : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_u8(const uint8_t* p, bool pred, uint32_t dflt) {
  uint32_t v;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.u32 %0, %3;\n\t@q ld.global.u8 %0, [%1];\n\t}"
               : "=r"(v)
               : "l"(p), "r"((uint32_t)pred), "r"(dflt)
               : "memory");
  return v;
}

// M^(i)_m: bound on |h^(i)_m| (max(u,0) for hidden layers, max(|x_lo|,|x_hi|) at the input)
__device__ __forceinline__ float hmax_hidden(float uv) { return fmaxf(uv, 0.f); }

// wm[p][hoff_i + j] = sum_m |W^(i)_jm| M^(i-1)_m, every product and sum rounded up (FP32),
// for the a priori contraction error of layer i.  One warp per output neuron.
__global__ void __launch_bounds__(256) k_absw_m(LayerGeom g, const float* __restrict__ W, int P, int H,
                                                long long hoff_i, long long hoff_prev, const float* __restrict__ u,
                                                const float* __restrict__ x_lo, const float* __restrict__ x_hi,
                                                int d0, float* __restrict__ wm) {
  const long long id = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)P * g.d_out;
  if (id >= total) return;
  const int p = (int)(id / g.d_out);
  const int j = (int)(id - (long long)p * g.d_out);
  auto M = [&](int m) -> float {
    if (hoff_prev < 0) return fmaxf(fabsf(x_lo[(size_t)p * d0 + m]), fabsf(x_hi[(size_t)p * d0 + m]));
    return hmax_hidden(u[(size_t)p * H + hoff_prev + m]);
  };
  float s = 0.f;
  if (g.kind == BCROWN_LAYER_FC) {
    const float* w = W + (size_t)j * g.d_in;
    for (int m = lane; m < g.d_in; m += 32) s = __fadd_ru(s, __fmul_ru(fabsf(w[m]), M(m)));
  } else {
    const int hw = g.out_h * g.out_w;
    const int co = j / hw, rem = j - co * hw, oy = rem / g.out_w, ox = rem - oy * g.out_w;
    const int kk = g.k * g.k;
    for (int t = lane; t < g.in_c * kk; t += 32) {
      const int ci = t / kk, r = t - ci * kk, ky = r / g.k, kx = r - ky * g.k;
      const int iy = oy * g.stride - g.pad + ky, ix = ox * g.stride - g.pad + kx;
      if (iy < 0 || iy >= g.in_h || ix < 0 || ix >= g.in_w) continue;
      const float w = fabsf(W[(((size_t)co * g.in_c + ci) * g.k + ky) * g.k + kx]);
      s = __fadd_ru(s, __fmul_ru(w, M((ci * g.in_h + iy) * g.in_w + ix)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) s = __fadd_ru(s, __shfl_xor_sync(0xffffffffu, s, o));
  if (lane == 0) wm[(size_t)p * H + hoff_i + j] = s;
}

// ----------------------------------------------------------------------------------------
// Top of the recursion: A^(L-1) = Wbar_k, c = bbar_k (Theorem 3.1 base case)
// ----------------------------------------------------------------------------------------
template <bool CERT>
__global__ void __launch_bounds__(256) k_init_top(RowsCtx c, int dtop, const float* __restrict__ Wbar,
                                                  const float* __restrict__ bbar, const double* __restrict__ bbar_rd,
                                                  const float* __restrict__ Wbar_err, long long hoff_top,
                                                  float* __restrict__ A, float* __restrict__ cf,
                                                  double* __restrict__ cd, double* __restrict__ E) {
  __shared__ float shf[32];
  int rl = blockIdx.x;
  int b, k, p;
  bool ok = row_prop(c, rl, &b, &k, &p);
  if (!ok) {
    if (threadIdx.x == 0) flag(c.status, BCROWN_ERR_ARG);
    p = 0;
  }
  const float* w = Wbar + (size_t)k * dtop;
  float e = 0.f;
  for (int j = threadIdx.x; j < dtop; j += blockDim.x) {
    A[(size_t)rl * dtop + j] = w[j];
    if (CERT) {
      float M = hoff_top >= 0 ? hmax_hidden(c.u[(size_t)p * c.tb.H + hoff_top + j])
                              : fmaxf(fabsf(c.x_lo[(size_t)p * dtop + j]), fabsf(c.x_hi[(size_t)p * dtop + j]));
      e = __fadd_ru(e, __fmul_ru(Wbar_err[(size_t)k * dtop + j], M));
    }
  }
  if (CERT) {
    e = block_fsum<2>(e, shf);
    if (threadIdx.x == 0) {
      cd[rl] = ok ? bbar_rd[k] : -INFINITY;
      E[rl] = e;
    }
  } else if (threadIdx.x == 0) {
    cf[rl] = ok ? bbar[k] : -INFINITY;
  }
}

// ----------------------------------------------------------------------------------------
// Relaxation + beta shift + bias (Eq. definition_D, definition_lowerb, definition_A):
//   Lambda_j = A_j D_j + beta_j S_jj ;  c += Lambda_j b_j + A_j lambda_j
// One warp per row (RELAX_ROWS rows per block): the row's splits of this layer are compacted
// into shared memory by ballots, neurons are strided over the lanes, sums are warp reductions.
// CERT: outward chord constants (from the tables), c summed rounded down, error terms rounded up.
// ----------------------------------------------------------------------------------------
constexpr int RELAX_WARPS = 8;   // warps per block; WPR of them share a row (wide layers: all 8)
// All four codes stable (active or inactive): no alpha, chord or split term.
__device__ __forceinline__ bool stable4(uchar4 c4) {
  return c4.x != CODE_UNSTABLE && c4.y != CODE_UNSTABLE && c4.z != CODE_UNSTABLE && c4.w != CODE_UNSTABLE;
}
__device__ __forceinline__ float d01(unsigned char code) { return code == CODE_ACTIVE ? 1.f : 0.f; }

// Relaxation of 4 consecutive neurons n .. n + 3 (n a multiple of 4, rows 16-byte aligned) of a
// group that holds an unstable or a split neuron, the group's loads issued together: the 4 ranks
// (one 16-byte load) where a neuron is unstable, the 4 chords where one takes the chord, then
// the alphas.  (The vectorised loops branch to it only for such groups: a version without the
// branch, every lane running these loads under predicates, measured 20 % slower.)
// alpha_row: the row's alpha block, checked against the array once per row (null: none).
// D, lambda per neuron (split neurons are left to the caller) and rk = the rank of an unstable
// neuron, -1 otherwise.
__device__ __forceinline__ void group4(const Tables& tb, size_t n, const float a[4], const uchar4 c4,
                                       const float* __restrict__ alpha_row, float D[4], float lm[4], int rk[4]) {
  const uint8_t cd[4] = {c4.x, c4.y, c4.z, c4.w};
  bool un[4], any_un = false, any_ch = false;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    un[v] = cd[v] == CODE_UNSTABLE;
    any_un |= un[v];
    any_ch |= un[v] && a[v] < 0.f;
  }
  int4 r4 = make_int4(-1, -1, -1, -1);
  float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f), i4 = s4;
  if (any_un) r4 = __ldg(reinterpret_cast<const int4*>(tb.rank + n));
  if (any_ch) {
    s4 = __ldg(reinterpret_cast<const float4*>(tb.slope + n));
    i4 = __ldg(reinterpret_cast<const float4*>(tb.icpt + n));
  }
  const int r[4] = {r4.x, r4.y, r4.z, r4.w};
  const float sl[4] = {s4.x, s4.y, s4.z, s4.w}, ic[4] = {i4.x, i4.y, i4.z, i4.w};
  float al[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) al[v] = (un[v] && a[v] >= 0.f && alpha_row != nullptr) ? alpha_row[r[v]] : 0.f;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    rk[v] = un[v] ? r[v] : -1;
    D[v] = cd[v] == CODE_ACTIVE ? 1.f : (un[v] ? (a[v] >= 0.f ? fminf(fmaxf(al[v], 0.f), 1.f) : sl[v]) : 0.f);
    lm[v] = (un[v] && a[v] < 0.f) ? ic[v] : 0.f;
  }
}

template <bool CERT, int WPR>
__global__ void __launch_bounds__(32 * RELAX_WARPS) k_relax(RowsCtx c, int layer, int d, long long hoff,
                                                           const float* __restrict__ Ain, float* __restrict__ Lam,
                                                           const float* __restrict__ bias,
                                                           const float* __restrict__ alpha, int64_t n_alpha,
                                                           const float* __restrict__ beta, int64_t n_beta,
                                                           float* __restrict__ cf, double* __restrict__ cd,
                                                           double* __restrict__ E, const float* __restrict__ wm,
                                                           double gamma) {
  constexpr int RPB = RELAX_WARPS / WPR;   // rows per block
  __shared__ SplitSlot slots[RPB][BCROWN_MAX_SPLITS];
  __shared__ int nslots[RPB];
  // split bitmask of a wide row (a whole block's row, up to SPLIT_MASK_WORDS * 32 neurons)
  constexpr int MW = WPR > 1 ? SPLIT_MASK_WORDS : 1;
  __shared__ uint32_t smask[RPB][MW];
  __shared__ float red[RELAX_WARPS][3];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rs = w / WPR, sub = w - rs * WPR;   // row slot in the block, warp within the row
  const int rl = blockIdx.x * RPB + rs;
  const bool live = rl < c.R;   // dead warps still take part in the block barriers
  int b = 0, k = 0, p = 0, cnt = 0, off = 0;
  if (live) {
    if (!row_prop(c, rl, &b, &k, &p)) p = 0;
    cnt = c.bt.split_cnt[b];
    off = c.bt.split_off[b];
    if (cnt < 0 || cnt > BCROWN_MAX_SPLITS) {
      if (lane == 0 && sub == 0) flag(c.status, BCROWN_ERR_ARG);
      cnt = 0;
    }
  }
  // this layer's splits of the row, in list order (first warp of the row)
  if (live && sub == 0) {
    int ns = 0;
    for (int t0 = 0; t0 < cnt; t0 += 32) {
      const int t = t0 + lane;
      bool keep = false;
      int j = 0, sg = 0;
      if (t < cnt) {
        const int ly = c.bt.split_layer[off + t];
        j = (int)c.bt.split_idx[off + t];
        sg = c.bt.split_sign[off + t];
        if (sg != -1 && sg != 1) flag(c.status, BCROWN_ERR_ARG);
        else if (ly == layer) {
          if (j < 0 || j >= d) flag(c.status, BCROWN_ERR_ARG);
          else keep = true;
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) slots[rs][ns + __popc(m & ((1u << lane) - 1u))] = SplitSlot{j, sg, t};
      ns += __popc(m);
    }
    if (lane == 0) nslots[rs] = ns;
  }
  if (WPR > 1) __syncthreads();
  else __syncwarp();
  const bool use_mask = WPR > 1 && d <= MW * 32;
  if (use_mask) {
    if (live)
      for (int q = sub * 32 + lane; q < (d + 31) / 32; q += 32 * WPR) smask[rs][q] = 0u;
    if (WPR > 1) __syncthreads();
    else __syncwarp();
    if (live)
      for (int q = sub * 32 + lane; q < nslots[rs]; q += 32 * WPR) {
        const int jj = slots[rs][q].idx;
        atomicOr(&smask[rs][jj >> 5], 1u << (jj & 31));
      }
    if (WPR > 1) __syncthreads();
    else __syncwarp();
  }
  float acc = 0.f, e1 = 0.f, e2 = 0.f;
  if (live) {
    const int ns = nslots[rs];
    const SplitSlot* sl_ = slots[rs];
    const int Up = c.tb.U[p];
    const long long abase = c.bt.alpha_off[b] + (long long)k * Up;
    const long long bbase = (long long)off * c.K + (long long)k * cnt;
    const float* a_row = Ain + (size_t)rl * d;
    float* lam_row = Lam + (size_t)rl * d;
    // CERT: acc is a lower bound of sum_j Lambda_j b_j + A_j lambda_j (every operation rounded
    // down); e1, e2 are upper bounds (rounded up) of the error terms below.
    const size_t n0 = (size_t)p * c.tb.H + hoff;
    // Rows of up to 2048 neurons (one warp each): one neuron per lane per step, the split list
    // scanned per neuron (short for these rows); measured faster there than the wide-row code
    // below, which the wide (conv) layers need.
    if (WPR == 1) {
  #pragma unroll 4
      for (int j = sub * 32 + lane; j < d; j += 32 * WPR) {
        const float a = a_row[j];
        const size_t n = (size_t)p * c.tb.H + hoff + j;
        int s = 0;
        float bet = 0.f;
        for (int q = 0; q < ns; ++q)
          if (sl_[q].idx == j) {
            s = sl_[q].sign;
            const long long bi = bbase + sl_[q].t;
            if (bi >= 0 && bi < n_beta) bet = fmaxf(beta[bi], 0.f);
            else flag(c.status, BCROWN_ERR_ARG);
          }
        float D = 0.f, lm = 0.f;
        const uint8_t code = c.tb.code[n];
        if (s == -1) D = 1.f;
        else if (s == 1) D = 0.f;
        else if (code == CODE_ACTIVE) D = 1.f;
        else if (code == CODE_INACTIVE) D = 0.f;
        else if (a >= 0.f) {
          const long long ai = abase + c.tb.rank[n];
          if (ai < 0 || ai >= n_alpha) {
            flag(c.status, BCROWN_ERR_ARG);
            D = 0.f;
          } else {
            D = fminf(fmaxf(alpha[ai], 0.f), 1.f);
          }
        } else {
          // upper chord, slope and intercept rounded up (outward) in the tables
          D = c.tb.slope[n];
          lm = c.tb.icpt[n];
        }
        const float L = fmaf(a, D, bet * (float)s);
        lam_row[j] = L;
        const float bj = bias[j];
        if (CERT) {
          acc = __fadd_rd(acc, __fadd_rd(__fmul_rd(L, bj), __fmul_rd(a, lm)));
          const bool exact = (s == 0) && (D == 0.f || D == 1.f);
          if (!exact) {
            // Lambda_j was rounded once: |error| <= 2^-23 |Lambda_j| (+ an underflow margin),
            // acting on |z_j| <= max(|l_j|, |u_j|)
            const float zmax = fmaxf(fabsf(c.l[n]), fabsf(c.u[n]));
            const float er = __fmaf_ru(fabsf(L), 0x1p-23f, 0x1p-140f);
            e1 = __fadd_ru(e1, __fmul_ru(er, zmax));
          }
          e2 = __fadd_ru(e2, __fmul_ru(fabsf(L), wm[n]));
        } else {
          acc = fmaf(L, bj, fmaf(a, lm, acc));
        }
      }
    }
    // FP32 form with 16-byte aligned rows: 4 consecutive neurons per lane (float4 A, bias and
    // Lambda, uchar4 codes); a group of stable, unsplit neurons needs no other load
    const bool vec4 = WPR > 1 && !CERT && ((d | (int)(n0 & 3)) & 3) == 0 &&
                      ((reinterpret_cast<uintptr_t>(a_row) | reinterpret_cast<uintptr_t>(lam_row) |
                        reinterpret_cast<uintptr_t>(bias)) & 15) == 0;
    if (vec4) {
      const uchar4* code4 = reinterpret_cast<const uchar4*>(c.tb.code + n0);
      // the row's alpha block, checked once against the array
      const float* alpha_row = (abase >= 0 && abase + Up <= n_alpha) ? alpha + abase : nullptr;
      if (!alpha_row && Up > 0 && lane == 0 && sub == 0) flag(c.status, BCROWN_ERR_ARG);
      for (int q = sub * 32 + lane; q < d / 4; q += 32 * WPR) {
        const int j = 4 * q;
        const float4 a4 = reinterpret_cast<const float4*>(a_row)[q];
        const float4 b4 = reinterpret_cast<const float4*>(bias)[q];
        const uchar4 c4 = code4[q];
        const uint32_t sb = ns == 0 ? 0u : (use_mask ? (smask[rs][j >> 5] >> (j & 31)) & 0xFu : 0xFu);
        float4 L;
        if (sb == 0u && stable4(c4)) {
          L.x = fmaf(a4.x, d01(c4.x), 0.f);
          L.y = fmaf(a4.y, d01(c4.y), 0.f);
          L.z = fmaf(a4.z, d01(c4.z), 0.f);
          L.w = fmaf(a4.w, d01(c4.w), 0.f);
          acc = fmaf(L.x, b4.x, fmaf(a4.x, 0.f, acc));
          acc = fmaf(L.y, b4.y, fmaf(a4.y, 0.f, acc));
          acc = fmaf(L.z, b4.z, fmaf(a4.z, 0.f, acc));
          acc = fmaf(L.w, b4.w, fmaf(a4.w, 0.f, acc));
        } else {
          const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
          float D[4], lm[4], Lv[4];
          int rk[4];
          group4(c.tb, n0 + j, av, c4, alpha_row, D, lm, rk);
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            float bs = 0.f;
            if ((sb >> v) & 1u)   // a split of the row may sit here
              for (int qq = 0; qq < ns; ++qq)
                if (sl_[qq].idx == j + v) {
                  const long long bi = bbase + sl_[qq].t;
                  if (bi >= 0 && bi < n_beta) bs = fmaxf(beta[bi], 0.f) * (float)sl_[qq].sign;
                  else flag(c.status, BCROWN_ERR_ARG);
                  D[v] = sl_[qq].sign == -1 ? 1.f : 0.f;
                  lm[v] = 0.f;
                }
            Lv[v] = fmaf(av[v], D[v], bs);
            acc = fmaf(Lv[v], bv[v], fmaf(av[v], lm[v], acc));
          }
          L = make_float4(Lv[0], Lv[1], Lv[2], Lv[3]);
        }
        reinterpret_cast<float4*>(lam_row)[q] = L;
      }
    }
    // RELAX_V neurons per lane per step, their loads issued in three rounds (A, code, bias; then
    // the unstable neurons' rank and chord; then alpha) instead of one dependent chain each
    constexpr int RELAX_V = 4;
    for (int j0 = sub * 32 + lane; WPR > 1 && !vec4 && j0 < d; j0 += RELAX_V * 32 * WPR) {
      float av[RELAX_V], bv[RELAX_V], sl[RELAX_V], ic[RELAX_V], al[RELAX_V];
      uint8_t cv[RELAX_V];
      int32_t rk[RELAX_V];
#pragma unroll
      for (int v = 0; v < RELAX_V; ++v) {
        const int j = j0 + v * 32 * WPR;
        const bool in = j < d;
        av[v] = ld_f32(a_row + j, in);
        bv[v] = ld_f32(bias + j, in);
        cv[v] = (uint8_t)ld_u8(c.tb.code + n0 + j, in, CODE_INACTIVE);
      }
#pragma unroll
      for (int v = 0; v < RELAX_V; ++v) {
        const int j = j0 + v * 32 * WPR;
        const bool un = cv[v] == CODE_UNSTABLE;
        rk[v] = ld_s32(c.tb.rank + n0 + j, un && av[v] >= 0.f);
        sl[v] = ld_f32(c.tb.slope + n0 + j, un && av[v] < 0.f);
        ic[v] = ld_f32(c.tb.icpt + n0 + j, un && av[v] < 0.f);
      }
#pragma unroll
      for (int v = 0; v < RELAX_V; ++v) {
        al[v] = 0.f;
        if (cv[v] == CODE_UNSTABLE && av[v] >= 0.f) {
          const long long ai = abase + rk[v];
          if (ai < 0 || ai >= n_alpha) flag(c.status, BCROWN_ERR_ARG);
          else al[v] = fminf(fmaxf(alpha[ai], 0.f), 1.f);
        }
      }
#pragma unroll
      for (int v = 0; v < RELAX_V; ++v) {
        const int j = j0 + v * 32 * WPR;
        if (j >= d) break;
        const float a = av[v];
        const size_t n = n0 + j;
        int s = 0;
        float bet = 0.f;
        if (ns > 0 && (!use_mask || split_bit(smask[rs], j)))
          for (int q = 0; q < ns; ++q)
            if (sl_[q].idx == j) {
              s = sl_[q].sign;
              const long long bi = bbase + sl_[q].t;
              if (bi >= 0 && bi < n_beta) bet = fmaxf(beta[bi], 0.f);
              else flag(c.status, BCROWN_ERR_ARG);
            }
        float D = 0.f, lm = 0.f;
        const uint8_t code = cv[v];
        if (s == -1) D = 1.f;
        else if (s == 1) D = 0.f;
        else if (code == CODE_ACTIVE) D = 1.f;
        else if (code == CODE_INACTIVE) D = 0.f;
        else if (a >= 0.f) D = al[v];
        else {
          // upper chord, slope and intercept rounded up (outward) in the tables
          D = sl[v];
          lm = ic[v];
        }
        const float L = fmaf(a, D, bet * (float)s);
        lam_row[j] = L;
        const float bj = bv[v];
        if (CERT) {
          acc = __fadd_rd(acc, __fadd_rd(__fmul_rd(L, bj), __fmul_rd(a, lm)));
          const bool exact = (s == 0) && (D == 0.f || D == 1.f);
          if (!exact) {
            // Lambda_j was rounded once: |error| <= 2^-23 |Lambda_j| (+ an underflow margin),
            // acting on |z_j| <= max(|l_j|, |u_j|)
            const float zmax = fmaxf(fabsf(c.l[n]), fabsf(c.u[n]));
            const float er = __fmaf_ru(fabsf(L), 0x1p-23f, 0x1p-140f);
            e1 = __fadd_ru(e1, __fmul_ru(er, zmax));
          }
          e2 = __fadd_ru(e2, __fmul_ru(fabsf(L), wm[n]));
        } else {
          acc = fmaf(L, bj, fmaf(a, lm, acc));
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      if (CERT) {
        acc = __fadd_rd(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        e1 = __fadd_ru(e1, __shfl_xor_sync(0xffffffffu, e1, o));
        e2 = __fadd_ru(e2, __shfl_xor_sync(0xffffffffu, e2, o));
      } else {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
      }
    }
  }
  if (WPR > 1) {
    // the row's warps combine their sums (same rounding directions)
    if (lane == 0) {
      red[w][0] = acc;
      red[w][1] = e1;
      red[w][2] = e2;
    }
    __syncthreads();
    if (live && sub == 0 && lane == 0)
      for (int q = 1; q < WPR; ++q) {
        if (CERT) {
          acc = __fadd_rd(acc, red[w + q][0]);
          e1 = __fadd_ru(e1, red[w + q][1]);
          e2 = __fadd_ru(e2, red[w + q][2]);
        } else {
          acc += red[w + q][0];
        }
      }
  }
  if (live && sub == 0 && lane == 0) {
    if (CERT) {
      cd[rl] = __dadd_rd(cd[rl], (double)acc);
      E[rl] = __dadd_ru(E[rl], __dadd_ru((double)e1, __dmul_ru(gamma, (double)e2)));
    } else {
      cf[rl] += acc;
    }
  }
}

// ----------------------------------------------------------------------------------------
// FP32 SIMT GEMM  C[M,N] = A[M,K] * B[K,N] (+ bias[N]); row-major, any shape.
// Each output is a sequential FMA chain over k (error <= gamma_K sum |a b|).
// ----------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                               const float* __restrict__ B, int ldb, float* __restrict__ C,
                                               int ldc, const float* __restrict__ bias) {
  constexpr int BM = 128, BN = 128, BK = 16;
  constexpr int LPT = BM * BK / 256;   // elements of each operand a thread stages per k step
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  // thread (tx, ty): rows 4ty..4ty+3 and 64+4ty..64+4ty+3, columns 4tx.. and 64+4tx.. of the
  // tile, so its shared-memory operands are two 16-byte loads per matrix per k
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float ra[LPT], rb[LPT];
  auto load_regs = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
      int e = tid + q * 256;
      int m = e / BK, kk = e % BK;
      int gm = m0 + m, gk = k0 + kk;
      ra[q] = (gm < M && gk < K) ? A[(size_t)gm * lda + gk] : 0.f;
      int kb = e / BN, n = e % BN;
      int gk2 = k0 + kb, gn = n0 + n;
      rb[q] = (gk2 < K && gn < N) ? B[(size_t)gk2 * ldb + gn] : 0.f;
    }
  };
  auto store_smem = [&](int buf) {
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
      int e = tid + q * 256;
      As[buf][e % BK][e / BK] = ra[q];
      Bs[buf][e / BN][e % BN] = rb[q];
    }
  };
  int nk = (K + BK - 1) / BK;
  load_regs(0);
  store_smem(0);
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    int buf = t & 1;
    if (t + 1 < nk) load_regs((t + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + 4 * ty]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * tx]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + 4 * tx]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (t + 1 < nk) store_smem(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int gm = m0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int gn = n0 + (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
      if (gn < N) C[(size_t)gm * ldc + gn] = acc[i][j] + (bias ? bias[gn] : 0.f);
    }
  }
}

// Convolutions, both directions, register-blocked: a thread owns one spatial position of one
// row and CB = 16 channels of the result; the weights of a slice of the summed channels are
// staged in shared memory as [channel][tap][CB result channels] (16-byte reads),
// the operand is read once per (channel, tap) and feeds CB FMAs.  Every output is still one
// sequential FMA chain over its terms (taps outer, channels inner), which the certifying pass's
// a priori error bound assumes.
constexpr int CONV_CB = 16;         // result channels per thread (multiple of 4)
constexpr int CONV_POS = 128;       // positions per block (threads)
constexpr int CONV_SMEM_FLOATS = 8192;   // 32 KB of staged weights per slice

// Backward (transposed convolution):
//   Ain[r, ci, iy, ix] = sum_{co, ky, kx: iy = oy*s - p + ky, ix = ox*s - p + kx} Lam[r, co, oy, ox] W[co, ci, ky, kx]
// grid: (position tiles, channel groups of CB, rows).
__global__ void __launch_bounds__(CONV_POS) k_conv_bwd(int R, LayerGeom g, const float* __restrict__ Lam,
                                                       const float* __restrict__ W, float* __restrict__ Ain) {
  __shared__ __align__(16) float Ws[CONV_SMEM_FLOATS];
  const int kk = g.k * g.k;
  const int r = blockIdx.z;
  const int ci0 = blockIdx.y * CONV_CB;
  const int hw_in = g.in_h * g.in_w, hw_out = g.out_h * g.out_w;
  const int pos = blockIdx.x * CONV_POS + threadIdx.x;
  const bool pin = pos < hw_in;
  const int iy = pin ? pos / g.in_w : 0, ix = pin ? pos - (pos / g.in_w) * g.in_w : 0;
  const float* lr = Lam + (size_t)r * g.d_out;
  float acc[CONV_CB];
#pragma unroll
  for (int c = 0; c < CONV_CB; ++c) acc[c] = 0.f;
  const int coch = max(1, CONV_SMEM_FLOATS / (kk * CONV_CB));   // output channels per slice
  for (int co0 = 0; co0 < g.out_c; co0 += coch) {
    const int nco = min(coch, g.out_c - co0);
    __syncthreads();
    for (int e = threadIdx.x; e < nco * kk * CONV_CB; e += CONV_POS) {
      const int c = e % CONV_CB, t = (e / CONV_CB) % kk, col = e / (CONV_CB * kk);
      const int ci = ci0 + c;
      Ws[e] = ci < g.in_c ? W[((size_t)(co0 + col) * g.in_c + ci) * kk + t] : 0.f;
    }
    __syncthreads();
    if (pin) {
      for (int ky = 0; ky < g.k; ++ky) {
        const int ty = iy + g.pad - ky;
        if (ty < 0 || ty % g.stride) continue;
        const int oy = ty / g.stride;
        if (oy >= g.out_h) continue;
        for (int kx = 0; kx < g.k; ++kx) {
          const int tx = ix + g.pad - kx;
          if (tx < 0 || tx % g.stride) continue;
          const int ox = tx / g.stride;
          if (ox >= g.out_w) continue;
          const float* lp = lr + (size_t)co0 * hw_out + (size_t)oy * g.out_w + ox;
          const float* wp = Ws + (ky * g.k + kx) * CONV_CB;
          for (int col = 0; col < nco; ++col) {
            const float v = lp[(size_t)col * hw_out];
#pragma unroll
            for (int q4 = 0; q4 < CONV_CB / 4; ++q4) {
              const float4 w = *reinterpret_cast<const float4*>(wp + (size_t)col * kk * CONV_CB + 4 * q4);
              acc[4 * q4 + 0] = fmaf(v, w.x, acc[4 * q4 + 0]);
              acc[4 * q4 + 1] = fmaf(v, w.y, acc[4 * q4 + 1]);
              acc[4 * q4 + 2] = fmaf(v, w.z, acc[4 * q4 + 2]);
              acc[4 * q4 + 3] = fmaf(v, w.w, acc[4 * q4 + 3]);
            }
          }
        }
      }
    }
  }
  if (pin) {
    float* ar = Ain + (size_t)r * g.d_in + pos;
#pragma unroll
    for (int c = 0; c < CONV_CB; ++c)
      if (ci0 + c < g.in_c) ar[(size_t)(ci0 + c) * hw_in] = acc[c];
  }
}

// Forward convolution (adjoint pass):
//   Z[r, co, oy, ox] = b[co] + sum_{ci, ky, kx} W[co, ci, ky, kx] h[r, ci, oy*s - p + ky, ox*s - p + kx]
// grid: (position tiles, channel groups of CB, rows).
__global__ void __launch_bounds__(CONV_POS) k_conv_fwd(int R, LayerGeom g, const float* __restrict__ h,
                                                       const float* __restrict__ W, const float* __restrict__ bias,
                                                       float* __restrict__ Z) {
  __shared__ __align__(16) float Ws[CONV_SMEM_FLOATS];
  const int kk = g.k * g.k;
  const int r = blockIdx.z;
  const int co0 = blockIdx.y * CONV_CB;
  const int hw_in = g.in_h * g.in_w, hw_out = g.out_h * g.out_w;
  const int pos = blockIdx.x * CONV_POS + threadIdx.x;
  const bool pin = pos < hw_out;
  const int oy = pin ? pos / g.out_w : 0, ox = pin ? pos - (pos / g.out_w) * g.out_w : 0;
  const float* hr = h + (size_t)r * g.d_in;
  float acc[CONV_CB];
#pragma unroll
  for (int c = 0; c < CONV_CB; ++c) acc[c] = 0.f;
  const int cich = max(1, CONV_SMEM_FLOATS / (kk * CONV_CB));   // input channels per slice
  for (int ci0 = 0; ci0 < g.in_c; ci0 += cich) {
    const int nci = min(cich, g.in_c - ci0);
    __syncthreads();
    for (int e = threadIdx.x; e < nci * kk * CONV_CB; e += CONV_POS) {
      const int c = e % CONV_CB, t = (e / CONV_CB) % kk, cl = e / (CONV_CB * kk);
      const int co = co0 + c;
      Ws[e] = co < g.out_c ? W[((size_t)co * g.in_c + ci0 + cl) * kk + t] : 0.f;
    }
    __syncthreads();
    if (pin) {
      for (int ky = 0; ky < g.k; ++ky) {
        const int iy = oy * g.stride - g.pad + ky;
        if (iy < 0 || iy >= g.in_h) continue;
        for (int kx = 0; kx < g.k; ++kx) {
          const int ix = ox * g.stride - g.pad + kx;
          if (ix < 0 || ix >= g.in_w) continue;
          const float* hp = hr + (size_t)ci0 * hw_in + (size_t)iy * g.in_w + ix;
          const float* wp = Ws + (ky * g.k + kx) * CONV_CB;
          for (int cl = 0; cl < nci; ++cl) {
            const float v = hp[(size_t)cl * hw_in];
#pragma unroll
            for (int q4 = 0; q4 < CONV_CB / 4; ++q4) {
              const float4 w = *reinterpret_cast<const float4*>(wp + (size_t)cl * kk * CONV_CB + 4 * q4);
              acc[4 * q4 + 0] = fmaf(w.x, v, acc[4 * q4 + 0]);
              acc[4 * q4 + 1] = fmaf(w.y, v, acc[4 * q4 + 1]);
              acc[4 * q4 + 2] = fmaf(w.z, v, acc[4 * q4 + 2]);
              acc[4 * q4 + 3] = fmaf(w.w, v, acc[4 * q4 + 3]);
            }
          }
        }
      }
    }
  }
  if (pin) {
    float* zr = Z + (size_t)r * g.d_out + pos;
#pragma unroll
    for (int c = 0; c < CONV_CB; ++c)
      if (co0 + c < g.out_c) zr[(size_t)(co0 + c) * hw_out] = acc[c] + bias[(size_t)(co0 + c) * hw_out + pos];
  }
}

// ----------------------------------------------------------------------------------------
// Concretisation over the box (Eq. beta_crown_lp, Hoelder for an L-infinity box):
//   lb = c + sum_m min(A_m x_lo_m, A_m x_hi_m)
// ----------------------------------------------------------------------------------------
template <bool CERT>
__global__ void __launch_bounds__(256) k_concretize(RowsCtx c, int d0, const float* __restrict__ A0,
                                                    const float* __restrict__ cf, const double* __restrict__ cd,
                                                    const double* __restrict__ E, float* __restrict__ lb) {
  __shared__ float shf[32];
  int rl = blockIdx.x;
  int b, k, p;
  if (!row_prop(c, rl, &b, &k, &p)) p = 0;
  const float* a = A0 + (size_t)rl * d0;
  const float* xl = c.x_lo + (size_t)p * d0;
  const float* xh = c.x_hi + (size_t)p * d0;
  float s = 0.f;
  for (int m = threadIdx.x; m < d0; m += blockDim.x) {
    float am = a[m];
    if (CERT) {
      // products rounded down, then summed rounded down: a lower bound of sum_m min(...)
      s = __fadd_rd(s, fminf(__fmul_rd(am, xl[m]), __fmul_rd(am, xh[m])));
    } else {
      s += fminf(am * xl[m], am * xh[m]);
    }
  }
  float out;
  if (CERT) {
    s = block_fsum<1>(s, shf);
    out = __double2float_rd(__dsub_rd(__dadd_rd(cd[rl], (double)s), E[rl]));
  } else {
    s = block_sum(s, shf);
    out = cf[rl] + s;
  }
  if (threadIdx.x == 0) {
    if (!isfinite(out)) {
      flag(c.status, BCROWN_ERR_NONFINITE);
      out = -INFINITY;
    }
    lb[c.r0 + rl] = out;
  }
}

// x*: the box corner minimising A^(0) x (x_lo where A^(0)_m >= 0)
__global__ void k_xstar(RowsCtx c, int d0, const float* __restrict__ A0, float* __restrict__ h0) {
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)c.R * d0) return;
  int rl = (int)(id / d0);
  int m = (int)(id - (long long)rl * d0);
  int b, k, p;
  if (!row_prop(c, rl, &b, &k, &p)) p = 0;
  h0[id] = A0[id] >= 0.f ? c.x_lo[(size_t)p * d0 + m] : c.x_hi[(size_t)p * d0 + m];
}

// ----------------------------------------------------------------------------------------
// Adjoint epilogue of hidden layer i: zhat = Z (+ bias already added); gradients
//   dalpha_j = A_j zhat_j (alpha in use), dbeta_j = S_jj zhat_j ; then h = D zhat + lambda.
// ----------------------------------------------------------------------------------------
// WIDE: rows of more than 2048 neurons (conv layers); the narrow instantiation keeps only the
// simple loop, and with it the register count of that loop.
template <bool WIDE>
__global__ void __launch_bounds__(256) k_fwd_epi(RowsCtx c, int layer, int d, long long hoff,
                                                 float* __restrict__ Z, const float* __restrict__ Ai,
                                                 const float* __restrict__ alpha, int64_t n_alpha,
                                                 float* __restrict__ dalpha, float* __restrict__ dbeta,
                                                 int64_t n_beta) {
  __shared__ SplitSlot slots[BCROWN_MAX_SPLITS];
  __shared__ int n_slots;
  int rl = blockIdx.x;
  int b, k, p;
  if (!row_prop(c, rl, &b, &k, &p)) p = 0;
  int ns = stage_splits(c, b, layer, d, slots, &n_slots);
  extern __shared__ uint32_t smask[];   // ceil(d / 32) words for wide rows (the launch sizes it)
  const bool use_mask = WIDE && ns > 0 && d <= SPLIT_MASK_WORDS * 32;
  if (use_mask) split_mask_block(slots, ns, d, smask);   // ns is uniform over the block
  int cnt = c.bt.split_cnt[b];
  int Up = c.tb.U[p];
  long long abase = c.bt.alpha_off[b] + (long long)k * Up;
  long long bbase = (long long)c.bt.split_off[b] * c.K + (long long)k * cnt;
  float* z_row = Z + (size_t)rl * d;
  const float* a_row = Ai + (size_t)rl * d;
  const size_t n0 = (size_t)p * c.tb.H + hoff;
  if constexpr (!WIDE) {
    // narrow rows: one neuron per thread, the split list scanned per neuron (measured faster
    // there than the wide-row code below)
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
      float z = z_row[j];
      float a = a_row[j];
      size_t n = (size_t)p * c.tb.H + hoff + j;
      int s = 0, t = -1;
      for (int q = 0; q < ns; ++q)
        if (slots[q].idx == j) {
          s = slots[q].sign;
          t = slots[q].t;
        }
      uint8_t code = c.tb.code[n];
      float D = 0.f, lm = 0.f;
      long long ai = -1;
      if (code == CODE_UNSTABLE) {
        ai = abase + c.tb.rank[n];
        if (ai < 0 || ai >= n_alpha) {
          flag(c.status, BCROWN_ERR_ARG);
          ai = -1;
        }
      }
      if (s == -1) D = 1.f;
      else if (s == 1) D = 0.f;
      else if (code == CODE_ACTIVE) D = 1.f;
      else if (code == CODE_INACTIVE) D = 0.f;
      else if (a >= 0.f) D = ai >= 0 ? fminf(fmaxf(alpha[ai], 0.f), 1.f) : 0.f;
      else {
        D = c.tb.slope[n];
        lm = c.tb.icpt[n];
      }
      if (ai >= 0) dalpha[ai] = (s == 0 && a >= 0.f) ? a * z : 0.f;
      if (s != 0) {
        long long bi = bbase + t;
        if (bi >= 0 && bi < n_beta) dbeta[bi] = (float)s * z;
        else flag(c.status, BCROWN_ERR_ARG);
      }
      z_row[j] = fmaf(D, z, lm);
    }
  } else {
  // 16-byte aligned rows: 4 consecutive neurons per thread (float4 zhat and A, uchar4 codes); a
  // group of stable, unsplit neurons writes h = D zhat and nothing else
  const bool vec4 = ((d | (int)(n0 & 3)) & 3) == 0 &&
                    ((reinterpret_cast<uintptr_t>(z_row) | reinterpret_cast<uintptr_t>(a_row)) & 15) == 0;
  if (vec4) {
    const uchar4* code4 = reinterpret_cast<const uchar4*>(c.tb.code + n0);
    // the row's alpha and dalpha blocks, checked once against the arrays
    const bool arow_ok = abase >= 0 && abase + Up <= n_alpha;
    const float* alpha_row = arow_ok ? alpha + abase : nullptr;
    float* dalpha_row = arow_ok ? dalpha + abase : nullptr;
    if (!arow_ok && Up > 0 && threadIdx.x == 0) flag(c.status, BCROWN_ERR_ARG);
    for (int q = threadIdx.x; q < d / 4; q += blockDim.x) {
      const int j = 4 * q;
      const float4 z4 = reinterpret_cast<const float4*>(z_row)[q];
      const float4 a4 = reinterpret_cast<const float4*>(a_row)[q];
      const uchar4 c4 = code4[q];
      const uint32_t sb = ns == 0 ? 0u : (use_mask ? (smask[j >> 5] >> (j & 31)) & 0xFu : 0xFu);
      if (sb == 0u && stable4(c4)) {
        const float4 h4 = make_float4(fmaf(d01(c4.x), z4.x, 0.f), fmaf(d01(c4.y), z4.y, 0.f),
                                      fmaf(d01(c4.z), z4.z, 0.f), fmaf(d01(c4.w), z4.w, 0.f));
        reinterpret_cast<float4*>(z_row)[q] = h4;
        continue;
      }
      const float zv[4] = {z4.x, z4.y, z4.z, z4.w}, av[4] = {a4.x, a4.y, a4.z, a4.w};
      float D[4], lm[4], hv[4];
      int rk[4];
      group4(c.tb, n0 + j, av, c4, alpha_row, D, lm, rk);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        int s = 0;
        if ((sb >> v) & 1u) {   // a split of the row may sit here
          int t = -1;
          for (int qq = 0; qq < ns; ++qq)
            if (slots[qq].idx == j + v) {
              s = slots[qq].sign;
              t = slots[qq].t;
            }
          if (s != 0) {
            D[v] = s == -1 ? 1.f : 0.f;
            lm[v] = 0.f;
            const long long bi = bbase + t;
            if (bi >= 0 && bi < n_beta) dbeta[bi] = (float)s * zv[v];
            else flag(c.status, BCROWN_ERR_ARG);
          }
        }
        if (rk[v] >= 0 && dalpha_row) dalpha_row[rk[v]] = (s == 0 && av[v] >= 0.f) ? av[v] * zv[v] : 0.f;
        hv[v] = fmaf(D[v], zv[v], lm[v]);
      }
      reinterpret_cast<float4*>(z_row)[q] = make_float4(hv[0], hv[1], hv[2], hv[3]);
    }
    return;
  }
  // EPI_V neurons per thread per step, their loads issued in three rounds (z, A, code; then the
  // unstable neurons' rank and chord; then alpha) instead of one dependent chain per neuron
  constexpr int EPI_V = 4;
  for (int j0 = threadIdx.x; j0 < d; j0 += EPI_V * blockDim.x) {
    float z[EPI_V], a[EPI_V], sl[EPI_V], ic[EPI_V], al[EPI_V];
    uint8_t code[EPI_V];
    int32_t rk[EPI_V];
#pragma unroll
    for (int v = 0; v < EPI_V; ++v) {
      const int j = j0 + v * blockDim.x;
      const bool in = j < d;
      z[v] = ld_f32(z_row + j, in);
      a[v] = ld_f32(a_row + j, in);
      code[v] = (uint8_t)ld_u8(c.tb.code + n0 + j, in, CODE_INACTIVE);
    }
#pragma unroll
    for (int v = 0; v < EPI_V; ++v) {
      const int j = j0 + v * blockDim.x;
      const bool un = code[v] == CODE_UNSTABLE;
      rk[v] = un ? ld_s32(c.tb.rank + n0 + j, true) : -1;
      sl[v] = ld_f32(c.tb.slope + n0 + j, un && a[v] < 0.f);
      ic[v] = ld_f32(c.tb.icpt + n0 + j, un && a[v] < 0.f);
    }
    long long ai[EPI_V];
#pragma unroll
    for (int v = 0; v < EPI_V; ++v) {
      ai[v] = -1;
      al[v] = 0.f;
      if (code[v] == CODE_UNSTABLE) {
        ai[v] = abase + rk[v];
        if (ai[v] < 0 || ai[v] >= n_alpha) {
          flag(c.status, BCROWN_ERR_ARG);
          ai[v] = -1;
        } else if (a[v] >= 0.f) {
          al[v] = alpha[ai[v]];
        }
      }
    }
#pragma unroll
    for (int v = 0; v < EPI_V; ++v) {
      const int j = j0 + v * blockDim.x;
      if (j >= d) break;
      int s = 0, t = -1;
      if (ns > 0 && (!use_mask || split_bit(smask, j)))
        for (int q = 0; q < ns; ++q)
          if (slots[q].idx == j) {
            s = slots[q].sign;
            t = slots[q].t;
          }
      float D = 0.f, lm = 0.f;
      if (s == -1) D = 1.f;
      else if (s == 1) D = 0.f;
      else if (code[v] == CODE_ACTIVE) D = 1.f;
      else if (code[v] == CODE_INACTIVE) D = 0.f;
      else if (a[v] >= 0.f) D = ai[v] >= 0 ? fminf(fmaxf(al[v], 0.f), 1.f) : 0.f;
      else {
        D = sl[v];
        lm = ic[v];
      }
      if (ai[v] >= 0) dalpha[ai[v]] = (s == 0 && a[v] >= 0.f) ? a[v] * z[v] : 0.f;
      if (s != 0) {
        long long bi = bbase + t;
        if (bi >= 0 && bi < n_beta) dbeta[bi] = (float)s * z[v];
        else flag(c.status, BCROWN_ERR_ARG);
      }
      z_row[j] = fmaf(D, z[v], lm);
    }
  }
  }
}

// ----------------------------------------------------------------------------------------
// Projected Adam ascent with best-row tracking (Eq. opt_alpha_beta; Appendix C.1).
// One block per row; the row's alpha block and beta block.
// ----------------------------------------------------------------------------------------
// One projected Adam step of one alpha (projection onto [0, 1]); ib1, ib2 are the reciprocals
// of the bias corrections, so an element costs one square root and one (fast) division.
__device__ __forceinline__ float adam_alpha(float th, float g, float& m, float& v, float lr, float beta1, float beta2,
                                            float eps, float ib1, float ib2) {
  m = beta1 * m + (1.f - beta1) * g;
  v = beta2 * v + (1.f - beta2) * g * g;
  th += __fdividef(lr * (m * ib1), sqrtf(v * ib2) + eps);
  return __saturatef(th);
}

// One warp per row: the row's alphas in 16-byte accesses where the arrays allow it.
constexpr int ADAM_ROWS_PER_BLOCK = 8;
__global__ void __launch_bounds__(32 * ADAM_ROWS_PER_BLOCK) k_adam(
    int R, int K, BatchView bt, const int32_t* __restrict__ U, int P, const float* __restrict__ lb_t,
    float* __restrict__ best_lb, float* __restrict__ a_cur, float* __restrict__ a_best,
    const float* __restrict__ ga, float* __restrict__ ma, float* __restrict__ va, float* __restrict__ b_cur,
    float* __restrict__ b_best, const float* __restrict__ gb, float* __restrict__ mb, float* __restrict__ vb,
    float lr_a, float lr_b, float beta1, float beta2, float eps, float bc1, float bc2, int64_t n_alpha,
    int64_t n_beta) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * ADAM_ROWS_PER_BLOCK + (threadIdx.x >> 5);
  if (r >= R) return;
  const int b = r / K, k = r - b * K;
  const int p = bt.prop_of[b];
  if (p < 0 || p >= P) return;
  const float cur = lb_t[r];
  const bool improved = cur > best_lb[r];
  const float ib1 = 1.f / bc1, ib2 = 1.f / bc2;
  const int Up = U[p];
  const long long abase = bt.alpha_off[b] + (long long)k * Up;
  // the row's alphas that lie in the array
  const long long aend = abase < 0 ? abase : min(abase + (long long)Up, (long long)n_alpha);
  auto one = [&](long long i) {
    const float th = a_cur[i];
    if (improved) a_best[i] = th;
    float m = ma[i], v = va[i];
    a_cur[i] = adam_alpha(th, ga[i], m, v, lr_a, beta1, beta2, eps, ib1, ib2);
    ma[i] = m;
    va[i] = v;
  };
  const bool vec = ((reinterpret_cast<uintptr_t>(a_cur) | reinterpret_cast<uintptr_t>(a_best) |
                     reinterpret_cast<uintptr_t>(ga) | reinterpret_cast<uintptr_t>(ma) |
                     reinterpret_cast<uintptr_t>(va)) & 15u) == 0;
  long long v0 = aend, v1 = aend;   // [v0, v1): 4-aligned body updated with 16-byte accesses
  if (vec && aend > abase) {
    v0 = min(aend, (abase + 3) & ~3LL);
    v1 = v0 + ((aend - v0) & ~3LL);
  }
  for (long long i = abase + lane; i < v0; i += 32) one(i);
  for (long long i = v1 + lane; i < aend; i += 32) one(i);
#pragma unroll 2
  for (long long i = v0 + 4 * lane; i < v1; i += 128) {
    const float4 th = *reinterpret_cast<const float4*>(a_cur + i);
    const float4 g = *reinterpret_cast<const float4*>(ga + i);
    float4 m = *reinterpret_cast<const float4*>(ma + i);
    float4 v = *reinterpret_cast<const float4*>(va + i);
    if (improved) *reinterpret_cast<float4*>(a_best + i) = th;
    float4 o;
    o.x = adam_alpha(th.x, g.x, m.x, v.x, lr_a, beta1, beta2, eps, ib1, ib2);
    o.y = adam_alpha(th.y, g.y, m.y, v.y, lr_a, beta1, beta2, eps, ib1, ib2);
    o.z = adam_alpha(th.z, g.z, m.z, v.z, lr_a, beta1, beta2, eps, ib1, ib2);
    o.w = adam_alpha(th.w, g.w, m.w, v.w, lr_a, beta1, beta2, eps, ib1, ib2);
    *reinterpret_cast<float4*>(a_cur + i) = o;
    *reinterpret_cast<float4*>(ma + i) = m;
    *reinterpret_cast<float4*>(va + i) = v;
  }
  const int cnt = bt.split_cnt[b];
  const long long bbase = (long long)bt.split_off[b] * K + (long long)k * cnt;
  for (int t = lane; t < cnt; t += 32) {
    const long long i = bbase + t;
    if (i < 0 || i >= n_beta) break;
    float th = b_cur[i];
    if (improved) b_best[i] = th;
    float g = gb[i];
    float m = beta1 * mb[i] + (1.f - beta1) * g;
    float v = beta2 * vb[i] + (1.f - beta2) * g * g;
    mb[i] = m;
    vb[i] = v;
    th += lr_b * (m / bc1) / (sqrtf(v / bc2) + eps);
    b_cur[i] = fmaxf(th, 0.f);
  }
  __syncwarp();
  if (lane == 0 && improved) best_lb[r] = cur;
}

// The same step with the gradient and both moments of alpha held in BF16 (the BF16 path's
// optimiser state): 22 instead of 32 bytes moved per alpha.  The moments are rounded to BF16
// after each update; beta's state stays FP32.
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
__device__ __forceinline__ uint32_t bf16_pack(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__global__ void __launch_bounds__(32 * ADAM_ROWS_PER_BLOCK) k_adam16(
    int R, int K, BatchView bt, const int32_t* __restrict__ U, int P, const float* __restrict__ lb_t,
    float* __restrict__ best_lb, float* __restrict__ a_cur, float* __restrict__ a_best,
    const __nv_bfloat16* __restrict__ ga, __nv_bfloat16* __restrict__ ma, __nv_bfloat16* __restrict__ va,
    float* __restrict__ b_cur, float* __restrict__ b_best, const float* __restrict__ gb, float* __restrict__ mb,
    float* __restrict__ vb, float lr_a, float lr_b, float beta1, float beta2, float eps, float bc1, float bc2,
    int64_t n_alpha, int64_t n_beta) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * ADAM_ROWS_PER_BLOCK + (threadIdx.x >> 5);
  if (r >= R) return;
  const int b = r / K, k = r - b * K;
  const int p = bt.prop_of[b];
  if (p < 0 || p >= P) return;
  const float cur = lb_t[r];
  const bool improved = cur > best_lb[r];
  const float ib1 = 1.f / bc1, ib2 = 1.f / bc2;
  const int Up = U[p];
  const long long abase = bt.alpha_off[b] + (long long)k * Up;
  const long long aend = abase < 0 ? abase : min(abase + (long long)Up, (long long)n_alpha);
  auto one = [&](long long i) {
    const float th = a_cur[i];
    if (improved) a_best[i] = th;
    float m = __bfloat162float(ma[i]), v = __bfloat162float(va[i]);
    a_cur[i] = adam_alpha(th, __bfloat162float(ga[i]), m, v, lr_a, beta1, beta2, eps, ib1, ib2);
    ma[i] = __float2bfloat16_rn(m);
    va[i] = __float2bfloat16_rn(v);
  };
  // 4-aligned body: 16-byte alpha accesses, 8-byte BF16 accesses
  const bool vec = ((reinterpret_cast<uintptr_t>(a_cur) | reinterpret_cast<uintptr_t>(a_best)) & 15u) == 0 &&
                   ((reinterpret_cast<uintptr_t>(ga) | reinterpret_cast<uintptr_t>(ma) |
                     reinterpret_cast<uintptr_t>(va)) & 7u) == 0;
  long long v0 = aend, v1 = aend;
  if (vec && aend > abase) {
    v0 = min(aend, (abase + 3) & ~3LL);
    v1 = v0 + ((aend - v0) & ~3LL);
  }
  for (long long i = abase + lane; i < v0; i += 32) one(i);
  for (long long i = v1 + lane; i < aend; i += 32) one(i);
#pragma unroll 2
  for (long long i = v0 + 4 * lane; i < v1; i += 128) {
    const float4 th = *reinterpret_cast<const float4*>(a_cur + i);
    const uint2 g2 = *reinterpret_cast<const uint2*>(ga + i);
    const uint2 m2 = *reinterpret_cast<const uint2*>(ma + i);
    const uint2 w2 = *reinterpret_cast<const uint2*>(va + i);
    if (improved) *reinterpret_cast<float4*>(a_best + i) = th;
    float m[4] = {bf16_lo(m2.x), bf16_hi(m2.x), bf16_lo(m2.y), bf16_hi(m2.y)};
    float v[4] = {bf16_lo(w2.x), bf16_hi(w2.x), bf16_lo(w2.y), bf16_hi(w2.y)};
    const float g[4] = {bf16_lo(g2.x), bf16_hi(g2.x), bf16_lo(g2.y), bf16_hi(g2.y)};
    float4 o;
    o.x = adam_alpha(th.x, g[0], m[0], v[0], lr_a, beta1, beta2, eps, ib1, ib2);
    o.y = adam_alpha(th.y, g[1], m[1], v[1], lr_a, beta1, beta2, eps, ib1, ib2);
    o.z = adam_alpha(th.z, g[2], m[2], v[2], lr_a, beta1, beta2, eps, ib1, ib2);
    o.w = adam_alpha(th.w, g[3], m[3], v[3], lr_a, beta1, beta2, eps, ib1, ib2);
    *reinterpret_cast<float4*>(a_cur + i) = o;
    *reinterpret_cast<uint2*>(ma + i) = make_uint2(bf16_pack(m[0], m[1]), bf16_pack(m[2], m[3]));
    *reinterpret_cast<uint2*>(va + i) = make_uint2(bf16_pack(v[0], v[1]), bf16_pack(v[2], v[3]));
  }
  const int cnt = bt.split_cnt[b];
  const long long bbase = (long long)bt.split_off[b] * K + (long long)k * cnt;
  for (int t = lane; t < cnt; t += 32) {
    const long long i = bbase + t;
    if (i < 0 || i >= n_beta) break;
    float th = b_cur[i];
    if (improved) b_best[i] = th;
    float g = gb[i];
    float m = beta1 * mb[i] + (1.f - beta1) * g;
    float v = beta2 * vb[i] + (1.f - beta2) * g * g;
    mb[i] = m;
    vb[i] = v;
    th += lr_b * (m / bc1) / (sqrtf(v / bc2) + eps);
    b_cur[i] = fmaxf(th, 0.f);
  }
  __syncwarp();
  if (lane == 0 && improved) best_lb[r] = cur;
}

// ----------------------------------------------------------------------------------------
// Neuron codes per (row, hidden neuron): split overrides stability
// ----------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_codes(RowsCtx c, int layer, int d, long long hoff, int H,
                                               int8_t* __restrict__ out) {
  __shared__ SplitSlot slots[BCROWN_MAX_SPLITS];
  __shared__ int n_slots;
  int rl = blockIdx.x;
  int b, k, p;
  if (!row_prop(c, rl, &b, &k, &p)) p = 0;
  int ns = stage_splits(c, b, layer, d, slots, &n_slots);
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    int s = 0;
    for (int q = 0; q < ns; ++q)
      if (slots[q].idx == j) s = slots[q].sign;
    uint8_t code = c.tb.code[(size_t)p * c.tb.H + hoff + j];
    int8_t v = (int8_t)code;
    if (s == -1) v = CODE_SPLIT_POS;
    if (s == 1) v = CODE_SPLIT_NEG;
    out[(size_t)(c.r0 + rl) * H + hoff + j] = v;
  }
}

// ----------------------------------------------------------------------------------------
// batch_split (Algorithm 1)
// ----------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_split_scan(BatchView bt, int K, const int32_t* __restrict__ U, int P,
                                                     int32_t* c_prop, int32_t* c_off, int32_t* c_cnt,
                                                     int64_t* c_aoff, int* status) {
  __shared__ long long w_s[32], w_a[32];
  __shared__ long long run_s, run_a;
  if (threadIdx.x == 0) {
    run_s = 0;
    run_a = 0;
  }
  __syncthreads();
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < bt.B; base += blockDim.x) {
    int b = base + threadIdx.x;
    long long ns = 0, na = 0;
    int p = 0, cnt = 0;
    if (b < bt.B) {
      p = bt.prop_of[b];
      cnt = bt.split_cnt[b];
      if (p < 0 || p >= P || cnt < 0 || cnt + 1 > BCROWN_MAX_SPLITS) {
        flag(status, BCROWN_ERR_ARG);
        p = 0;
        cnt = 0;
      }
      ns = 2LL * (cnt + 1);
      na = 2LL * (long long)U[p] * K;
    }
    // inclusive warp scans
    long long xs = ns, xa = na;
    for (int o = 1; o < 32; o <<= 1) {
      long long ys = __shfl_up_sync(0xffffffffu, xs, o), ya = __shfl_up_sync(0xffffffffu, xa, o);
      if (lane >= o) {
        xs += ys;
        xa += ya;
      }
    }
    if (lane == 31) {
      w_s[w] = xs;
      w_a[w] = xa;
    }
    __syncthreads();
    long long os = 0, oa = 0, ts = 0, ta = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      if (q < w) {
        os += w_s[q];
        oa += w_a[q];
      }
      ts += w_s[q];
      ta += w_a[q];
    }
    if (b < bt.B) {
      long long s0 = run_s + os + xs - ns, a0 = run_a + oa + xa - na;
      for (int h = 0; h < 2; ++h) {
        c_prop[2 * b + h] = p;
        c_cnt[2 * b + h] = cnt + 1;
        c_off[2 * b + h] = (int32_t)(s0 + h * (cnt + 1));
        c_aoff[2 * b + h] = a0 + h * (long long)U[p] * K;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      run_s += ts;
      run_a += ta;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(128) k_split_copy(BatchView bt, int K, const int32_t* __restrict__ U, int P,
                                                    const uint8_t* __restrict__ pick_layer,
                                                    const uint32_t* __restrict__ pick_idx,
                                                    const float* __restrict__ alpha, const float* __restrict__ beta,
                                                    const int32_t* __restrict__ c_off,
                                                    const int64_t* __restrict__ c_aoff, uint8_t* c_layer,
                                                    uint32_t* c_idx, int8_t* c_sign, float* c_alpha,
                                                    float* c_beta) {
  int child = blockIdx.x;
  int b = child >> 1, h = child & 1;
  int p = bt.prop_of[b];
  int cnt = bt.split_cnt[b];
  if (p < 0 || p >= P || cnt < 0 || cnt + 1 > BCROWN_MAX_SPLITS) return;
  int po = bt.split_off[b];
  int co = c_off[child];
  for (int t = threadIdx.x; t <= cnt; t += blockDim.x) {
    if (t < cnt) {
      c_layer[co + t] = bt.split_layer[po + t];
      c_idx[co + t] = bt.split_idx[po + t];
      c_sign[co + t] = bt.split_sign[po + t];
    } else {
      c_layer[co + t] = pick_layer[b];
      c_idx[co + t] = pick_idx[b];
      c_sign[co + t] = h == 0 ? (int8_t)-1 : (int8_t)1;
    }
  }
  long long n = (long long)U[p] * K;
  const float* src = alpha + bt.alpha_off[b];
  float* dst = c_alpha + c_aoff[child];
  for (long long t = threadIdx.x; t < n; t += blockDim.x) dst[t] = src[t];
  for (int k = 0; k < K; ++k) {
    const float* bs = beta + (long long)po * K + (long long)k * cnt;
    float* bd = c_beta + (long long)co * K + (long long)k * (cnt + 1);
    for (int t = threadIdx.x; t <= cnt; t += blockDim.x) bd[t] = t < cnt ? bs[t] : 0.f;
  }
}

// ----------------------------------------------------------------------------------------
// Root bounds: rows (j, sign) for hidden layer `top`; the top of the recursion is
// Lambda = +-e_j at layer `top`, c = +-b_j.
// ----------------------------------------------------------------------------------------
__global__ void k_root_top(int q0, int Rc, int d_top, const float* __restrict__ b_top, float* __restrict__ Lam,
                           float* __restrict__ cf, double* __restrict__ cd, double* __restrict__ E) {
  long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)Rc * d_top) return;
  int rl = (int)(id / d_top);
  int j = (int)(id - (long long)rl * d_top);
  int q = q0 + rl;
  int jj = q < d_top ? q : q - d_top;
  float sg = q < d_top ? 1.f : -1.f;
  Lam[id] = (j == jj) ? sg : 0.f;
  if (j == 0) {
    float bv = sg * b_top[jj];
    if (cf) cf[rl] = bv;
    if (cd) cd[rl] = (double)bv;
    if (E) E[rl] = 0.0;
  }
}

// Relaxation for root rows: no splits, alpha' from the rule.
template <bool CERT>
__global__ void __launch_bounds__(256) k_relax_root(int Rc, int p, int H, int d, long long hoff,
                                                    const float* __restrict__ l, const float* __restrict__ u,
                                                    Tables tb, int rule, float rule_value,
                                                    const float* __restrict__ Ain, float* __restrict__ Lam,
                                                    const float* __restrict__ bias, float* __restrict__ cf,
                                                    double* __restrict__ cd, double* __restrict__ E,
                                                    const float* __restrict__ wm, double gamma) {
  __shared__ float shf[32];
  int rl = blockIdx.x;
  const float* a_row = Ain + (size_t)rl * d;
  float* lam_row = Lam + (size_t)rl * d;
  // CERT: acc rounded down, e1 and e2 rounded up (as in k_relax)
  float acc = 0.f, e1 = 0.f, e2 = 0.f;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    float a = a_row[j];
    size_t n = (size_t)p * H + hoff + j;
    uint8_t code = tb.code[n];
    float lv = l[n], uv = u[n];
    float D = 0.f, lm = 0.f;
    if (code == CODE_ACTIVE) D = 1.f;
    else if (code == CODE_INACTIVE) D = 0.f;
    else if (a >= 0.f) D = rule == BCROWN_ALPHA_ADAPTIVE ? (uv >= -lv ? 1.f : 0.f) : rule_value;
    else {
      D = tb.slope[n];
      lm = tb.icpt[n];
    }
    float L = a * D;
    lam_row[j] = L;
    float bj = bias[j];
    if (CERT) {
      acc = __fadd_rd(acc, __fadd_rd(__fmul_rd(L, bj), __fmul_rd(a, lm)));
      if (!(D == 0.f || D == 1.f)) {
        float zmax = fmaxf(fabsf(lv), fabsf(uv));
        float er = __fmaf_ru(fabsf(L), 0x1p-23f, 0x1p-140f);
        e1 = __fadd_ru(e1, __fmul_ru(er, zmax));
      }
      e2 = __fadd_ru(e2, __fmul_ru(fabsf(L), wm[n]));
    } else {
      acc = fmaf(L, bj, fmaf(a, lm, acc));
    }
  }
  if (CERT) {
    acc = block_fsum<1>(acc, shf);
    e1 = block_fsum<2>(e1, shf);
    e2 = block_fsum<2>(e2, shf);
    if (threadIdx.x == 0) {
      cd[rl] = __dadd_rd(cd[rl], (double)acc);
      E[rl] = __dadd_ru(E[rl], __dadd_ru((double)e1, __dmul_ru(gamma, (double)e2)));
    }
  } else {
    acc = block_sum(acc, shf);
    if (threadIdx.x == 0) cf[rl] += acc;
  }
}

template <bool CERT>
__global__ void __launch_bounds__(256) k_concretize_root(int q0, int Rc, int p, int d0, int d_top, int H,
                                                         long long hoff_top, const float* __restrict__ x_lo,
                                                         const float* __restrict__ x_hi,
                                                         const float* __restrict__ A0, const float* __restrict__ cf,
                                                         const double* __restrict__ cd, const double* __restrict__ E,
                                                         float* __restrict__ l, float* __restrict__ u) {
  __shared__ float shf[32];
  int rl = blockIdx.x;
  const float* a = A0 + (size_t)rl * d0;
  const float* xl = x_lo + (size_t)p * d0;
  const float* xh = x_hi + (size_t)p * d0;
  float s = 0.f;
  for (int m = threadIdx.x; m < d0; m += blockDim.x) {
    float am = a[m];
    if (CERT) s = __fadd_rd(s, fminf(__fmul_rd(am, xl[m]), __fmul_rd(am, xh[m])));
    else s += fminf(am * xl[m], am * xh[m]);
  }
  float out;
  if (CERT) {
    s = block_fsum<1>(s, shf);
    out = __double2float_rd(__dsub_rd(__dadd_rd(cd[rl], (double)s), E[rl]));
  } else {
    s = block_sum(s, shf);
    out = cf[rl] + s;
  }
  if (threadIdx.x == 0) {
    int q = q0 + rl;
    if (q < d_top) l[(size_t)p * H + hoff_top + q] = isfinite(out) ? out : -INFINITY;
    else u[(size_t)p * H + hoff_top + (q - d_top)] = isfinite(out) ? -out : INFINITY;
  }
}

__global__ void k_count_unstable(int P, int H, const int32_t* __restrict__ U, int32_t* __restrict__ out) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P) out[p] = U[p];
}

// ----------------------------------------------------------------------------------------
// Host launchers
// ----------------------------------------------------------------------------------------
void launch_tables(int P, int H, const float* l, const float* u, Tables& t, uint8_t* code, int32_t* rank,
                   float* slope, float* icpt, int32_t* U, cudaStream_t s) {
  if (P > 0) {
    const int nseg = std::max(1, (H + TAB_SEG - 1) / TAB_SEG);
    if (nseg > 1) {
      k_tables_count<<<dim3(P, nseg), 1024, 0, s>>>(H, l, u, rank);
      k_tables_scan<<<P, 32, 0, s>>>(H, nseg, rank, U);
      g_launches += 2;
    }
    k_tables<<<dim3(P, nseg), 1024, 0, s>>>(H, nseg, l, u, code, rank, slope, icpt, U);
    ++g_launches;
  }
  t.P = P;
  t.H = H;
  t.code = code;
  t.rank = rank;
  t.slope = slope;
  t.icpt = icpt;
  t.U = U;
}

void launch_absw_m(const LayerGeom& g, const float* W, int P, int H, long long hoff_i, long long hoff_prev,
                   const float* u, const float* x_lo, const float* x_hi, int d0, float* wm, cudaStream_t s) {
  long long n = (long long)P * g.d_out;
  if (n > 0) { k_absw_m<<<grid1d(n * 32, 256), 256, 0, s>>>(g, W, P, H, hoff_i, hoff_prev, u, x_lo, x_hi, d0, wm); ++g_launches; }
}

void launch_init_top(bool cert, const RowsCtx& c, int dtop, const bcrown_net* net, long long hoff_top, float* A,
                     float* cf, double* cd, double* E, cudaStream_t s) {
  if (c.R <= 0) return;
  if (cert)
    { k_init_top<true><<<c.R, 256, 0, s>>>(c, dtop, net->Wbar, net->bbar, net->bbar_rd, net->Wbar_err, hoff_top, A,
                                         cf, cd, E); ++g_launches; }
  else
    { k_init_top<false><<<c.R, 256, 0, s>>>(c, dtop, net->Wbar, net->bbar, net->bbar_rd, net->Wbar_err, hoff_top,
                                          A, cf, cd, E); ++g_launches; }
}

void launch_relax(bool cert, const RowsCtx& c, int layer, int d, long long hoff, const float* Ain, float* Lam,
                  const float* bias, const float* alpha, int64_t n_alpha, const float* beta, int64_t n_beta, float* cf,
                  double* cd, double* E, const float* wm, double gamma, cudaStream_t s) {
  if (c.R <= 0) return;
  // one warp per row up to 2048 neurons, a whole block per row beyond
  const bool wide = d > 2048;
  const int rpb = wide ? 1 : RELAX_WARPS;
  const int grid = (c.R + rpb - 1) / rpb;
  if (cert && wide)
    k_relax<true, RELAX_WARPS><<<grid, 32 * RELAX_WARPS, 0, s>>>(c, layer, d, hoff, Ain, Lam, bias, alpha, n_alpha, beta, n_beta, cf, cd, E, wm, gamma);
  else if (cert)
    k_relax<true, 1><<<grid, 32 * RELAX_WARPS, 0, s>>>(c, layer, d, hoff, Ain, Lam, bias, alpha, n_alpha, beta, n_beta, cf, cd, E, wm, gamma);
  else if (wide)
    k_relax<false, RELAX_WARPS><<<grid, 32 * RELAX_WARPS, 0, s>>>(c, layer, d, hoff, Ain, Lam, bias, alpha, n_alpha, beta, n_beta, cf, cd, E, wm, gamma);
  else
    k_relax<false, 1><<<grid, 32 * RELAX_WARPS, 0, s>>>(c, layer, d, hoff, Ain, Lam, bias, alpha, n_alpha, beta, n_beta, cf, cd, E, wm, gamma);
  ++g_launches;
}

void launch_sgemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                  const float* bias, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + 127) / 128, (M + 127) / 128);
  { k_sgemm<<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias); ++g_launches; }
}

void launch_conv_bwd(int R, const LayerGeom& g, const float* Lam, const float* W, float* Ain, cudaStream_t s) {
  if (R <= 0 || g.d_in <= 0) return;
  // rows on grid.z (at most 65535 per launch)
  for (int r0 = 0; r0 < R; r0 += 65535) {
    const int rn = std::min(R - r0, 65535);
    dim3 grid((g.in_h * g.in_w + CONV_POS - 1) / CONV_POS, (g.in_c + CONV_CB - 1) / CONV_CB, rn);
    k_conv_bwd<<<grid, CONV_POS, 0, s>>>(rn, g, Lam + (size_t)r0 * g.d_out, W, Ain + (size_t)r0 * g.d_in);
    ++g_launches;
  }
}

void launch_conv_fwd(int R, const LayerGeom& g, const float* h, const float* W, const float* bias, float* Z,
                     cudaStream_t s) {
  if (R <= 0 || g.d_out <= 0) return;
  for (int r0 = 0; r0 < R; r0 += 65535) {
    const int rn = std::min(R - r0, 65535);
    dim3 grid((g.out_h * g.out_w + CONV_POS - 1) / CONV_POS, (g.out_c + CONV_CB - 1) / CONV_CB, rn);
    k_conv_fwd<<<grid, CONV_POS, 0, s>>>(rn, g, h + (size_t)r0 * g.d_in, W, bias, Z + (size_t)r0 * g.d_out);
    ++g_launches;
  }
}

void launch_concretize(bool cert, const RowsCtx& c, int d0, const float* A0, const float* cf, const double* cd,
                       const double* E, float* lb, cudaStream_t s) {
  if (c.R <= 0) return;
  if (cert) { k_concretize<true><<<c.R, 256, 0, s>>>(c, d0, A0, cf, cd, E, lb); ++g_launches; }
  else { k_concretize<false><<<c.R, 256, 0, s>>>(c, d0, A0, cf, cd, E, lb); ++g_launches; }
}

void launch_xstar(const RowsCtx& c, int d0, const float* A0, float* h0, cudaStream_t s) {
  long long n = (long long)c.R * d0;
  if (n > 0) { k_xstar<<<grid1d(n, 256), 256, 0, s>>>(c, d0, A0, h0); ++g_launches; }
}

void launch_fwd_epi(const RowsCtx& c, int layer, int d, long long hoff, float* Z, const float* Ai,
                    const float* alpha, int64_t n_alpha, float* dalpha, float* dbeta, int64_t n_beta,
                    cudaStream_t s) {
  if (c.R <= 0) return;
  if (d <= 2048) {
    k_fwd_epi<false><<<c.R, 256, 0, s>>>(c, layer, d, hoff, Z, Ai, alpha, n_alpha, dalpha, dbeta, n_beta);
  } else {
    const size_t smem = d <= SPLIT_MASK_WORDS * 32 ? (size_t)(d + 31) / 32 * sizeof(uint32_t) : 0;
    k_fwd_epi<true><<<c.R, 256, smem, s>>>(c, layer, d, hoff, Z, Ai, alpha, n_alpha, dalpha, dbeta, n_beta);
  }
  ++g_launches;
}

void launch_adam(int R, int K, const BatchView& bt, const int32_t* U, int P, const float* lb_t, float* best_lb,
                 float* a_cur, float* a_best, const float* ga, float* ma, float* va, float* b_cur, float* b_best,
                 const float* gb, float* mb, float* vb, float lr_a, float lr_b, float beta1, float beta2, float eps,
                 float bc1, float bc2, int64_t n_alpha, int64_t n_beta, cudaStream_t s) {
  if (R <= 0) return;
  if (R > 0) {
    k_adam<<<(R + ADAM_ROWS_PER_BLOCK - 1) / ADAM_ROWS_PER_BLOCK, 32 * ADAM_ROWS_PER_BLOCK, 0, s>>>(
        R, K, bt, U, P, lb_t, best_lb, a_cur, a_best, ga, ma, va, b_cur, b_best, gb, mb, vb, lr_a, lr_b, beta1, beta2,
        eps, bc1, bc2, n_alpha, n_beta);
    ++g_launches;
  }
}

void launch_adam16(int R, int K, const BatchView& bt, const int32_t* U, int P, const float* lb_t, float* best_lb,
                   float* a_cur, float* a_best, const __nv_bfloat16* ga, __nv_bfloat16* ma, __nv_bfloat16* va,
                   float* b_cur, float* b_best, const float* gb, float* mb, float* vb, float lr_a, float lr_b,
                   float beta1, float beta2, float eps, float bc1, float bc2, int64_t n_alpha, int64_t n_beta,
                   cudaStream_t s) {
  if (R <= 0) return;
  k_adam16<<<(R + ADAM_ROWS_PER_BLOCK - 1) / ADAM_ROWS_PER_BLOCK, 32 * ADAM_ROWS_PER_BLOCK, 0, s>>>(
      R, K, bt, U, P, lb_t, best_lb, a_cur, a_best, ga, ma, va, b_cur, b_best, gb, mb, vb, lr_a, lr_b, beta1, beta2,
      eps, bc1, bc2, n_alpha, n_beta);
  ++g_launches;
}

void launch_codes(const RowsCtx& c, int layer, int d, long long hoff, int H, int8_t* out, cudaStream_t s) {
  if (c.R > 0) { k_codes<<<c.R, 256, 0, s>>>(c, layer, d, hoff, H, out); ++g_launches; }
}

void launch_split(const BatchView& bt, int K, const int32_t* U, int P, const uint8_t* pick_layer,
                  const uint32_t* pick_idx, const float* alpha, const float* beta, int32_t* c_prop, int32_t* c_off,
                  int32_t* c_cnt, int64_t* c_aoff, uint8_t* c_layer, uint32_t* c_idx, int8_t* c_sign,
                  float* c_alpha, float* c_beta, int* status, cudaStream_t s) {
  if (bt.B <= 0) return;
  { k_split_scan<<<1, 1024, 0, s>>>(bt, K, U, P, c_prop, c_off, c_cnt, c_aoff, status); ++g_launches; }
  { k_split_copy<<<2 * bt.B, 128, 0, s>>>(bt, K, U, P, pick_layer, pick_idx, alpha, beta, c_off, c_aoff, c_layer, c_idx,
                                        c_sign, c_alpha, c_beta); ++g_launches; }
}

void launch_root_top(int q0, int Rc, int d_top, const float* b_top, float* Lam, float* cf, double* cd, double* E,
                     cudaStream_t s) {
  long long n = (long long)Rc * d_top;
  if (n > 0) { k_root_top<<<grid1d(n, 256), 256, 0, s>>>(q0, Rc, d_top, b_top, Lam, cf, cd, E); ++g_launches; }
}

void launch_relax_root(bool cert, int Rc, int p, int H, int d, long long hoff, const float* l, const float* u,
                       const Tables& tb, int rule, float rule_value, const float* Ain, float* Lam, const float* bias,
                       float* cf, double* cd, double* E, const float* wm, double gamma, cudaStream_t s) {
  if (Rc <= 0) return;
  if (cert)
    { k_relax_root<true><<<Rc, 256, 0, s>>>(Rc, p, H, d, hoff, l, u, tb, rule, rule_value, Ain, Lam, bias, cf, cd, E,
                                          wm, gamma); ++g_launches; }
  else
    { k_relax_root<false><<<Rc, 256, 0, s>>>(Rc, p, H, d, hoff, l, u, tb, rule, rule_value, Ain, Lam, bias, cf, cd, E,
                                           wm, gamma); ++g_launches; }
}

void launch_concretize_root(bool cert, int q0, int Rc, int p, int d0, int d_top, int H, long long hoff_top,
                            const float* x_lo, const float* x_hi, const float* A0, const float* cf, const double* cd,
                            const double* E, float* l, float* u, cudaStream_t s) {
  if (Rc <= 0) return;
  if (cert)
    { k_concretize_root<true><<<Rc, 256, 0, s>>>(q0, Rc, p, d0, d_top, H, hoff_top, x_lo, x_hi, A0, cf, cd, E, l, u); ++g_launches; }
  else
    { k_concretize_root<false><<<Rc, 256, 0, s>>>(q0, Rc, p, d0, d_top, H, hoff_top, x_lo, x_hi, A0, cf, cd, E, l, u); ++g_launches; }
}

__global__ void k_fill(float* p, long long n, float v) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

void launch_fill(float* p, long long n, float v, cudaStream_t s) {
  if (n > 0) { k_fill<<<grid1d(n, 256), 256, 0, s>>>(p, n, v); ++g_launches; }
}

// ReLU in place (the plain network evaluation of bcrown_forward).
__global__ void k_relu(float* __restrict__ z, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = fmaxf(z[i], 0.f);
}
void launch_relu(float* z, long long n, cudaStream_t s) {
  if (n > 0) { k_relu<<<grid1d(n, 256), 256, 0, s>>>(z, n); ++g_launches; }
}

// out[r][k] = bbar_k + sum_j h[r][j] Wbar[k][j] (the specifications merged into the last layer):
// one warp per (row, spec).
__global__ void k_spec_out(int R, int K, int d, const float* __restrict__ h, const float* __restrict__ Wbar,
                           const float* __restrict__ bbar, float* __restrict__ out) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (long long)R * K) return;
  const int r = (int)(w / K), k = (int)(w - (long long)r * K);
  float acc = 0.f;
  for (int j = lane; j < d; j += 32) acc = fmaf(h[(size_t)r * d + j], Wbar[(size_t)k * d + j], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[w] = acc + bbar[k];
}
void launch_spec_out(int R, int K, int d, const float* h, const float* Wbar, const float* bbar, float* out,
                     cudaStream_t s) {
  const long long n = (long long)R * K * 32;
  if (n > 0) { k_spec_out<<<grid1d(n, 256), 256, 0, s>>>(R, K, d, h, Wbar, bbar, out); ++g_launches; }
}

// FP32 <-> BF16 copies (the BF16 optimiser keeps alpha's moments in BF16 inside a call).
__global__ void k_f32_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}
__global__ void k_bf16_to_f32(const __nv_bfloat16* __restrict__ src, float* __restrict__ dst, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __bfloat162float(src[i]);
}
void launch_f32_to_bf16(const float* src, __nv_bfloat16* dst, long long n, cudaStream_t s) {
  if (n > 0) { k_f32_to_bf16<<<grid1d(n, 256), 256, 0, s>>>(src, dst, n); ++g_launches; }
}
void launch_bf16_to_f32(const __nv_bfloat16* src, float* dst, long long n, cudaStream_t s) {
  if (n > 0) { k_bf16_to_f32<<<grid1d(n, 256), 256, 0, s>>>(src, dst, n); ++g_launches; }
}

void launch_copy_count(int P, int H, const int32_t* U, int32_t* out, cudaStream_t s) {
  if (P > 0 && out) { k_count_unstable<<<grid1d(P, 128), 128, 0, s>>>(P, H, U, out); ++g_launches; }
}

}  // namespace bcrown
