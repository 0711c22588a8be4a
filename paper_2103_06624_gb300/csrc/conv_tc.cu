// Convolution layers as tcgen05 GEMMs (sm_103a) for the BF16 precision of the layer-by-layer
// path: Eq. definition_A's contraction A^(i-1) = Lambda^(i) W^(i) is the transposed
// convolution, and the adjoint's zhat^(i) = W^(i) h^(i-1) + b^(i) the convolution itself.
// Both become GEMMs over an im2col operand gathered into BF16, multiplied on the tensor cores
// with FP32 accumulation in TMEM.
//
// Every mbarrier wait is bounded; on expiry the kernel records BCROWN_ERR_TIMEOUT, raises its
// abort flag, waits (bounded) for its copies in flight, frees TMEM and returns.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "conv_tc.cuh"
#include "tc_ptx.cuh"

namespace bcrown {

extern std::atomic<long long> g_launches;

namespace tc {

// Convolutions on the tensor cores (BF16 precision of the layer-by-layer path): the contraction
// of a conv layer as GEMMs over an im2col operand.
//   forward:   Z[r][co][p] = sum_K Col[(r, p)][K] Wf[co][K] + b,   K = (ci, ky, kx)
//   backward:  the transposed convolution Ain[r][ci][p] = sum Lambda[r][co][q] W[co][ci][tap]
//              over the (q, tap) with p = q * s - pad + tap.  For stride s the input positions
//              fall into s x s phases (p_y mod s, p_x mod s); within a phase only the taps
//              ky = ky0 + s * dy (dy < ceil(k / s)) reach the stride grid, and the source
//              position is q_y = i + off - dy for the phase's i-th row.  Each phase is one GEMM
//              with K = (co, dy, dx) and its own weight matrix, so the operand holds no
//              structural zeros of the stride.
// k_tcg<true> multiplies Col with the BF16 weights without storing Col: gather warps build each
// 128 x 64 K block of it in shared memory from a per-K table (source offset and tap offsets: no
// divisions in the inner loop) while TMA streams the weights; M = rows x positions (tiles of
// 128 on the TMEM lanes), N = channels (padded to 16).  k_im2col + k_tcg<false> is the same
// product with Col written to an HBM buffer and read back by TMA (fully connected layers, and
// conv layers when BCROWN_CONV_IM2COL=1 selects it for comparison).
// ------------------------------------------------------------------------------------------
constexpr int TCG_NS = 4;         // pipeline stages (A: 128 x 64, B: Np x 64)
// Warp roles of k_tcg: epilogue warps 0 .. EPI-1 (TMEM lane quadrant warp % 4, column chunks
// warp / 4 + EPI / 4 * i), the TMA warp EPI, the MMA warp EPI + 1, and in gather mode the warps
// from EPI + 2 on, which build the A operand in shared memory (gather warp w fills the chunks
// 8 / GPS * (w / NS) .. of ring slot w % NS), so the im2col operand never goes through HBM.
template <bool GATHER>
struct TcgRoles {
  static constexpr int EPI = GATHER ? 4 : 8;
  static constexpr int TMA = EPI, MMA = EPI + 1, GATHER0 = EPI + 2;
  static constexpr int GPS = 4;                          // gather warps per ring slot
  static constexpr int GW = GATHER ? GPS * TCG_NS : 0;
  static constexpr int THREADS = (EPI + 2 + GW) * 32;
};
constexpr int TCG_BIAS_MAX = 4096;  // channel biases staged in shared memory up to this many
// Dynamic shared memory of k_tcg: 1 KB alignment slack, the stages, barriers, staged biases,
// and in gather mode the K table (kp_gather entries).
__host__ __device__ inline int tcg_bias_bytes(int N, bool bias) { return bias && N <= TCG_BIAS_MAX ? (N + 3) / 4 * 16 : 0; }
inline int tcg_smem(int Np, int N, bool bias, int kp_gather = 0) {
  return 1024 + TCG_NS * (16384 + Np * 128) + 256 + tcg_bias_bytes(N, bias) + kp_gather * (int)sizeof(int2);
}

// One gather: row m = (r, pp), pp = i * nJ + j; source position (y0 + dy_K, x0 + dx_K) with
// y0 = i * ms + cy, x0 = j * ms + cx, in a [C][Hs][Ws] map of row r (d_src floats per row).
struct Im2colPass {
  long long M;
  int Pm, nJ, ms, cy, cx, Hs, Ws, d_src, Kp;
  // [Kp]: {source offset c * Hs * Ws + dy * Ws + dx; (dy & 0xffff) | dx << 16}, a zero column
  // (K padding, a tap off the stride grid) with dy = -32768, which no bounds test passes
  const int2* tab;
};

// 32 consecutive rows m per block.  Lanes walk the 32 rows for 16 K at a time (K uniform per
// warp: coalesced source reads) into a shared tile [32][Kp + 8], whose rows then leave in
// 16-byte stores.
constexpr int IM2COL_ROWS = 32;
constexpr int IM2COL_MAX_KP = 2048;
inline int im2col_smem(int Kp) { return Kp * (int)sizeof(int2) + IM2COL_ROWS * (Kp + 8) * 2; }
__global__ void __launch_bounds__(256) k_im2col(Im2colPass q, const float* __restrict__ src,
                                                __nv_bfloat16* __restrict__ col) {
  extern __shared__ __align__(16) uint8_t im_raw[];
  const int Kp = q.Kp, S = Kp + 8;  // row stride (bf16), 16-byte aligned rows
  int2* tab = reinterpret_cast<int2*>(im_raw);
  __nv_bfloat16* tile = reinterpret_cast<__nv_bfloat16*>(im_raw + (size_t)Kp * sizeof(int2));
  for (int k = threadIdx.x; k < Kp; k += 256) tab[k] = q.tab[k];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long m0 = (long long)blockIdx.x * IM2COL_ROWS;
  const long long m = m0 + lane;
  const bool mv = m < q.M;
  const int r = mv ? (int)(m / q.Pm) : 0;
  const int pp = mv ? (int)(m - (long long)r * q.Pm) : 0;
  const int i = pp / q.nJ, j = pp - (pp / q.nJ) * q.nJ;
  // a row past M gets y0 = -32768: no bounds test passes
  const int y0 = mv ? i * q.ms + q.cy : -32768, x0 = j * q.ms + q.cx;
  const float* sr = src + (size_t)r * q.d_src + (mv ? y0 * q.Ws + x0 : 0);
  __syncthreads();
  // 16 K per lane per step: 16 independent loads in flight before the first use
  for (int K0 = 16 * w; K0 < Kp; K0 += 128) {
    float v[16];
#pragma unroll
    for (int e = 0; e < 16; e += 2) {
      const int4 t2 = *reinterpret_cast<const int4*>(tab + K0 + e);
      const int ya = y0 + (int)(short)(t2.y & 0xffff), xa = x0 + (t2.y >> 16);
      const int yb = y0 + (int)(short)(t2.w & 0xffff), xb = x0 + (t2.w >> 16);
      v[e] = ((unsigned)ya < (unsigned)q.Hs && (unsigned)xa < (unsigned)q.Ws) ? sr[t2.x] : 0.f;
      v[e + 1] = ((unsigned)yb < (unsigned)q.Hs && (unsigned)xb < (unsigned)q.Ws) ? sr[t2.z] : 0.f;
    }
    uint32_t pk[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
      pk[e] = *reinterpret_cast<uint32_t*>(&b2);
    }
    uint4* d = reinterpret_cast<uint4*>(tile + lane * S + K0);
    d[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    d[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
  }
  __syncthreads();
  const int cpr = Kp / 8;
  for (int row = w; row < IM2COL_ROWS; row += 8) {
    if (m0 + row >= q.M) break;
    uint4* dst = reinterpret_cast<uint4*>(col + (m0 + row) * Kp);
    const uint4* sv = reinterpret_cast<const uint4*>(tile + row * S);
    for (int c = lane; c < cpr; c += 32) dst[c] = sv[c];
  }
}

// Fully connected operand: row r of src (d floats) to BF16 [M][Kp], zero past d.  One thread per
// 8 columns (one 16-byte store); consecutive threads walk a row.
__global__ void k_rows_bf16(long long M, int d, int Kp, const float* __restrict__ src,
                            __nv_bfloat16* __restrict__ col) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int cpr = Kp / 8;
  if (id >= M * cpr) return;
  const long long r = id / cpr;
  const int k0 = (int)(id - r * cpr) * 8;
  const float* sr = src + r * d;
  float v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = k0 + e < d ? sr[k0 + e] : 0.f;
  uint32_t pk[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    pk[e] = *reinterpret_cast<uint32_t*>(&b2);
  }
  *reinterpret_cast<uint4*>(col + r * Kp + k0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
}

// Where k_tcg writes: row m = (r, pp), pp = i * nJ + j, goes to position
// p = (a + so * i) * Wo + (b + so * j) of out[r * stride + n * P + p] (+ bias[n * P + p]).
// A fully connected layer is the case P = 1 (one position per row).
struct TcgOut {
  long long M;
  int N, Np, ntn, nkb, brow;  // N in ntn tiles of Np; brow: first row of the weight operand in its map
  int Pm, nJ, a, b, so, Wo, P;
  long long stride;
};

// Bounded wait for k_tcg (same limit and error reporting as mbar_wait).
__device__ __forceinline__ bool tcg_wait(uint64_t* b, uint32_t parity, volatile int* abort, int* status) {
  if (mbar_try(b, parity)) return true;
  long long t0 = clock64();
  while (true) {
    if (mbar_try_sleep(b, parity, 20000u)) return true;
    if (*abort) return false;
    if (clock64() - t0 > 4000000000LL) {
      atomicCAS(status, 0, BCROWN_ERR_TIMEOUT);
      *abort = 1;
      return false;
    }
  }
}

// Predicated FP32 load issued where it is written (0 when pred is false).
__device__ __forceinline__ float ld_f32_pred(const float* p, bool pred) {
  float v;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.f32 %0, 0f00000000;\n\t@q ld.global.f32 %0, [%1];\n\t}"
               : "=f"(v)
               : "l"(p), "r"((uint32_t)pred)
               : "memory");
  return v;
}

// One 8-K chunk of gather mode: rows ln + 32 q (q < 4) of the A stage, K = K0 .. K0 + 7, from
// the table entries t[0..7] (sr[q]: the row's source at its base position (y0, x0), which a
// row past M sets to y0 = -32768); written in the 128-byte-swizzled K-major layout (16-byte chunk c
// of row m at chunk position c ^ (m & 7)).
__device__ __forceinline__ void gather_chunk(uint8_t* stage, int c, int ln, const int4 (&t4)[4],
                                             const float* const (&sr)[4], const int (&y0)[4], const int (&x0)[4],
                                             int Hs, int Ws) {
  float v[4][8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int4 tt = t4[e >> 1];
    const int off = (e & 1) ? tt.z : tt.x;
    const int pk = (e & 1) ? tt.w : tt.y;
    const int dy = (int)(short)(pk & 0xffff), dx = pk >> 16;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool ok = (unsigned)(y0[q] + dy) < (unsigned)Hs && (unsigned)(x0[q] + dx) < (unsigned)Ws;
      v[q][e] = ld_f32_pred(sr[q] + off, ok);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t pk[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      __nv_bfloat162 b2 = __floats2bfloat162_rn(v[q][2 * e], v[q][2 * e + 1]);
      pk[e] = *reinterpret_cast<uint32_t*>(&b2);
    }
    const int m = ln + 32 * q;
    *reinterpret_cast<uint4*>(stage + m * 128 + ((c ^ (m & 7)) << 4)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

// out[r * stride + n * P + p] = (Col x W^T)[m = r * P + p][n] (+ bias[n * P + p]) for n < N.
// The bias is per channel (constant over the positions p, as conv biases are stored): it is
// read at p = 0, into shared memory when N <= TCG_BIAS_MAX.
// GATHER = false: Col is read by TMA through mapA.  GATHER = true: Col is never stored; gather
// warps build each A stage from src with the im2col pass q (mapA unused).
template <bool GATHER>
__global__ void __launch_bounds__(TcgRoles<GATHER>::THREADS, 1)
    k_tcg(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcgOut o, Im2colPass gq,
          const float* __restrict__ src, float* __restrict__ out, const float* __restrict__ bias, int* status) {
  const long long M = o.M;
  const int N = o.N, Np = o.Np, nkb = o.nkb;
  using R = TcgRoles<GATHER>;
  extern __shared__ __align__(1024) uint8_t tsm_raw[];
  const uint32_t pad = (1024u - (su32(tsm_raw) & 1023u)) & 1023u;
  uint8_t* base = tsm_raw + pad;
  const int bbytes = Np * 128;
  uint8_t* sA = base;                                  // TCG_NS x 16 KB
  uint8_t* sB = base + TCG_NS * 16384;                 // TCG_NS x Np*128
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + TCG_NS * bbytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + TCG_NS;
  uint64_t* acc_full = bars + 2 * TCG_NS;
  uint64_t* acc_empty = bars + 2 * TCG_NS + 2;
  uint32_t* tbase_sm = reinterpret_cast<uint32_t*>(bars + 2 * TCG_NS + 4);
  volatile int* abort = reinterpret_cast<volatile int*>(tbase_sm + 1);
  float* sbias = reinterpret_cast<float*>(bars + 32);  // 256 bytes past the barriers
  const bool stage_bias = bias != nullptr && N <= TCG_BIAS_MAX;
  int2* stab = reinterpret_cast<int2*>(reinterpret_cast<uint8_t*>(sbias) + tcg_bias_bytes(N, bias != nullptr));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long ntiles = (M + 127) / 128 * o.ntn;   // tile = m tile * ntn + n tile
  // two accumulators of Np columns, allocated as a power of two >= 32
  const uint32_t tcols = Np <= 16 ? 32u : (Np <= 32 ? 64u : (Np <= 64 ? 128u : (Np <= 128 ? 256u : 512u)));
  if (threadIdx.x == 0) {
    for (int i = 0; i < TCG_NS; ++i) {
      mbar_init(&full[i], 1 + R::GPS * GATHER);   // the TMA transaction (+ the gather warps' arrivals)
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], R::EPI);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == R::MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tbase_sm)), "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase_sm;
  if (warp == R::TMA) {
    if (lane == 0) {
      uint32_t seq = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        // the tile's coordinates once per tile: the K loop of this one thread holds no division
        const long long mt = tile / o.ntn;
        const int arow = (int)(mt * 128), brow = o.brow + (int)(tile - mt * o.ntn) * Np;
        for (int kb = 0; kb < nkb; ++kb, ++seq) {
          const int st = seq % TCG_NS;
          if (!tcg_wait(&empty[st], ((seq / TCG_NS) & 1) ^ 1, abort, status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[st], (GATHER ? 0u : 16384u) + (uint32_t)bbytes);
          if (!GATHER) tma_load_2d(sA + st * 16384, &mapA, kb * 64, arow, &full[st]);
          tma_load_2d(sB + st * bbytes, &mapB, kb * 64, brow, &full[st]);
        }
      }
      if (!ok) {
        for (uint32_t q = (seq > TCG_NS ? seq - TCG_NS : 0); q < seq; ++q) {
          long long t0 = clock64();
          while (!mbar_try(&full[q % TCG_NS], (q / TCG_NS) & 1) && clock64() - t0 < 200000000LL) {
          }
        }
      }
    }
  } else if (warp == R::MMA) {
    if (lane == 0) {
      uint32_t seq = 0, accseq = 0;
      bool ok = true;
      const uint32_t idesc = idesc_bf16(Np);
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++accseq) {
        const int buf = accseq & 1;
        if (!tcg_wait(&acc_empty[buf], ((accseq >> 1) & 1) ^ 1, abort, status)) break;
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * Np);
        for (int kb = 0; kb < nkb; ++kb, ++seq) {
          const int st = seq % TCG_NS;
          if (!tcg_wait(&full[st], (seq / TCG_NS) & 1, abort, status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          umma_kblock(dt, sdesc(su32(sA + st * 16384)), sdesc(su32(sB + st * bbytes)), idesc, kb != 0 ? 1u : 0u);
          umma_commit(&empty[st]);
        }
        if (!ok) break;
        umma_commit(&acc_full[buf]);
      }
    }
  } else if (GATHER && warp >= R::GATHER0) {
    // ring slot g takes sequence numbers g, g + TCG_NS, ... of the (tile, K block) order the
    // MMA warp consumes; this warp fills its share of the slot's 8 chunks
    const int g = (warp - R::GATHER0) % TCG_NS, part = (warp - R::GATHER0) / TCG_NS;
    constexpr int CPW = 8 / R::GPS;   // chunks per gather warp
    for (int k = threadIdx.x - R::GATHER0 * 32; k < gq.Kp; k += R::GW * 32) stab[k] = gq.tab[k];
    asm volatile("bar.sync 2, %0;" ::"n"(R::GW * 32) : "memory");
    uint32_t seq = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      // this lane's rows ln + 32 q of the tile
      const float* sr[4];
      int y0[4], x0[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long m = tile / o.ntn * 128 + lane + 32 * q;
        const bool mv = m < M;
        const long long r = mv ? m / gq.Pm : 0;
        const int pp = mv ? (int)(m - r * gq.Pm) : 0;
        const int i = pp / gq.nJ, j = pp - (pp / gq.nJ) * gq.nJ;
        y0[q] = mv ? i * gq.ms + gq.cy : -32768;
        x0[q] = j * gq.ms + gq.cx;
        sr[q] = src + r * gq.d_src + (mv ? y0[q] * gq.Ws + x0[q] : 0);
      }
      for (int kb = 0; kb < nkb; ++kb, ++seq) {
        if ((int)(seq % TCG_NS) != g) continue;
        int okw = 1;
        if (lane == 0) okw = tcg_wait(&empty[g], ((seq / TCG_NS) & 1) ^ 1, abort, status) ? 1 : 0;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) {
          ok = false;
          break;
        }
        uint8_t* stage = sA + g * 16384;
#pragma unroll 1
        for (int c = CPW * part; c < CPW * part + CPW; ++c) {
          int4 t4[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) t4[e] = reinterpret_cast<const int4*>(stab + kb * 64 + c * 8)[e];
          gather_chunk(stage, c, lane, t4, sr, y0, x0, gq.Hs, gq.Ws);
        }
        fence_proxy_async();   // the stage's generic-proxy stores, before the MMA reads it
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[g]);
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes (tile rows) 32 (w % 4) .. + 31, column chunks w / 4,
    // w / 4 + EPI / 4, ...
    const int q4 = warp & 3, half = warp >> 2;
    if (stage_bias) {
      for (int n = threadIdx.x; n < N; n += R::EPI * 32) sbias[n] = bias[(size_t)n * o.P];
      asm volatile("bar.sync 1, %0;" ::"n"(R::EPI * 32) : "memory");
    }
    const bool vec = o.P == 1 && (o.stride & 3) == 0 &&
                     ((reinterpret_cast<uintptr_t>(out) | (stage_bias ? 0 : reinterpret_cast<uintptr_t>(bias))) &
                      15) == 0;
    uint32_t accseq = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++accseq) {
      const int buf = accseq & 1;
      int okw = 1;
      if (lane == 0) okw = tcg_wait(&acc_full[buf], (accseq >> 1) & 1, abort, status) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      tc_fence_after();
      const long long m = tile / o.ntn * 128 + 32 * q4 + lane;
      const int nb = (int)(tile % o.ntn) * Np;
      const bool min_ = m < M;
      const long long r = min_ ? m / o.Pm : 0;
      const int pp = min_ ? (int)(m - r * o.Pm) : 0;
      const int i = pp / o.nJ, j = pp - (pp / o.nJ) * o.nJ;
      const int p = (o.a + o.so * i) * o.Wo + o.b + o.so * j;
      float* orow = out + r * o.stride + p;
      for (int n0 = 16 * half; n0 < Np; n0 += 16 * (R::EPI / 4)) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(buf * Np + n0), v);
        if (min_) {
          if (vec && nb + n0 + 16 <= N) {
            // one position per row: the 16 channels are contiguous
#pragma unroll
            for (int e = 0; e < 16; e += 4) {
              const int n = nb + n0 + e;
              float4 x = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
              if (bias) {
                const float4 bb = stage_bias ? *reinterpret_cast<const float4*>(sbias + n)
                                             : *reinterpret_cast<const float4*>(bias + n);
                x.x += bb.x, x.y += bb.y, x.z += bb.z, x.w += bb.w;
              }
              *reinterpret_cast<float4*>(orow + n) = x;
            }
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int n = nb + n0 + e;
              if (n < N)
                orow[(size_t)n * o.P] =
                    v[e] + (stage_bias ? sbias[n] : (bias ? bias[(size_t)n * o.P] : 0.f));
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == R::MMA) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
  }
}

}  // namespace tc

using namespace tc;

// Conv passes gather their operand inside the GEMM kernel, except on BCROWN_PATH_LAYER_IM2COL
// (an im2col buffer in HBM read by TMA), the configuration of the call in progress.
static bool tcg_gather(const bcrown_net* net) { return net->launch_now.path != BCROWN_PATH_LAYER_IM2COL; }

namespace {

// col2im of the scatter form: A[r][ci][yi][xi] = sum over (ky, kx), in that order, of
// P[r][(ci k + ky) k + kx][y][x] where yi = y s + ky - pad and xi = x s + kx - pad.
struct Col2im {
  int C, H, W, k, s, pad, oh, ow;
};
__global__ void __launch_bounds__(256) k_col2im(long long total, Col2im g, const float* __restrict__ P,
                                                float* __restrict__ out, int d_in) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= total) return;
  const long long r = id / d_in;
  const int e = (int)(id - r * d_in);
  const int HW = g.H * g.W, ci = e / HW, rem = e - ci * HW, yi = rem / g.W, xi = rem - (rem / g.W) * g.W;
  const int OP = g.oh * g.ow;
  const float* pr = P + (size_t)r * g.C * g.k * g.k * OP;
  float acc = 0.f;
  for (int ky = 0; ky < g.k; ++ky) {
    const int yy = yi + g.pad - ky;
    if (yy < 0 || yy % g.s != 0 || yy / g.s >= g.oh) continue;
    const int y = yy / g.s;
    for (int kx = 0; kx < g.k; ++kx) {
      const int xx = xi + g.pad - kx;
      if (xx < 0 || xx % g.s != 0 || xx / g.s >= g.ow) continue;
      acc += pr[(size_t)((ci * g.k + ky) * g.k + kx) * OP + y * g.ow + xx / g.s];
    }
  }
  out[id] = acc;
}

// Per-layer BF16 weights, gather tables and tensor maps of one net, built on first use.
struct ConvTc {
  struct ConvW {
    int Np_b = 0, Kp_b = 0, Np_f = 0, Kp_f = 0, ntn_b = 1, ntn_f = 1;  // N in ntn tiles of Np
    CUtensorMap mb, mf;              // mb: the s * s phase matrices stacked, Np_b rows each
    int2 *tab_b = nullptr, *tab_f = nullptr;  // gather tables: [s * s][Kp_b], [Kp_f]
    __nv_bfloat16 *wb = nullptr, *wf = nullptr;  // fc: the B operands behind mb, mf
    // scatter form of the backward pass (layers with in_c k^2 <= SCATTER_MAX_N): one GEMM
    // P = Lambda^T W' over the output channels (K = out_c, N = in_c k^2), then col2im
    bool scat = false;
    int Np_s = 0, Kp_s = 0;
    CUtensorMap ms;
    int2* tab_s = nullptr;
  };
  std::vector<ConvW> conv;  // conv[i]: paper layer i
  std::vector<void*> bufs;
  bool ready = false;
};

std::mutex g_conv_mu;
std::vector<std::pair<const bcrown_net*, ConvTc*>> g_conv;

ConvTc* conv_of(const bcrown_net* net) {
  std::lock_guard<std::mutex> g(g_conv_mu);
  for (auto& e : g_conv)
    if (e.first == net) return e.second;
  ConvTc* t = new ConvTc();
  g_conv.push_back({net, t});
  return t;
}

int pad_to(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

// Phase a of one spatial axis of a stride-s transposed convolution: the taps ky0 + s * dy
// (dy < nk) that reach the stride grid from input rows a + s * i (i < n), whose source row is
// i + off - dy.
struct ConvPhase {
  int k0, nk, off, n;
};
static ConvPhase conv_phase(int a, int k, int s, int pad, int in) {
  ConvPhase c;
  c.k0 = (a + pad) % s;
  c.nk = c.k0 < k ? (k - c.k0 + s - 1) / s : 0;
  c.off = (a + pad - c.k0) / s;
  c.n = a < in ? (in - a + s - 1) / s : 0;
  return c;
}
static int taps_per_axis(const LayerDev& l) { return (l.k + l.stride - 1) / l.stride; }
static int kp_bwd(const LayerDev& l) { return pad_to(l.out_c * taps_per_axis(l) * taps_per_axis(l), 64); }
static int kp_fwd(const LayerDev& l) { return pad_to(l.in_c * l.k * l.k, 64); }
// The transposed convolution of a layer with few input channels is computed as
//   P[(y, x)][(ci, ky, kx)] = sum_co Lambda[co][y][x] W[co][ci][ky][kx]   (one GEMM, K = out_c)
//   A[ci][yi][xi] = sum over the taps (ky, kx) that reach (yi, xi) of P[(y, x)][(ci, ky, kx)]
// instead of gathering out_c x taps source values per input position: for conv_big's first
// layer (3 input channels, 3x3) that is K = 64 gathered values per position instead of 576.
constexpr int SCATTER_MAX_N = 64;
static bool scatter_form(const LayerDev& l) {
  return l.kind == BCROWN_LAYER_CONV && l.in_c * l.k * l.k <= SCATTER_MAX_N && l.out_c <= 256;
}
// Gather table entry: source offset chan_off + dy * Ws + dx from a row's base position, and the
// tap offsets for the bounds test; kNoTap marks a zero column.
static int2 tab_entry(int chan_off, int dy, int dx, int Ws) {
  return make_int2(chan_off + dy * Ws + dx, (int)(((uint32_t)dy & 0xffffu) | ((uint32_t)dx << 16)));
}
static const int2 kNoTap = make_int2(0, 0x8000);   // dy = -32768

// N tile of a GEMM with N outputs: the whole of N up to 256, else tiles of 256.
static void n_tiles(int N, int* Np, int* ntn) {
  *Np = N <= 256 ? pad_to(N, 16) : 256;
  *ntn = (N + *Np - 1) / *Np;
}

bool tcg_supported(const bcrown_net* net) {
  for (int i = 0; i < net->L - 1; ++i) {
    const LayerDev& l = net->ly[i];
    if (l.kind != BCROWN_LAYER_CONV) {
      if (l.d_in > 65536 || l.d_out > 65536) return false;
      continue;
    }
    if (pad_to(l.in_c, 16) > 256 || pad_to(l.out_c, 16) > 256) return false;
    if (kp_bwd(l) > IM2COL_MAX_KP || kp_fwd(l) > IM2COL_MAX_KP) return false;
  }
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaGetLastError();
  return major == 10 && minor == 3;
}

size_t tcg_col_bytes_per_row(const bcrown_net* net, bool gather) {
  size_t b = 0;
  for (int i = 0; i < net->L - 1; ++i) {
    const LayerDev& l = net->ly[i];
    if (l.kind != BCROWN_LAYER_CONV) {
      b = std::max(b, (size_t)std::max(pad_to(l.d_in, 64), pad_to(l.d_out, 64)) * sizeof(__nv_bfloat16));
      continue;
    }
    if (gather) {   // conv operands are gathered in shared memory; the scatter form keeps P here
      if (scatter_form(l)) b = std::max(b, (size_t)l.in_c * l.k * l.k * l.out_h * l.out_w * sizeof(float));
      continue;
    }
    const size_t ph = (size_t)((l.in_h + l.stride - 1) / l.stride) * ((l.in_w + l.stride - 1) / l.stride);
    const size_t bwd = ph * kp_bwd(l);
    const size_t fwd = (size_t)l.out_h * l.out_w * kp_fwd(l);
    b = std::max(b, std::max(bwd, fwd) * sizeof(__nv_bfloat16));
  }
  return b;
}

// Fully connected layer i as the case of one position per row: B operands W^(i)^T (backward,
// [d_in][d_out]) and W^(i) (forward, [d_out][d_in]) in BF16, K padded to 64, N to whole tiles.
static int fc_prepare(const LayerDev& l, ConvTc* t, ConvTc::ConvW& c) {
  std::vector<float> w((size_t)l.d_out * l.d_in);
  if (cudaMemcpy(w.data(), l.W, w.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(BCROWN_ERR_CUDA, "copy of fc weights");
  n_tiles(l.d_in, &c.Np_b, &c.ntn_b);
  n_tiles(l.d_out, &c.Np_f, &c.ntn_f);
  c.Kp_b = pad_to(l.d_out, 64);
  c.Kp_f = pad_to(l.d_in, 64);
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  std::vector<__nv_bfloat16> wb((size_t)c.ntn_b * c.Np_b * c.Kp_b, zero), wf((size_t)c.ntn_f * c.Np_f * c.Kp_f, zero);
  for (int o = 0; o < l.d_out; ++o)
    for (int n = 0; n < l.d_in; ++n) {
      const __nv_bfloat16 v = __float2bfloat16_rn(w[(size_t)o * l.d_in + n]);
      wb[(size_t)n * c.Kp_b + o] = v;
      wf[(size_t)o * c.Kp_f + n] = v;
    }
  __nv_bfloat16 *db = nullptr, *df = nullptr;
  if (cudaMalloc(&db, wb.size() * 2) != cudaSuccess || cudaMalloc(&df, wf.size() * 2) != cudaSuccess)
    return fail(BCROWN_ERR_OOM, "bf16 fc weights");
  t->bufs.push_back(db);
  t->bufs.push_back(df);
  if (cudaMemcpy(db, wb.data(), wb.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(df, wf.data(), wf.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(BCROWN_ERR_CUDA, "bf16 fc weights upload");
  BC_CHECK(encode_map(&c.mb, db, c.ntn_b * c.Np_b, c.Kp_b, c.Np_b));
  BC_CHECK(encode_map(&c.mf, df, c.ntn_f * c.Np_f, c.Kp_f, c.Np_f));
  c.wb = db;
  c.wf = df;
  return BCROWN_OK;
}

static int tcg_prepare(bcrown_net* net, ConvTc* t) {
  if (t->ready) return BCROWN_OK;
  t->conv.assign(net->L + 1, ConvTc::ConvW());
  // layers 1 .. L-1 (the last one enters only through C W^(L))
  for (int i = 1; i <= net->L - 1; ++i) {
    const LayerDev& l = net->ly[i - 1];
    if (l.kind != BCROWN_LAYER_CONV) {
      BC_CHECK(fc_prepare(l, t, t->conv[i]));
      continue;
    }
    const int kk = l.k * l.k, s = l.stride, T = taps_per_axis(l);
    std::vector<float> w((size_t)l.out_c * l.in_c * kk);
    if (cudaMemcpy(w.data(), l.W, w.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(BCROWN_ERR_CUDA, "copy of conv weights");
    ConvTc::ConvW& c = t->conv[i];
    c.Np_b = pad_to(l.in_c, 16);
    c.Kp_b = kp_bwd(l);
    c.Np_f = pad_to(l.out_c, 16);
    c.Kp_f = kp_fwd(l);
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    std::vector<__nv_bfloat16> wb((size_t)s * s * c.Np_b * c.Kp_b, zero);
    std::vector<__nv_bfloat16> wf((size_t)c.Np_f * c.Kp_f, zero);
    std::vector<int2> tb((size_t)s * s * c.Kp_b, kNoTap), tf((size_t)c.Kp_f, kNoTap);
    // forward: K = (ci, ky, kx), source (oy * s - pad + ky, ox * s - pad + kx) of channel ci
    for (int co = 0; co < l.out_c; ++co)
      for (int ci = 0; ci < l.in_c; ++ci)
        for (int q = 0; q < kk; ++q)
          wf[(size_t)co * c.Kp_f + ci * kk + q] = __float2bfloat16_rn(w[((size_t)co * l.in_c + ci) * kk + q]);
    for (int ci = 0; ci < l.in_c; ++ci)
      for (int q = 0; q < kk; ++q) tf[ci * kk + q] = tab_entry(ci * l.in_h * l.in_w, q / l.k, q % l.k, l.in_w);
    // backward, phase (a, b): K = (co, dy, dx), tap (ky0 + s dy, kx0 + s dx), source q = (i + off - dy, ...)
    for (int a = 0; a < s; ++a)
      for (int b = 0; b < s; ++b) {
        const ConvPhase py = conv_phase(a, l.k, s, l.pad, l.in_h), px = conv_phase(b, l.k, s, l.pad, l.in_w);
        const size_t ph = (size_t)a * s + b;
        for (int co = 0; co < l.out_c; ++co)
          for (int dy = 0; dy < py.nk; ++dy)
            for (int dx = 0; dx < px.nk; ++dx) {
              const int K = co * T * T + dy * T + dx;
              const int ky = py.k0 + s * dy, kx = px.k0 + s * dx;
              tb[ph * c.Kp_b + K] = tab_entry(co * l.out_h * l.out_w, -dy, -dx, l.out_w);
              for (int ci = 0; ci < l.in_c; ++ci)
                wb[(ph * c.Np_b + ci) * c.Kp_b + K] =
                    __float2bfloat16_rn(w[((size_t)co * l.in_c + ci) * kk + ky * l.k + kx]);
            }
      }
    __nv_bfloat16 *db = nullptr, *df = nullptr;
    if (cudaMalloc(&db, wb.size() * 2) != cudaSuccess || cudaMalloc(&df, wf.size() * 2) != cudaSuccess ||
        cudaMalloc(&c.tab_b, tb.size() * sizeof(int2)) != cudaSuccess ||
        cudaMalloc(&c.tab_f, tf.size() * sizeof(int2)) != cudaSuccess)
      return fail(BCROWN_ERR_OOM, "bf16 conv weights");
    t->bufs.push_back(db);
    t->bufs.push_back(df);
    t->bufs.push_back(c.tab_b);
    t->bufs.push_back(c.tab_f);
    if (cudaMemcpy(db, wb.data(), wb.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(df, wf.data(), wf.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c.tab_b, tb.data(), tb.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c.tab_f, tf.data(), tf.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(BCROWN_ERR_CUDA, "bf16 conv weights upload");
    BC_CHECK(encode_map(&c.mb, db, s * s * c.Np_b, c.Kp_b, c.Np_b));
    BC_CHECK(encode_map(&c.mf, df, c.Np_f, c.Kp_f, c.Np_f));
    if (scatter_form(l)) {
      // B operand [n = (ci, ky, kx)][K = co], K-major; gather table: channel co at the position itself
      c.scat = true;
      c.Np_s = pad_to(l.in_c * kk, 16);
      c.Kp_s = pad_to(l.out_c, 64);
      std::vector<__nv_bfloat16> ws((size_t)c.Np_s * c.Kp_s, zero);
      std::vector<int2> ts((size_t)c.Kp_s, kNoTap);
      for (int co = 0; co < l.out_c; ++co) {
        ts[co] = tab_entry(co * l.out_h * l.out_w, 0, 0, l.out_w);
        for (int ci = 0; ci < l.in_c; ++ci)
          for (int q = 0; q < kk; ++q)
            ws[(size_t)(ci * kk + q) * c.Kp_s + co] = __float2bfloat16_rn(w[((size_t)co * l.in_c + ci) * kk + q]);
      }
      __nv_bfloat16* dws = nullptr;
      if (cudaMalloc(&dws, ws.size() * 2) != cudaSuccess || cudaMalloc(&c.tab_s, ts.size() * sizeof(int2)) != cudaSuccess)
        return fail(BCROWN_ERR_OOM, "bf16 conv weights (scatter form)");
      t->bufs.push_back(dws);
      t->bufs.push_back(c.tab_s);
      if (cudaMemcpy(dws, ws.data(), ws.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(c.tab_s, ts.data(), ts.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(BCROWN_ERR_CUDA, "bf16 conv weights upload (scatter form)");
      BC_CHECK(encode_map(&c.ms, dws, c.Np_s, c.Kp_s, c.Np_s));
    }
  }
  BC_CUDA(cudaFuncSetAttribute(k_tcg<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               tcg_smem(256, TCG_BIAS_MAX, true)));
  BC_CUDA(cudaFuncSetAttribute(k_tcg<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               tcg_smem(256, 256, true, IM2COL_MAX_KP)));
  BC_CUDA(cudaFuncSetAttribute(k_im2col, cudaFuncAttributeMaxDynamicSharedMemorySize, im2col_smem(IM2COL_MAX_KP)));
  t->ready = true;
  return BCROWN_OK;
}

// One im2col + GEMM pass (a phase of a backward layer, or the forward layer; for a fully
// connected layer, q.tab == nullptr, the operand is the source row converted to BF16).
static int tcg_pass(bcrown_net* net, const Im2colPass& q, const CUtensorMap& mB, const TcgOut& o, const float* src,
                    float* dst, const float* bias, char* col, size_t col_bytes, cudaStream_t s) {
  if (q.M <= 0) return BCROWN_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (q.M + 127) / 128 * o.ntn;
  const int gps = net->launch_now.grid_per_sm > 0 ? net->launch_now.grid_per_sm : 2;   // CTAs per SM
  const int grid = (int)std::min<long long>(ntiles, (long long)gps * sms);
  if (q.tab && tcg_gather(net)) {
    // conv layers: the gather warps build the operand in shared memory (mapA unused)
    const int smem = tcg_smem(o.Np, o.N, bias != nullptr, q.Kp);
    k_tcg<true><<<grid, TcgRoles<true>::THREADS, smem, s>>>(mB, mB, o, q, src, dst, bias, net->status);
    ++g_launches;
    BC_CUDA(cudaGetLastError());
    return BCROWN_OK;
  }
  if ((size_t)q.M * q.Kp * sizeof(__nv_bfloat16) > col_bytes) return fail(BCROWN_ERR_OOM, "im2col workspace too small");
  __nv_bfloat16* cb = reinterpret_cast<__nv_bfloat16*>(col);
  if (q.tab)
    k_im2col<<<(unsigned)((q.M + IM2COL_ROWS - 1) / IM2COL_ROWS), 256, im2col_smem(q.Kp), s>>>(q, src, cb);
  else
    k_rows_bf16<<<(unsigned)((q.M * (q.Kp / 8) + 255) / 256), 256, 0, s>>>(q.M, q.d_src, q.Kp, src, cb);
  ++g_launches;
  CUtensorMap mA;
  BC_CHECK(encode_map(&mA, cb, (int)q.M, q.Kp, 128));
  const int smem = tcg_smem(o.Np, o.N, bias != nullptr);
  k_tcg<false><<<grid, TcgRoles<false>::THREADS, smem, s>>>(mA, mB, o, q, src, dst, bias, net->status);
  ++g_launches;
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

int tcg_conv(bcrown_net* net, int i, bool fwd, int R, const float* src, float* dst, const float* bias, char* col,
             size_t col_bytes, cudaStream_t s) {
  ConvTc* t = conv_of(net);
  BC_CHECK(tcg_prepare(net, t));
  const LayerDev& l = net->ly[i - 1];
  const ConvTc::ConvW& c = t->conv[i];
  if (R <= 0) return BCROWN_OK;
  if (l.kind != BCROWN_LAYER_CONV) {
    const int dsrc = fwd ? l.d_in : l.d_out, ddst = fwd ? l.d_out : l.d_in;
    const int Kp = fwd ? c.Kp_f : c.Kp_b;
    const Im2colPass q{(long long)R, 1, 1, 0, 0, 0, 1, 1, dsrc, Kp, nullptr};
    // Few row tiles (a small chunk, a long K): narrower N tiles until the grid covers the SMs;
    // each halving still divides the padded rows of the weight operand.
    int Np = fwd ? c.Np_f : c.Np_b;
    const int rows = Np * (fwd ? c.ntn_f : c.ntn_b);
    const long long mt = ((long long)R + 127) / 128;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    while (Np % 32 == 0 && Np > 32 && mt * ((ddst + Np - 1) / Np) < sms) Np /= 2;
    CUtensorMap mB = fwd ? c.mf : c.mb;
    if (Np != (fwd ? c.Np_f : c.Np_b)) BC_CHECK(encode_map(&mB, fwd ? c.wf : c.wb, rows, Kp, Np));
    const TcgOut o{q.M, ddst, Np, (ddst + Np - 1) / Np, Kp / 64, 0, 1, 1, 0, 0, 1, 1, 1, (long long)ddst};
    return tcg_pass(net, q, mB, o, src, dst, fwd ? bias : nullptr, col, col_bytes, s);
  }
  if (fwd) {
    const int P = l.out_h * l.out_w;
    const Im2colPass q{(long long)R * P, P, l.out_w, l.stride, -l.pad, -l.pad, l.in_h, l.in_w, l.d_in, c.Kp_f, c.tab_f};
    const TcgOut o{q.M, l.out_c, c.Np_f, 1, c.Kp_f / 64, 0, P, l.out_w, 0, 0, 1, l.out_w, P, (long long)l.d_out};
    return tcg_pass(net, q, c.mf, o, src, dst, bias, col, col_bytes, s);
  }
  if (c.scat && tcg_gather(net)) {
    const int P = l.out_h * l.out_w, Ns = l.in_c * l.k * l.k;
    if ((size_t)R * Ns * P * sizeof(float) > col_bytes) return fail(BCROWN_ERR_OOM, "scatter-form workspace too small");
    float* tmp = reinterpret_cast<float*>(col);
    const Im2colPass q{(long long)R * P, P, l.out_w, 1, 0, 0, l.out_h, l.out_w, l.d_out, c.Kp_s, c.tab_s};
    const TcgOut o{q.M, Ns, c.Np_s, 1, c.Kp_s / 64, 0, P, l.out_w, 0, 0, 1, l.out_w, P, (long long)Ns * P};
    BC_CHECK(tcg_pass(net, q, c.ms, o, src, tmp, nullptr, col, col_bytes, s));
    const Col2im g{l.in_c, l.in_h, l.in_w, l.k, l.stride, l.pad, l.out_h, l.out_w};
    const long long total = (long long)R * l.d_in;
    k_col2im<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(total, g, tmp, dst, l.d_in);
    ++g_launches;
    BC_CUDA(cudaGetLastError());
    return BCROWN_OK;
  }
  const int st = l.stride;
  for (int a = 0; a < st; ++a)
    for (int b = 0; b < st; ++b) {
      const ConvPhase py = conv_phase(a, l.k, st, l.pad, l.in_h), px = conv_phase(b, l.k, st, l.pad, l.in_w);
      const int Pm = py.n * px.n;
      if (Pm == 0) continue;
      const int ph = a * st + b;
      const Im2colPass q{(long long)R * Pm, Pm, px.n, 1, py.off, px.off, l.out_h, l.out_w, l.d_out, c.Kp_b,
                         c.tab_b + (size_t)ph * c.Kp_b};
      const TcgOut o{q.M, l.in_c, c.Np_b, 1, c.Kp_b / 64, ph * c.Np_b, Pm, px.n, a, b, st, l.in_w,
                     l.in_h * l.in_w, (long long)l.d_in};
      BC_CHECK(tcg_pass(net, q, c.mb, o, src, dst, nullptr, col, col_bytes, s));
    }
  return BCROWN_OK;
}

void tcg_release(const bcrown_net* net) {
  std::lock_guard<std::mutex> g(g_conv_mu);
  for (size_t i = 0; i < g_conv.size(); ++i)
    if (g_conv[i].first == net) {
      for (void* b : g_conv[i].second->bufs) cudaFree(b);
      delete g_conv[i].second;
      g_conv.erase(g_conv.begin() + i);
      return;
    }
}

}  // namespace bcrown
