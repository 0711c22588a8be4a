// BF16 layer-by-layer bound pass (sm_103a: tcgen05 + TMA) for the networks the fused kernel does
// not take: convolutional networks and fully connected layers wider than 256 neurons.
//
// The recursion of Theorem 3.1 (Eq. definition_A) runs one contraction per launch, and each
// launch's epilogue takes the next step of the recursion on the accumulator it just produced,
// so no FP32 intermediate goes through HBM:
//
//   backward, layer i:  A^(i-1) = Lambda^(i) W^(i)   (a transposed convolution: one GEMM per
//                       stride phase; a fully connected layer: one GEMM)
//                       epilogue: the relaxation of layer i-1 (Lemma 2.1 / Eq. definition_D with
//                       split overriding stability), Lambda^(i-1) = A D + beta S, the bias sums
//                       c += Lambda b + A lambda, and Lambda^(i-1) stored in BF16 as the next
//                       GEMM's operand; for i = 1 the concretisation over the box (Eq.
//                       beta_crown_lp) and x* (x_lo where A^(0) >= 0, else x_hi).
//   forward (adjoint), layer i:  zhat^(i) = W^(i) h^(i-1) + b^(i)
//                       epilogue: dalpha = A zhat (unstable, unsplit, A >= 0), dbeta = S zhat,
//                       h^(i) = D zhat + lambda stored in BF16 as the next operand.
//
// Activations are BF16 in NHWC order (channels innermost, padded to a multiple of 8), so that the
// GEMM operand -- rows = (subdomain row, output position), K = (tap, channel) -- is gathered into
// shared memory in 16-byte pieces of 8 channels, one load each; gather warps write it in the
// 128-byte-swizzled K-major layout the MMA reads, TMA streams the weights, one thread issues the
// MMAs into one of three TMEM accumulators (two for 256-column tiles), and three groups of 4
// epilogue warps read them with tcgen05.ld, each group every third tile, so that up to three
// tiles' epilogues run at once (576 threads: 12 epilogue, 1 TMA, 1 MMA and 4 gather warps).
// The bias sums of each row are written as partial sums (one slot per position block and column
// group) and added in a fixed order at the end, so the result does not depend on scheduling.
// A at the unstable neurons is stashed in BF16, laid out like alpha, for the adjoint pass; its
// sign is kept even where it rounds to zero, so both passes take the same relaxation branch.
//
// Every mbarrier wait is bounded; on expiry the kernel records BCROWN_ERR_TIMEOUT, raises its
// abort flag, waits (bounded) for its copies in flight, frees TMEM and returns.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "layer_tc.cuh"
#include "tc_ptx.cuh"

namespace bcrown {

extern std::atomic<long long> g_launches;

namespace lt {

using namespace tc;

constexpr int NS = 4;                       // pipeline stages (A: 128 x 64, B: Np x 64)
// Warp roles.  Gathered A operand: 12 epilogue warps (three groups of 4, every third tile) and 4
// gather warps (one per ring slot).  A operand by TMA: 16 epilogue warps (four groups).  Both with
// the TMA and the MMA warp: 18 warps, which leaves 96 registers a thread.
// LT_TA_GROUPS: epilogue groups of the TMA form (4: 18 warps, 96 registers a thread -- 5 warps on
// two of the SM's four schedulers; 3: 14 warps, 128 registers).
#ifndef LT_TA_GROUPS
#define LT_TA_GROUPS 4
#endif
#ifndef LT_FWD_PREFETCH
#define LT_FWD_PREFETCH 0
#endif
template <bool TA>
struct LtRoles {
  static constexpr int EPI = TA ? 4 * LT_TA_GROUPS : 12;   // epilogue warps
  static constexpr int NGRP = EPI / 4;       // epilogue groups, one TMEM accumulator each
  static constexpr int GW = TA ? 0 : NS;     // gather warps, one per ring slot
  static constexpr int TMA_W = EPI, MMA_W = EPI + 1, GATHER0 = EPI + 2;
  static constexpr int THREADS = (EPI + 2 + GW) * 32;
};
constexpr int MAX_NP = 256;
constexpr int MAX_KP = 2048;
constexpr int MAX_KEEP = 6;                 // splits of a row kept in registers per tile

enum { EPI_RELAX = 0, EPI_CONCRETIZE = 1, EPI_FWD = 2 };

// One GEMM launch: M = (row, position of this pass) pairs, N = output channels (or, for a fully
// connected pass over a map, NHWC output indices), K = (tap, input channel).
struct Pass {
  long long M;
  int Pm, nJ;                // positions per row in this pass; the pass grid's width
  int N, Np, ntn, nkb, brow; // N in ntn tiles of Np; K blocks; first row of the B matrix in its map
  // gather source: NHWC BF16 map, row stride src_stride elements; the base position of
  // (row, pp = i * nJ + j) is (i * ms + cy, j * ms + cx); table entries per 8-channel chunk of K
  const __nv_bfloat16* src;
  long long src_stride;
  int Hs, Ws, Cps, ms, cy, cx, kchunks;
  const int2* tab;           // [kchunks]: {element offset, dy & 0xffff | dx << 16}; null: chunk
                             // kc is elements 8 kc .. 8 kc + 7 of the row (fully connected)
  // output position of (row, pp): (oa + os * i) * Wo + ob + os * j; npos: position from n
  int oa, ob, os, Wo, npos;
  int Co, HWo, Cpo;          // output map: channels, positions, padded channels
  __nv_bfloat16* dst;        // NHWC BF16 output (null: none)
  long long dst_stride;
  int layer;                 // hidden layer of the epilogue (0: the input)
  long long hoff;            // its first global hidden index
  const float* bias;         // its bias, expanded per neuron (channel-major)
  const float* bnhwc;        // its bias in NHWC order (padded channels 0)
  const uint32_t* ntab;      // its neurons in NHWC order, property 0 (stride Ctx::NH per property):
                             // code (0 inactive, 1 active, 2 unstable) | rank among the unstable << 2
  int slot0;                 // first partial-sum slot of this pass
  // A operand by TMA instead of the gather warps: 0 gathered; 4: one box [64 channels][bw][bh][br]
  // of the NHWC source per (tap, 64-channel block) -- an M tile is br rows x bh x bw positions;
  // 2: one box [64][128 rows] of a fully connected pass's linear source; 8: a source of 8 (padded)
  // channels, one unswizzled box [8][bw][bh][br] per tap, 8 taps per K block
  int ta = 0, bw = 0, bh = 0, br = 0;
  const int4* ktab = nullptr;   // ta == 4: per K block {first channel, dy, dx, tap in use};
                                // ta == 8: the same per tap (8 per K block)
};

// Per-call context of the epilogues.
struct Ctx {
  int r0, R, K, P, H, d0, S;
  BatchView bt;
  Tables tb;
  const float* x_lo;
  const float* x_hi;
  const float* alpha;
  const float* beta;
  int64_t n_alpha, n_beta;
  float* dalpha;
  float* dbeta;
  __nv_bfloat16* stash;      // A at the unstable neurons (alpha layout), or null
  float* cpart;              // [R][S] partial sums of c
  int* status;
  // built once per call by k_lt_rows (rows indexed from 0 = the call's first row)
  const int4* rowinfo;       // [B*K]: {abase lo, abase hi, bbase, prop | valid << 31}
  const uint32_t* ssplit;    // [B][64]: a subdomain's splits sorted by layer, j | t << 20 | (S = +1) << 26
  const int* slayer;         // [B][L + 1]: start of layer l's entries in the subdomain's sorted list
  int L;
  long long NH;              // entries per property in the NHWC neuron table (all hidden layers)
  const float2* chord;       // [P][H]: upper chord (slope, intercept) of the property's unstable
                             // neuron of each rank
};

// Packed split entry of the sorted lists (neuron index j < 2^20, list position t < 64).
__device__ __forceinline__ int sp_j(uint32_t e) { return (int)(e & 0xFFFFFu); }
__device__ __forceinline__ int sp_t(uint32_t e) { return (int)((e >> 20) & 63u); }
__device__ __forceinline__ int sp_s(uint32_t e) { return (e >> 26) & 1u ? 1 : -1; }

__device__ __forceinline__ bool lt_wait(uint64_t* b, uint32_t parity, volatile int* abort, int* status) {
  if (mbar_try(b, parity)) return true;
  long long t0 = clock64();
  while (true) {
    // try_wait without a suspend-time hint: the hardware's own short wait window, then a re-poll
    if (mbar_try(b, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > 4000000000LL) {
      atomicCAS(status, 0, BCROWN_ERR_TIMEOUT);
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ uint4 ldg_nc_v4(const void* p, bool pred) {
  uint4 v;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\tmov.b32 %0, 0;\n\tmov.b32 %1, 0;\n\tmov.b32 %2, 0;\n\t"
      "mov.b32 %3, 0;\n\t@q ld.global.nc.v4.b32 {%0, %1, %2, %3}, [%4];\n\t}"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "r"((uint32_t)pred)
      : "memory");
  return v;
}

// BF16 of a, rounded to nearest, keeping a < 0 negative (the smallest negative subnormal where it
// would round to -0), so a sign test on the stash agrees with the one on a.
__device__ __forceinline__ __nv_bfloat16 bf16_signed(float a) {
  __nv_bfloat16 h = __float2bfloat16_rn(a);
  if (a < 0.f && !(__bfloat162float(h) < 0.f)) h = __ushort_as_bfloat16((unsigned short)0x8001u);
  return h;
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float lt_warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int MODE, bool TA>
__global__ void __launch_bounds__(LtRoles<TA>::THREADS, 1)
    k_lt(const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapA, const Pass ps,
         const Ctx cx) {
  using RL = LtRoles<TA>;
  const long long M = ps.M;
  const int Np = ps.Np, nkb = ps.nkb;
  extern __shared__ __align__(1024) uint8_t lsm_raw[];
  const uint32_t pad = (1024u - (su32(lsm_raw) & 1023u)) & 1023u;
  uint8_t* base = lsm_raw + pad;
  const int bbytes = Np * 128;
  uint8_t* sA = base;                                  // NS x 16 KB
  uint8_t* sB = base + NS * 16384;                     // NS x Np * 128
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + NS * bbytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + NS;
  uint64_t* acc_full = bars + 2 * NS;        // up to 4 accumulators
  uint64_t* acc_empty = bars + 2 * NS + 4;
  uint32_t* tbase_sm = reinterpret_cast<uint32_t*>(bars + 2 * NS + 8);
  volatile int* abort = reinterpret_cast<volatile int*>(tbase_sm + 1);
  int2* stab = reinterpret_cast<int2*>(bars + 32);     // 256 bytes past the barriers
  float* sbias = reinterpret_cast<float*>(stab + MAX_KP / 8);   // conv passes: the layer's channel biases
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long ntiles = (M + 127) / 128 * ps.ntn;   // tile = m tile * ntn + n tile
  // accumulators in use: one per epilogue group, as many groups as their Np columns each fit in
  // TMEM's 512 (the other groups then idle)
  const int ngrp = RL::NGRP * Np <= 512 ? RL::NGRP : (3 * Np <= 512 ? min(3, RL::NGRP) : 2);
  const uint32_t need = (uint32_t)(ngrp * Np);
  const uint32_t tcols = need <= 32 ? 32u : (need <= 64 ? 64u : (need <= 128 ? 128u : (need <= 256 ? 256u : 512u)));
  if (threadIdx.x == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(&full[i], TA ? 1 : 2);   // the TMA transaction (and the stage's gather warp)
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < RL::NGRP; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);   // the 4 warps of the epilogue group of buffer i
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == RL::MMA_W) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tbase_sm)), "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase_sm;

  if (warp == RL::TMA_W) {
    // ------------------------------------------------------------ weights (B) by TMA, and A with TA
    // One thread issues every copy, so its loop holds no division and no global load per K
    // block: the tile's coordinates are worked out once per tile, the tap table is in shared
    // memory (the gathering kernel's table space).
    int4* sktab = reinterpret_cast<int4*>(stab);
    if (TA && (ps.ta == 4 || ps.ta == 8)) {
      for (int k = lane; k < (ps.ta == 8 ? 8 * nkb : nkb); k += 32) sktab[k] = ps.ktab[k];
      __syncwarp();
    }
    if (lane == 0) {
      uint32_t seq = 0;
      int st = 0;
      uint32_t ph = 0;   // parity of the current pass over the ring
      bool ok = true;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long mt = tile / ps.ntn;
        const int brow = ps.brow + (int)(tile - mt * ps.ntn) * Np;
        int ax = 0, ay = 0, ar = 0;   // TA: the box origin of the tile's first position, tap 0
        if constexpr (TA) {
          const long long m0 = mt * 128;
          if (ps.ta == 2) {
            ar = (int)m0;
          } else {
            const long long r0 = m0 / ps.Pm;
            const int pp0 = (int)(m0 - r0 * ps.Pm);
            const int i0 = pp0 / ps.nJ;
            ax = (pp0 - i0 * ps.nJ) * ps.ms + ps.cx;
            ay = i0 * ps.ms + ps.cy;
            ar = (int)r0;
          }
        }
        for (int kb = 0; kb < nkb; ++kb, ++seq) {
          if (!lt_wait(&empty[st], ph ^ 1, abort, cx.status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[st], (TA ? 16384u : 0u) + (uint32_t)bbytes);
          if constexpr (TA) {
            if (ps.ta == 2) {
              tma_load_2d(sA + st * 16384, &mapA, kb * 64, ar, &full[st]);
            } else if (ps.ta == 8) {
              // 8 channels per tap: the K block is 8 taps, one box of 16-byte rows each, 2 KB apart
#pragma unroll 1
              for (int j = 0; j < 8; ++j) {
                const int4 kt = sktab[kb * 8 + j];
                const int y = kt.w ? ay + kt.y : -(1 << 20);
                tma_load_4d(sA + st * 16384 + j * 2048, &mapA, 0, ax + kt.z, y, ar, &full[st]);
              }
            } else {
              const int4 kt = sktab[kb];
              // a K block past the phase's taps reads a box outside the map: zeros
              const int y = kt.w ? ay + kt.y : -(1 << 20);
              tma_load_4d(sA + st * 16384, &mapA, kt.x, ax + kt.z, y, ar, &full[st]);
            }
          }
          tma_load_2d(sB + st * bbytes, &mapB, kb * 64, brow, &full[st]);
          if (++st == NS) st = 0, ph ^= 1;
        }
      }
      if (!ok) {
        for (uint32_t q = (seq > NS ? seq - NS : 0); q < seq; ++q) {
          long long t0 = clock64();
          while (!mbar_try(&full[q % NS], (q / NS) & 1) && clock64() - t0 < 200000000LL) {
          }
        }
      }
    }
  } else if (warp == RL::MMA_W) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t seq = 0, accseq = 0;
      bool ok = true;
      const uint32_t idesc = idesc_bf16(Np);
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++accseq) {
        const int buf = (int)(accseq % (uint32_t)ngrp);
        if (!lt_wait(&acc_empty[buf], ((accseq / (uint32_t)ngrp) & 1) ^ 1, abort, cx.status)) break;
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * Np);
        for (int kb = 0; kb < nkb; ++kb, ++seq) {
          const int st = seq % NS;
          if (!lt_wait(&full[st], (seq / NS) & 1, abort, cx.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (TA && ps.ta == 8)   // A without swizzle: core matrices 128 B apart along M, 2 KB along K
            umma_kblock_astep(dt, sdesc_plain(su32(sA + st * 16384), 2048, 128), sdesc(su32(sB + st * bbytes)),
                              idesc, kb != 0 ? 1u : 0u, 4096 >> 4);
          else
            umma_kblock(dt, sdesc(su32(sA + st * 16384)), sdesc(su32(sB + st * bbytes)), idesc, kb != 0 ? 1u : 0u);
          umma_commit(&empty[st]);
        }
        if (!ok) break;
        umma_commit(&acc_full[buf]);
      }
    }
  } else if (!TA && warp >= RL::GATHER0) {
    // ------------------------------------------------------------ operand (A) gather
    // ring slot g takes sequence numbers g, g + NS, ... of the (tile, K block) order; this warp
    // writes chunks CPW part .. CPW part + CPW - 1 (of 8 per row) of its slot's stages
    const int g = (warp - RL::GATHER0) % NS, part = 0;
    constexpr int CPW = 8;
    constexpr int GW = RL::GW > 0 ? RL::GW : 1;
    const bool linear = ps.tab == nullptr;
    if (!linear)
      for (int k = threadIdx.x - RL::GATHER0 * 32; k < ps.kchunks; k += GW * 32) stab[k] = ps.tab[k];
    asm volatile("bar.sync 2, %0;" ::"n"(GW * 32) : "memory");
    uint32_t seq = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const __nv_bfloat16* srow[4];
      int y0[4], x0[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long m = tile / ps.ntn * 128 + lane + 32 * q;
        const bool mv = m < M;
        const long long r = mv ? m / ps.Pm : 0;
        const int pp = mv ? (int)(m - r * ps.Pm) : 0;
        const int i = pp / ps.nJ, j = pp - (pp / ps.nJ) * ps.nJ;
        y0[q] = mv ? i * ps.ms + ps.cy : -32768;
        x0[q] = j * ps.ms + ps.cx;
        srow[q] = ps.src + r * ps.src_stride + (mv ? ((long long)y0[q] * ps.Ws + x0[q]) * ps.Cps : 0);
      }
      for (int kb = 0; kb < nkb; ++kb, ++seq) {
        if ((int)(seq % NS) != g) continue;
        int okw = 1;
        if (lane == 0) okw = lt_wait(&empty[g], ((seq / NS) & 1) ^ 1, abort, cx.status) ? 1 : 0;
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) {
          ok = false;
          break;
        }
        uint8_t* stage = sA + g * 16384;
        // 4 chunks (of 4 rows each) in flight at a time: 16 loads of 16 bytes per lane
#pragma unroll
        for (int c0 = 0; c0 < CPW; c0 += 4) {
          uint4 v[4][4];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int kc = kb * 8 + CPW * part + c0 + cc;
            const int2 t = kc < ps.kchunks ? (linear ? make_int2(8 * kc, 0) : stab[kc]) : make_int2(0, 0x8000);
            const int dy = (int)(short)(t.y & 0xffff), dx = t.y >> 16;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const bool in = (unsigned)(y0[q] + dy) < (unsigned)ps.Hs && (unsigned)(x0[q] + dx) < (unsigned)ps.Ws;
              v[cc][q] = ldg_nc_v4(srow[q] + t.x, in);
            }
          }
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int c = CPW * part + c0 + cc;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int m = lane + 32 * q;
              *reinterpret_cast<uint4*>(stage + m * 128 + ((c ^ (m & 7)) << 4)) = v[cc][q];
            }
          }
        }
        fence_proxy_async();   // generic-proxy stores of the stage, before the MMA reads it
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[g]);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // ngrp groups of 4 warps take every ngrp-th tile (group g: accumulator buffer g), so that
    // their tiles' epilogues overlap; warp w of a group reads TMEM lanes 32 (w % 4) .. + 31 (M
    // rows) and every column chunk of 8
    const int q4 = warp & 3, eg = warp >> 2;
    uint32_t accseq = eg;   // this group takes the CTA's tiles eg, eg + ngrp, ...
    const bool sb_smem = MODE != EPI_CONCRETIZE && !ps.npos && ps.Cpo <= MAX_NP;
    if (sb_smem) {
      // a conv layer's bias is per channel: bnhwc at position 0
      for (int c = threadIdx.x; c < MAX_NP; c += RL::EPI * 32) sbias[c] = c < ps.Cpo ? ps.bnhwc[c] : 0.f;
      asm volatile("bar.sync 1, %0;" ::"n"(RL::EPI * 32) : "memory");
    }
    const bool warp_sum_ok = (ps.Pm & 31) == 0;   // 32 lanes = 32 positions of one row
    for (long long tile = blockIdx.x + (long long)eg * gridDim.x; eg < ngrp && tile < ntiles;
         tile += (long long)ngrp * gridDim.x, accseq += ngrp) {
      const int buf = eg;
      const int nt = (int)(tile % ps.ntn);
      const long long m = tile / ps.ntn * 128 + 32 * q4 + lane;
      const bool mv = m < M;
      const int rl = mv ? (int)(m / ps.Pm) : 0;              // row within the chunk
      const int pp = mv ? (int)(m - (long long)rl * ps.Pm) : 0;
      const int pi = pp / ps.nJ, pj = pp - (pp / ps.nJ) * ps.nJ;
      const int pm = ps.npos ? 0 : (ps.oa + ps.os * pi) * ps.Wo + ps.ob + ps.os * pj;
      // the row: subdomain b, spec k, property p (one 16-byte load of the row table)
      const int r = cx.r0 + rl;
      const int b = r / cx.K;
      const int4 ri = mv ? cx.rowinfo[r] : make_int4(0, 0, 0, 0);
      const long long abase = ((long long)(uint32_t)ri.y << 32) | (uint32_t)ri.x;
      const long long bbase = ri.z;
      const int prop = ri.w & 0x7FFFFFFF;
      const bool rv = mv && (ri.w < 0);
      // the row's splits in this layer that fall on this thread's elements of the tile
      // kept splits, packed: n | t << 20 | (S == +1) << 27 (n < 2^20, t < 64); -1: none
      int kp_[MAX_KEEP];
#pragma unroll
      for (int q = 0; q < MAX_KEEP; ++q) kp_[q] = -1;
      int nkeep = 0;
      bool many = false;
      int s0 = 0, s1 = 0;
      const int nlo = nt * Np, nhi = min(nt * Np + Np, ps.N);
      if (rv && MODE != EPI_CONCRETIZE) {
        const int* sl = cx.slayer + (size_t)b * (cx.L + 1) + ps.layer;
        s0 = b * BCROWN_MAX_SPLITS + sl[0];
        s1 = b * BCROWN_MAX_SPLITS + sl[1];
        for (int q = s0; q < s1; ++q) {
          const uint32_t e = cx.ssplit[q];
          const int jn = sp_j(e);
          const int c_s = jn / ps.HWo, p_s = jn - c_s * ps.HWo;
          const int nn = ps.npos ? p_s * ps.Cpo + c_s : c_s;   // the element's n
          const bool mine = nn >= nlo && nn < nhi && (ps.npos || p_s == pm);
          if (!mine) continue;
          // register slot nkeep (constant indices keep the arrays in registers)
#pragma unroll
          for (int u = 0; u < MAX_KEEP; ++u)
            if (u == nkeep) {
              kp_[u] = nn | (sp_t(e) << 20) | ((sp_s(e) == 1 ? 1 : 0) << 27);
            }
          if (nkeep < MAX_KEEP) ++nkeep;
          else many = true;
        }
      }
      int okw = 1;
      if (lane == 0) okw = lt_wait(&acc_full[buf], (accseq / (uint32_t)ngrp) & 1, abort, cx.status) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      tc_fence_after();
      float acc = 0.f;
      // per-tile bases: the row's alpha block (and stash, gradient), the property's tables
      const float* alpha_r = cx.alpha + abase;
      __nv_bfloat16* stash_r = cx.stash ? cx.stash + abase : nullptr;
      float* dalpha_r = cx.dalpha ? cx.dalpha + abase : nullptr;
      const float2* chord_p = cx.chord + (size_t)prop * cx.H;
      const uint32_t* tab_p = MODE == EPI_CONCRETIZE ? nullptr : ps.ntab + (size_t)prop * cx.NH;
      // the chunk's NHWC index: conv, (pm, channels nb ..); fully connected over a map, nb itself
      auto nhwc = [&](int nb) -> long long { return ps.npos ? (long long)nb : (long long)pm * ps.Cpo + nb; };
      // the neuron entries of a chunk are loaded one chunk ahead, so that the dependent loads of
      // the unstable elements' operands do not wait for them as well
      // (not in the adjoint epilogue unless LT_FWD_PREFETCH: its registers are at the limit, and
      // the spills it then needs cost more than the prefetch gains: 3.03k against 3.12k subdomains/s)
      constexpr bool PF = MODE == EPI_RELAX || (MODE == EPI_FWD && LT_FWD_PREFETCH);
      uint4 tn0 = make_uint4(0, 0, 0, 0), tn1 = tn0;
      if (PF && mv && nlo < ps.N) {
        const uint4* tp = reinterpret_cast<const uint4*>(tab_p + nhwc(nlo));
        tn0 = tp[0], tn1 = tp[1];
      }
      for (int n0 = 0; n0 < Np; n0 += 8) {
        // 8 columns per step (one 16-byte chunk of the BF16 NHWC output): the element loop's
        // registers fit the 96 a thread has at 18 warps per SM
        uint4 t0 = tn0, t1 = tn1;
        if (PF && mv && n0 + 8 < Np && nlo + n0 + 8 < ps.N) {
          const uint4* tp = reinterpret_cast<const uint4*>(tab_p + nhwc(nlo + n0 + 8));
          tn0 = tp[0], tn1 = tp[1];
        }
        if (!PF && MODE != EPI_CONCRETIZE && mv && nlo + n0 < ps.N) {
          const uint4* tp = reinterpret_cast<const uint4*>(tab_p + nhwc(nlo + n0));
          t0 = tp[0], t1 = tp[1];
        }
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(buf * Np + n0), v);
        const int nb = nlo + n0;   // first n of the chunk
        if (mv && nb < ps.N) {
        uint32_t o2[4];            // the chunk's results, packed in BF16 pairs
        const long long nn0 = nhwc(nb);
        const int lim = ps.npos ? ps.N : ps.Cpo;   // elements of the chunk that exist in the map
        if (MODE == EPI_CONCRETIZE) {
          float o[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int n = nb + e;
            o[e] = 0.f;
            if (!rv || n >= ps.Co) continue;
            const int jl = n * ps.HWo + pm;   // input coordinate (channel-major)
            const float a = v[e];
            const float xl = cx.x_lo[(size_t)prop * cx.d0 + jl], xh = cx.x_hi[(size_t)prop * cx.d0 + jl];
            acc += fminf(a * xl, a * xh);
            o[e] = a >= 0.f ? xl : xh;   // x* minimises A^(0) x over the box
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) o2[e] = pack2(o[2 * e], o[2 * e + 1]);
        } else {
          // the 8 elements' neuron entries (loaded with the previous chunk)
          uint32_t ent[8];
          ent[0] = t0.x, ent[1] = t0.y, ent[2] = t0.z, ent[3] = t0.w;
          ent[4] = t1.x, ent[5] = t1.y, ent[6] = t1.z, ent[7] = t1.w;
          // elements of the chunk with a split of the row (all of them when the row's list overflowed)
          uint32_t smask = many ? 0xFFu : 0u;
          if (nkeep > 0) {   // most threads hold no split in the tile: skip the scan
#pragma unroll
            for (int q = 0; q < MAX_KEEP; ++q)
              if (q < nkeep && (unsigned)((kp_[q] & 0xFFFFF) - nb) < 8u) smask |= 1u << ((kp_[q] & 0xFFFFF) - nb);
          }
          float o[8];
#pragma unroll
          for (int hb = 0; hb < 8; hb += 4) {
            // the unstable elements' operands of 4 elements, issued together before any is used:
            // alpha, the chord and, in the adjoint, the stash
            float al[4], st[4], bv[4];
            float2 ch[4];
#pragma unroll
            for (int uu = 0; uu < 4; ++uu) {
              const int u = hb + uu;
              const bool un = rv && nb + u < lim && (ent[u] & 3u) == CODE_UNSTABLE;
              const int rk = (int)(ent[u] >> 2);
              al[uu] = un ? alpha_r[rk] : 0.f;
              ch[uu] = un ? chord_p[rk] : make_float2(0.f, 0.f);
              st[uu] = (MODE == EPI_FWD && un) ? __bfloat162float(stash_r[rk]) : 0.f;
              // biases: a conv layer's are per channel (shared memory, up to MAX_NP channels); a
              // fully connected pass's per n, and a wider layer's channels from global memory
              if (MODE != EPI_FWD || !sb_smem)
                bv[uu] = ps.npos ? ps.bnhwc[nn0 + u]
                                 : (sb_smem ? sbias[min(nb + u, MAX_NP - 1)] : (nb + u < lim ? ps.bnhwc[nb + u] : 0.f));
            }
            if (MODE == EPI_FWD && sb_smem) {
              // the adjoint: 4 channel biases in one shared-memory load (nb + hb + 3 < MAX_NP); in the
              // relaxation the 4 registers this holds at once would spill
              const float4 b4 = *reinterpret_cast<const float4*>(sbias + nb + hb);
              bv[0] = b4.x, bv[1] = b4.y, bv[2] = b4.z, bv[3] = b4.w;
            }
#pragma unroll
            for (int uu = 0; uu < 4; ++uu) {
              const int u = hb + uu;
              const int n = nb + u;
              const bool valid = rv && n < lim;
              const int code = (int)(ent[u] & 3u);
              const int rk = (int)(ent[u] >> 2);
              // split of this element (sign s, list position t): rare
              int s = 0, ts = 0;
              if (valid && ((smask >> u) & 1u)) {
                int c = n, p = pm;
                if (ps.npos) {
                  p = n / ps.Cpo;
                  c = n - p * ps.Cpo;
                }
                const int jl = c * ps.HWo + p;   // neuron of the layer (channel-major)
#pragma unroll
                for (int q = 0; q < MAX_KEEP; ++q)
                  if (q < nkeep && (kp_[q] & 0xFFFFF) == n) {
                    s = (kp_[q] >> 27) & 1 ? 1 : -1;
                    ts = (kp_[q] >> 20) & 127;
                  }
                if (many && s == 0)
                  for (int q = s0; q < s1; ++q) {
                    const uint32_t e2 = cx.ssplit[q];
                    if (sp_j(e2) == jl) {
                      s = sp_s(e2);
                      ts = sp_t(e2);
                    }
                  }
              }
              const bool unst = valid && s == 0 && code == CODE_UNSTABLE;
              if (MODE == EPI_RELAX) {
                const float a = v[u];
                float D = code == CODE_ACTIVE ? 1.f : 0.f, lm = 0.f, bs = 0.f;
                if (unst) {
                  if (a >= 0.f) {
                    D = __saturatef(al[uu]);
                  } else {
                    D = ch[uu].x;
                    lm = ch[uu].y;
                  }
                  if (stash_r) stash_r[rk] = bf16_signed(a);
                }
                if (s != 0) {
                  D = s == -1 ? 1.f : 0.f;
                  const long long bi = bbase + ts;
                  if (bi < cx.n_beta) bs = fmaxf(cx.beta[bi], 0.f) * (float)s;
                  else atomicCAS(cx.status, 0, BCROWN_ERR_ARG);
                }
                const float L = valid ? fmaf(a, D, bs) : 0.f;
                acc = fmaf(L, bv[uu], fmaf(valid ? a : 0.f, lm, acc));
                o[u] = L;
              } else {   // EPI_FWD
                const float z = v[u] + bv[uu];
                float hv = code == CODE_ACTIVE ? z : 0.f;
                if (unst) {
                  if (st[uu] >= 0.f) {
                    hv = __saturatef(al[uu]) * z;
                    dalpha_r[rk] = st[uu] * z;
                  } else {
                    hv = fmaf(ch[uu].x, z, ch[uu].y);
                    dalpha_r[rk] = 0.f;
                  }
                }
                if (s != 0) {
                  const long long bi = bbase + ts;
                  if (bi < cx.n_beta) cx.dbeta[bi] = (float)s * z;
                  else atomicCAS(cx.status, 0, BCROWN_ERR_ARG);
                  hv = s == -1 ? z : 0.f;
                  // a split unstable neuron keeps its alpha slot, which the bound does not use
                  if (code == CODE_UNSTABLE) dalpha_r[rk] = 0.f;
                }
                o[u] = valid ? hv : 0.f;
              }
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) o2[u] = pack2(o[2 * u], o[2 * u + 1]);
        }
        if (ps.dst && nb + 8 <= lim) {
          // the chunk's elements are contiguous in the NHWC output
          *reinterpret_cast<uint4*>(ps.dst + (long long)rl * ps.dst_stride + nn0) =
              make_uint4(o2[0], o2[1], o2[2], o2[3]);
        }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
      if (MODE != EPI_FWD) {
        // partial sum of c for (row, this thread's positions and columns); a fixed slot each
        if (warp_sum_ok) {
          const float sw = lt_warp_sum(acc);
          if (lane == 0 && mv)
            cx.cpart[(size_t)rl * cx.S + ps.slot0 + ((size_t)nt * ps.Pm + pp) / 32] = sw;
        } else if (mv) {
          cx.cpart[(size_t)rl * cx.S + ps.slot0 + (size_t)nt * ps.Pm + pp] = acc;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == RL::MMA_W) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
  }
}

// Top of the recursion: A^(L-1) = Wbar_k, relaxed (layer L-1) into Lambda^(L-1) (NHWC BF16), its
// bias sum into slot 0 and A at the unstable neurons into the stash.  One warp per row.
__global__ void __launch_bounds__(256) k_lt_top(Ctx cx, int layer, long long hoff, int Co, int HWo, int Cpo,
                                                const float* __restrict__ Wbar, const float* __restrict__ bias,
                                                __nv_bfloat16* __restrict__ dst, long long dst_stride) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rl = blockIdx.x * 8 + w;
  if (rl >= cx.R) return;
  const int r = cx.r0 + rl;
  const int b = r / cx.K, k = r - b * cx.K;
  const int4 ri = cx.rowinfo[r];
  const long long abase = ((long long)(uint32_t)ri.y << 32) | (uint32_t)ri.x;
  const long long bbase = ri.z;
  const int prop = ri.w & 0x7FFFFFFF;
  const bool rv = ri.w < 0;
  const int* sl = cx.slayer + (size_t)b * (cx.L + 1) + layer;
  const int s0 = b * BCROWN_MAX_SPLITS + sl[0], s1 = b * BCROWN_MAX_SPLITS + sl[1];
  const int d = Co * HWo;
  float acc = 0.f;
  const size_t ng0 = (size_t)prop * cx.H + hoff;
  for (int q = lane; q < HWo * Cpo; q += 32) {
    // NHWC index q = p * Cpo + c
    const int p = q / Cpo, c = q - (q / Cpo) * Cpo;
    float L = 0.f;
    if (rv && c < Co) {
      const int jl = c * HWo + p;
      const float a = Wbar[(size_t)k * d + jl];
      int s = 0, ts = 0;
      for (int u = s0; u < s1; ++u) {
        const uint32_t e = cx.ssplit[u];
        if (sp_j(e) == jl) {
          s = sp_s(e);
          ts = sp_t(e);
        }
      }
      float D, lm = 0.f, bs = 0.f;
      const size_t ng = ng0 + jl;
      if (s != 0) {
        D = s == -1 ? 1.f : 0.f;
        const long long bi = bbase + ts;
        if (bi < cx.n_beta) bs = fmaxf(cx.beta[bi], 0.f) * (float)s;
        else atomicCAS(cx.status, 0, BCROWN_ERR_ARG);
      } else {
        const uint8_t code = cx.tb.code[ng];
        if (code == CODE_ACTIVE) D = 1.f;
        else if (code == CODE_INACTIVE) D = 0.f;
        else {
          const int rk = cx.tb.rank[ng];
          if (a >= 0.f) D = __saturatef(cx.alpha[abase + rk]);
          else {
            D = cx.tb.slope[ng];
            lm = cx.tb.icpt[ng];
          }
          if (cx.stash) cx.stash[abase + rk] = bf16_signed(a);
        }
      }
      L = fmaf(a, D, bs);
      acc = fmaf(L, bias[jl], fmaf(a, lm, acc));
    }
    dst[(size_t)rl * dst_stride + q] = __float2bfloat16_rn(L);
  }
  acc = lt_warp_sum(acc);
  if (lane == 0) cx.cpart[(size_t)rl * cx.S] = acc;
}

// Per row (once per call): where its alpha and beta start, its property, and whether its batch
// entries are consistent (otherwise the row is skipped and BCROWN_ERR_ARG recorded).
__global__ void __launch_bounds__(256) k_lt_rowinfo(int R, int K, int P, BatchView bt, const int32_t* __restrict__ U,
                                                    int64_t n_alpha, int4* __restrict__ rowinfo, int* status) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int b = r / K, k = r - b * K;
  int prop = bt.prop_of[b];
  bool v = prop >= 0 && prop < P;
  if (!v) prop = 0;
  const int cnt = bt.split_cnt[b], off = bt.split_off[b];
  const int Up = U[prop];
  const long long abase = bt.alpha_off[b] + (long long)k * Up;
  const long long bbase = (long long)off * K + (long long)k * cnt;
  v = v && cnt >= 0 && cnt <= BCROWN_MAX_SPLITS && off >= 0 && abase >= 0 && abase + Up <= n_alpha &&
      bbase <= 0x7FFFFFFFLL;
  if (!v) atomicCAS(status, 0, BCROWN_ERR_ARG);
  rowinfo[r] = make_int4((int)(uint32_t)(abase & 0xFFFFFFFFLL), (int)(abase >> 32), v ? (int)bbase : 0,
                         prop | (v ? (int)0x80000000 : 0));
}

// Per subdomain (once per call, one warp each): its splits sorted by hidden layer (list order
// within a layer) as packed entries, and where each layer's entries start.  Entries with a
// layer, index or sign out of range are dropped and BCROWN_ERR_ARG recorded.
__global__ void __launch_bounds__(256) k_lt_splits(int B, int L, const int* __restrict__ width, BatchView bt,
                                                   uint32_t* __restrict__ ssplit, int* __restrict__ slayer,
                                                   int* status) {
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (b >= B) return;
  int cnt = bt.split_cnt[b];
  const int off = bt.split_off[b];
  if (cnt < 0 || cnt > BCROWN_MAX_SPLITS || off < 0) cnt = 0;   // flagged by k_lt_rowinfo
  int ly[2], pk[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = lane + 32 * h;
    ly[h] = 0;
    pk[h] = 0;
    if (t < cnt) {
      const int l = bt.split_layer[off + t];
      const int j = (int)bt.split_idx[off + t];
      const int sg = bt.split_sign[off + t];
      if (l < 1 || l > L - 1 || j < 0 || j >= width[l] || j >= (1 << 20) || (sg != 1 && sg != -1)) {
        atomicCAS(status, 0, BCROWN_ERR_ARG);
      } else {
        ly[h] = l;
        pk[h] = (int)((uint32_t)j | ((uint32_t)t << 20) | ((sg == 1 ? 1u : 0u) << 26));
      }
    }
  }
  int start = 0;
  for (int l = 0; l <= L; ++l) {
    if (lane == 0) slayer[(size_t)b * (L + 1) + l] = start;
    if (l == 0 || l == L) continue;
    const unsigned m0 = __ballot_sync(0xffffffffu, ly[0] == l), m1 = __ballot_sync(0xffffffffu, ly[1] == l);
    const unsigned below = (1u << lane) - 1u;
    if (ly[0] == l) ssplit[(size_t)b * BCROWN_MAX_SPLITS + start + __popc(m0 & below)] = (uint32_t)pk[0];
    if (ly[1] == l) ssplit[(size_t)b * BCROWN_MAX_SPLITS + start + __popc(m0) + __popc(m1 & below)] = (uint32_t)pk[1];
    start += __popc(m0) + __popc(m1);
  }
}

// lb = bbar_k + the row's partial sums, added in slot order (one warp per row: lane-strided
// sums, then a fixed shuffle tree).
__global__ void __launch_bounds__(256) k_lt_lb(Ctx cx, const float* __restrict__ bbar, float* __restrict__ lb) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rl = blockIdx.x * 8 + w;
  if (rl >= cx.R) return;
  const int r = cx.r0 + rl;
  const int k = r % cx.K;
  float s = 0.f;
  for (int q = lane; q < cx.S; q += 32) s += cx.cpart[(size_t)rl * cx.S + q];
  s = lt_warp_sum(s);
  if (lane == 0) {
    float v = bbar[k] + s;
    if (!isfinite(v)) {
      atomicCAS(cx.status, 0, BCROWN_ERR_NONFINITE);
      v = -INFINITY;
    }
    lb[r] = v;
  }
}

// The neurons of one hidden layer in NHWC order per property, so that an epilogue reads 16
// channels' entries with four 16-byte loads: code (0 inactive, 1 active, 2 unstable) | rank << 2;
// and the upper chord of each unstable neuron by rank.
__global__ void k_lt_ntab(int P, long long H, long long hoff, int C, int HW, int Cp, long long NH, long long off,
                          Tables tb, uint32_t* __restrict__ ntab, float2* __restrict__ chord) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long d = (long long)C * HW;
  if (id >= (long long)P * d) return;
  const int p = (int)(id / d);
  const int j = (int)(id - (long long)p * d);
  const int c = j / HW, pos = j - c * HW;
  const size_t n = (size_t)p * H + hoff + j;
  const uint32_t code = tb.code[n];
  const int rk = tb.rank[n];
  ntab[(size_t)p * NH + off + (size_t)pos * Cp + c] = code | ((uint32_t)max(rk, 0) << 2);
  if (code == CODE_UNSTABLE && rk >= 0) chord[(size_t)p * H + rk] = make_float2(tb.slope[n], tb.icpt[n]);
}

inline int lt_smem(int Np) {
  return 1024 + NS * (16384 + Np * 128) + 256 + (MAX_KP / 8) * (int)sizeof(int2) + MAX_NP * (int)sizeof(float);
}

}  // namespace lt

using namespace lt;

namespace {

int pad_to(int x, int m) { return (x + m - 1) / m * m; }

// NHWC map of hidden layer l (0: the input): channels, height, width, padded channels.
struct MapDims {
  int C, H, W, Cp;
  int HW() const { return H * W; }
};

MapDims map_of(const bcrown_net* net, int l) {
  MapDims m;
  if (l == 0) {
    const LayerDev& f = net->ly[0];
    m = MapDims{f.in_c, f.in_h, f.in_w, 0};
    if (f.kind != BCROWN_LAYER_CONV) m = MapDims{f.d_in, 1, 1, 0};
  } else {
    const LayerDev& f = net->ly[l - 1];
    m = f.kind == BCROWN_LAYER_CONV ? MapDims{f.out_c, f.out_h, f.out_w, 0} : MapDims{f.d_out, 1, 1, 0};
  }
  m.Cp = pad_to(m.C, 8);
  return m;
}

// One prepared GEMM of a layer: B matrix rows [brow, brow + ntn * Np) of the layer's weight map,
// the gather table, and the pass geometry except the per-call pointers.
struct PassPrep {
  Pass p;
  int2* tab = nullptr;
};

struct LayerPrep {
  CUtensorMap mb, mf;                 // backward (phases stacked) and forward B matrices
  std::vector<PassPrep> bwd;          // one per stride phase (fc: one)
  PassPrep fwd;
};

struct LtNet {
  bool ready = false;
  std::vector<LayerPrep> ly;          // ly[i]: paper layer i (1..L-1)
  std::vector<void*> bufs;
  int S = 0;                          // partial-sum slots per row
  long long act_elems = 0;            // elements of one NHWC activation buffer per row
  int* width = nullptr;               // device [L]: d_0 .. d_{L-1}
  std::vector<float*> bnhwc;          // [l]: bias of hidden layer l in NHWC order (padded)
  std::vector<long long> nhwc_off;    // [l]: first code of hidden layer l in a property's NHWC codes
  long long NH = 0;                   // NHWC codes per property (all hidden layers, padded)
};

std::mutex g_lt_mu;
std::vector<std::pair<const bcrown_net*, LtNet*>> g_lt;

LtNet* lt_of(const bcrown_net* net) {
  std::lock_guard<std::mutex> g(g_lt_mu);
  for (auto& e : g_lt)
    if (e.first == net) return e.second;
  LtNet* t = new LtNet();
  g_lt.push_back({net, t});
  return t;
}

// Phase a of one spatial axis of a stride-s transposed convolution: taps k0 + s * d (d < nk)
// reach input rows a + s * i (i < n), whose source row is i + off - d.
struct Phase {
  int k0, nk, off, n;
};
Phase phase_of(int a, int k, int s, int pad, int in) {
  Phase c;
  c.k0 = (a + pad) % s;
  c.nk = c.k0 < k ? (k - c.k0 + s - 1) / s : 0;
  c.off = (a + pad - c.k0) / s;
  c.n = a < in ? (in - a + s - 1) / s : 0;
  return c;
}

int2 tap_entry(int elem_off, int dy, int dx) {
  return make_int2(elem_off, (int)(((uint32_t)dy & 0xffffu) | ((uint32_t)dx << 16)));
}
const int2 kNoChunk = make_int2(0, 0x8000);   // dy = -32768: no bounds test passes

int upload(LtNet* t, const void* host, size_t bytes, void** dev) {
  if (cudaMalloc(dev, bytes) != cudaSuccess) return fail(BCROWN_ERR_OOM, "layer path: device weights");
  t->bufs.push_back(*dev);
  if (cudaMemcpy(*dev, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(BCROWN_ERR_CUDA, "layer path: weight upload");
  return BCROWN_OK;
}

void n_tiles(int N, int* Np, int* ntn) {
  *Np = N <= MAX_NP ? pad_to(N, 16) : MAX_NP;
  *ntn = (N + *Np - 1) / *Np;
}

int prepare(bcrown_net* net, LtNet* t) {
  if (t->ready) return BCROWN_OK;
  const int L = net->L;
  t->ly.assign(L, LayerPrep());
  long long act = 0;
  for (int l = 0; l < L; ++l) {
    const MapDims m = map_of(net, l);
    act = std::max(act, (long long)m.HW() * m.Cp);
  }
  t->act_elems = pad_to((int)act, 64);
  // biases in NHWC order and the NHWC code table's layout, per hidden layer
  t->bnhwc.assign(L, nullptr);
  t->nhwc_off.assign(L, 0);
  long long nh = 0;
  for (int l = 1; l <= L - 1; ++l) {
    const MapDims m = map_of(net, l);
    const LayerDev& f = net->ly[l - 1];
    std::vector<float> bexp((size_t)f.d_out);
    if (cudaMemcpy(bexp.data(), f.b, bexp.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(BCROWN_ERR_CUDA, "layer path: copy of biases");
    std::vector<float> bn((size_t)m.HW() * m.Cp + 16, 0.f);
    for (int c = 0; c < m.C; ++c)
      for (int pos = 0; pos < m.HW(); ++pos) bn[(size_t)pos * m.Cp + c] = bexp[(size_t)c * m.HW() + pos];
    void* d = nullptr;
    BC_CHECK(upload(t, bn.data(), bn.size() * 4, &d));
    t->bnhwc[l] = reinterpret_cast<float*>(d);
    t->nhwc_off[l] = nh;
    nh += (long long)m.HW() * m.Cp;
  }
  t->NH = nh + 16;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  int slot = 1;   // slot 0: the top relaxation
  for (int i = L - 1; i >= 1; --i) {
    // backward slots are assigned top-down, in the order the passes run
    const LayerDev& l = net->ly[i - 1];
    const MapDims mi = map_of(net, i), mo = map_of(net, i - 1);   // GEMM source, output
    std::vector<float> w(l.kind == BCROWN_LAYER_CONV ? (size_t)l.out_c * l.in_c * l.k * l.k
                                                     : (size_t)l.d_out * l.d_in);
    if (cudaMemcpy(w.data(), l.W, w.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(BCROWN_ERR_CUDA, "layer path: copy of weights");
    LayerPrep& P = t->ly[i];
    auto finish_pass = [&](PassPrep& pp, std::vector<int2>& tab) -> int {
      void* d = nullptr;
      BC_CHECK(upload(t, tab.data(), tab.size() * sizeof(int2), &d));
      pp.tab = reinterpret_cast<int2*>(d);
      pp.p.tab = pp.tab;
      // The A operand by TMA where an M tile is one box of the NHWC source (whole rows of the
      // pass's position grid, or whole grids of consecutive subdomain rows) and each K block is
      // one tap's 64-channel block (source channels a multiple of 64).  A position step ms > 1
      // (a strided convolution's forward pass) is the box's traversal step in x and y: the box
      // spans ms times the positions it holds.
      Pass& q = pp.p;
      int bw = 0, bh = 0, br = 0;
      const bool narrow = q.Cps == 8 && q.nkb <= 16;   // 8 channels: one box per tap
      if (q.ms >= 1 && q.ms <= 8 && (q.Cps % 64 == 0 || narrow) && q.nJ > 0 && q.Pm > 0) {
        if (q.Pm % 128 == 0) {
          if (q.nJ <= 128 && 128 % q.nJ == 0) bw = q.nJ, bh = 128 / q.nJ, br = 1;
          else if (q.nJ % 128 == 0) bw = 128, bh = 1, br = 1;
        } else if (128 % q.Pm == 0 && q.Pm % q.nJ == 0) {
          bw = q.nJ, bh = q.Pm / q.nJ, br = 128 / q.Pm;
        }
      }
      if (bw > 0 && bw * bh * br == 128 && bw * q.ms <= 256 && bh * q.ms <= 256 && (size_t)q.nkb * 8 == tab.size() &&
          narrow) {
        std::vector<int4> kt(tab.size());
        for (size_t kc = 0; kc < tab.size(); ++kc) {
          const int dy = (int)(short)(tab[kc].y & 0xffff), dx = tab[kc].y >> 16;
          const bool used = dy != -32768;
          kt[kc] = make_int4(0, used ? dy : 0, used ? dx : 0, used ? 1 : 0);
        }
        void* dk = nullptr;
        BC_CHECK(upload(t, kt.data(), kt.size() * sizeof(int4), &dk));
        q.ktab = reinterpret_cast<const int4*>(dk);
        q.ta = 8, q.bw = bw, q.bh = bh, q.br = br;
      } else if (bw > 0 && bw * bh * br == 128 && bw * q.ms <= 256 && bh * q.ms <= 256 &&
                 (size_t)q.nkb * 8 == tab.size()) {
        const int cpb = q.Cps / 64;
        std::vector<int4> kt((size_t)q.nkb);
        for (int kb = 0; kb < q.nkb; ++kb) {
          const int2 e = tab[(size_t)kb * 8];
          const int dy = (int)(short)(e.y & 0xffff), dx = e.y >> 16;
          const bool used = dy != -32768;
          kt[kb] = make_int4((kb % cpb) * 64, used ? dy : 0, used ? dx : 0, used ? 1 : 0);
        }
        void* dk = nullptr;
        BC_CHECK(upload(t, kt.data(), kt.size() * sizeof(int4), &dk));
        q.ktab = reinterpret_cast<const int4*>(dk);
        q.ta = 4, q.bw = bw, q.bh = bh, q.br = br;
      }
      return BCROWN_OK;
    };
    if (l.kind == BCROWN_LAYER_CONV) {
      const int s = l.stride, k = l.k;
      const int T = (k + s - 1) / s;
      // backward: per phase (a, b), N = input channels, K = (dy, dx, output channel)
      int Np = 0, ntn = 0;
      n_tiles(mo.C, &Np, &ntn);
      const int kp = pad_to(T * T * mi.Cp, 64);
      std::vector<__nv_bfloat16> wb((size_t)s * s * Np * kp, zero);
      for (int a = 0; a < s; ++a)
        for (int bb = 0; bb < s; ++bb) {
          const Phase py = phase_of(a, k, s, l.pad, l.in_h), px = phase_of(bb, k, s, l.pad, l.in_w);
          const int ph = a * s + bb;
          PassPrep pp;
          Pass& q = pp.p;
          q.Pm = py.n * px.n;
          q.nJ = px.n;
          q.N = mo.C;
          q.Np = Np;
          q.ntn = ntn;
          q.nkb = kp / 64;
          q.brow = ph * Np;
          q.Hs = mi.H;
          q.Ws = mi.W;
          q.Cps = mi.Cp;
          q.ms = 1;
          q.cy = py.off;
          q.cx = px.off;
          q.kchunks = kp / 8;
          q.oa = a;
          q.ob = bb;
          q.os = s;
          q.Wo = mo.W;
          q.npos = 0;
          q.Co = mo.C;
          q.HWo = mo.HW();
          q.Cpo = mo.Cp;
          q.layer = i - 1;
          q.hoff = i >= 2 ? net->hoff[i - 2] : 0;
          q.bias = i >= 2 ? net->ly[i - 2].b : nullptr;
          q.bnhwc = i >= 2 ? t->bnhwc[i - 1] : nullptr;
          std::vector<int2> tab((size_t)kp / 8, kNoChunk);
          for (int dy = 0; dy < py.nk; ++dy)
            for (int dx = 0; dx < px.nk; ++dx) {
              const int tap = dy * px.nk + dx;
              for (int c8 = 0; c8 < mi.Cp / 8; ++c8)
                tab[(size_t)tap * (mi.Cp / 8) + c8] = tap_entry((-dy * mi.W - dx) * mi.Cp + 8 * c8, -dy, -dx);
              const int ky = py.k0 + s * dy, kx = px.k0 + s * dx;
              for (int co = 0; co < l.out_c; ++co)
                for (int ci = 0; ci < l.in_c; ++ci)
                  wb[((size_t)ph * Np + ci) * kp + (size_t)tap * mi.Cp + co] =
                      __float2bfloat16_rn(w[(((size_t)co * l.in_c + ci) * k + ky) * k + kx]);
            }
          if (q.Pm > 0) {
            BC_CHECK(finish_pass(pp, tab));
            q.slot0 = slot;
            slot += (q.Pm % 32 == 0) ? ntn * q.Pm / 32 : ntn * q.Pm;
            P.bwd.push_back(pp);
          }
        }
      void* db = nullptr;
      BC_CHECK(upload(t, wb.data(), wb.size() * 2, &db));
      BC_CHECK(encode_map(&P.mb, db, s * s * Np, kp, Np));
      // forward: N = output channels, K = (ky, kx, input channel)
      int Npf = 0, ntnf = 0;
      n_tiles(mi.C, &Npf, &ntnf);
      const int kpf = pad_to(k * k * mo.Cp, 64);
      std::vector<__nv_bfloat16> wf((size_t)ntnf * Npf * kpf, zero);
      std::vector<int2> tab((size_t)kpf / 8, kNoChunk);
      for (int ky = 0; ky < k; ++ky)
        for (int kx = 0; kx < k; ++kx) {
          const int tap = ky * k + kx;
          for (int c8 = 0; c8 < mo.Cp / 8; ++c8)
            tab[(size_t)tap * (mo.Cp / 8) + c8] = tap_entry((ky * mo.W + kx) * mo.Cp + 8 * c8, ky, kx);
          for (int co = 0; co < l.out_c; ++co)
            for (int ci = 0; ci < l.in_c; ++ci)
              wf[(size_t)co * kpf + (size_t)tap * mo.Cp + ci] =
                  __float2bfloat16_rn(w[(((size_t)co * l.in_c + ci) * k + ky) * k + kx]);
        }
      Pass& q = P.fwd.p;
      q.Pm = mi.HW();
      q.nJ = mi.W;
      q.N = mi.C;
      q.Np = Npf;
      q.ntn = ntnf;
      q.nkb = kpf / 64;
      q.brow = 0;
      q.Hs = mo.H;
      q.Ws = mo.W;
      q.Cps = mo.Cp;
      q.ms = s;
      q.cy = -l.pad;
      q.cx = -l.pad;
      q.kchunks = kpf / 8;
      q.oa = 0;
      q.ob = 0;
      q.os = 1;
      q.Wo = mi.W;
      q.npos = 0;
      q.Co = mi.C;
      q.HWo = mi.HW();
      q.Cpo = mi.Cp;
      q.layer = i;
      q.hoff = net->hoff[i - 1];
      q.bias = l.b;
      q.bnhwc = t->bnhwc[i];
      q.slot0 = 0;
      BC_CHECK(finish_pass(P.fwd, tab));
      void* df = nullptr;
      BC_CHECK(upload(t, wf.data(), wf.size() * 2, &df));
      BC_CHECK(encode_map(&P.mf, df, ntnf * Npf, kpf, Npf));
    } else {
      // fully connected: input = map mo (NHWC index p * Cp + c of neuron c * HW + p), output a vector
      const int din_n = mo.HW() * mo.Cp;   // NHWC-padded input length
      // backward: N = din_n (npos), K = output neurons (padded to 8, then 64)
      int Np = 0, ntn = 0;
      n_tiles(din_n, &Np, &ntn);
      const int kp = pad_to(mi.Cp, 64);
      std::vector<__nv_bfloat16> wb((size_t)ntn * Np * kp, zero);
      for (int o = 0; o < l.d_out; ++o)
        for (int c = 0; c < mo.C; ++c)
          for (int p = 0; p < mo.HW(); ++p)
            wb[((size_t)p * mo.Cp + c) * kp + o] = __float2bfloat16_rn(w[(size_t)o * l.d_in + (size_t)c * mo.HW() + p]);
      PassPrep pp;
      Pass& q = pp.p;
      q.Pm = 1;
      q.nJ = 1;
      q.N = din_n;
      q.Np = Np;
      q.ntn = ntn;
      q.nkb = kp / 64;
      q.brow = 0;
      q.Hs = 1;
      q.Ws = 1;
      q.Cps = mi.Cp;
      q.ms = 1;
      q.cy = 0;
      q.cx = 0;
      q.oa = 0;
      q.ob = 0;
      q.os = 1;
      q.Wo = 1;
      q.npos = 1;
      q.Co = mo.C;
      q.HWo = mo.HW();
      q.Cpo = mo.Cp;
      q.layer = i - 1;
      q.hoff = i >= 2 ? net->hoff[i - 2] : 0;
      q.bias = i >= 2 ? net->ly[i - 2].b : nullptr;
      q.bnhwc = i >= 2 ? t->bnhwc[i - 1] : nullptr;
      q.kchunks = mi.Cp / 8;   // K chunks past the layer's padded width read as zero
      q.tab = nullptr;
      q.ta = 2;   // the linear source: the A operand by TMA, 64 x 128-row boxes
      q.slot0 = slot;
      slot += ntn;
      P.bwd.push_back(pp);
      void* db = nullptr;
      BC_CHECK(upload(t, wb.data(), wb.size() * 2, &db));
      BC_CHECK(encode_map(&P.mb, db, ntn * Np, kp, Np));
      // forward: N = output neurons, K = din_n (padded to 64)
      int Npf = 0, ntnf = 0;
      n_tiles(mi.C, &Npf, &ntnf);
      const int kpf = pad_to(din_n, 64);
      std::vector<__nv_bfloat16> wf((size_t)ntnf * Npf * kpf, zero);
      for (int o = 0; o < l.d_out; ++o)
        for (int c = 0; c < mo.C; ++c)
          for (int p = 0; p < mo.HW(); ++p)
            wf[(size_t)o * kpf + (size_t)p * mo.Cp + c] = __float2bfloat16_rn(w[(size_t)o * l.d_in + (size_t)c * mo.HW() + p]);
      Pass& f = P.fwd.p;
      f = q;
      f.N = mi.C;
      f.Np = Npf;
      f.ntn = ntnf;
      f.nkb = kpf / 64;
      f.Cps = mo.Cp;
      f.kchunks = din_n / 8;
      f.tab = nullptr;
      f.ta = 2;
      f.npos = 0;
      f.Co = mi.C;
      f.HWo = 1;
      f.Cpo = mi.Cp;
      f.Wo = 1;
      f.layer = i;
      f.hoff = net->hoff[i - 1];
      f.bias = l.b;
      f.bnhwc = t->bnhwc[i];
      f.slot0 = 0;
      void* df = nullptr;
      BC_CHECK(upload(t, wf.data(), wf.size() * 2, &df));
      BC_CHECK(encode_map(&P.mf, df, ntnf * Npf, kpf, Npf));
    }
  }
  t->S = slot;
  {
    std::vector<int> wd(net->d.begin(), net->d.begin() + L);
    void* d = nullptr;
    BC_CHECK(upload(t, wd.data(), wd.size() * sizeof(int), &d));
    t->width = reinterpret_cast<int*>(d);
  }
  BC_CUDA(cudaFuncSetAttribute(k_lt<EPI_RELAX, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lt_smem(MAX_NP)));
  BC_CUDA(cudaFuncSetAttribute(k_lt<EPI_CONCRETIZE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               lt_smem(MAX_NP)));
  BC_CUDA(cudaFuncSetAttribute(k_lt<EPI_FWD, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lt_smem(MAX_NP)));
  BC_CUDA(cudaFuncSetAttribute(k_lt<EPI_RELAX, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lt_smem(MAX_NP)));
  BC_CUDA(cudaFuncSetAttribute(k_lt<EPI_CONCRETIZE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               lt_smem(MAX_NP)));
  BC_CUDA(cudaFuncSetAttribute(k_lt<EPI_FWD, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lt_smem(MAX_NP)));
  t->ready = true;
  return BCROWN_OK;
}

int launch_pass(bcrown_net* net, const CUtensorMap& mB, Pass q, int mode, const Ctx& cx, cudaStream_t s) {
  q.M = (long long)cx.R * q.Pm;
  if (q.M <= 0) return BCROWN_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (q.M + 127) / 128 * q.ntn;
  const int grid = (int)std::min<long long>(ntiles, sms);
  const int smem = lt_smem(q.Np);
  ProfScope pr(net, BCROWN_PROF_LAYER_GEMM, s);
  // the A operand's map for this launch (the source buffer and the rows of this chunk)
  CUtensorMap mA = mB;   // unused by the gathering kernel
  if (q.ta == 4 || q.ta == 8) {
    const cuuint64_t dims[4] = {(cuuint64_t)q.Cps, (cuuint64_t)q.Ws, (cuuint64_t)q.Hs, (cuuint64_t)cx.R};
    const cuuint64_t strides[3] = {(cuuint64_t)q.Cps * 2, (cuuint64_t)q.Ws * q.Cps * 2, (cuuint64_t)q.src_stride * 2};
    // a strided pass: boxes of ms bw x ms bh source positions, every ms-th one loaded (bw x bh)
    const cuuint32_t box[4] = {q.ta == 8 ? 8u : 64u, (cuuint32_t)(q.bw * q.ms), (cuuint32_t)(q.bh * q.ms),
                               (cuuint32_t)q.br};
    const cuuint32_t es[4] = {1, (cuuint32_t)q.ms, (cuuint32_t)q.ms, 1};
    BC_CHECK(encode_map_nd(&mA, const_cast<__nv_bfloat16*>(q.src), 4, dims, strides, box, es, q.ta == 4));
  } else if (q.ta == 2) {
    const cuuint64_t dims[2] = {(cuuint64_t)q.kchunks * 8, (cuuint64_t)cx.R};
    const cuuint64_t strides[1] = {(cuuint64_t)q.src_stride * 2};
    const cuuint32_t box[2] = {64, 128};
    BC_CHECK(encode_map_nd(&mA, const_cast<__nv_bfloat16*>(q.src), 2, dims, strides, box));
  }
  if (q.ta) {
    if (mode == EPI_RELAX) k_lt<EPI_RELAX, true><<<grid, LtRoles<true>::THREADS, smem, s>>>(mB, mA, q, cx);
    else if (mode == EPI_CONCRETIZE) k_lt<EPI_CONCRETIZE, true><<<grid, LtRoles<true>::THREADS, smem, s>>>(mB, mA, q, cx);
    else k_lt<EPI_FWD, true><<<grid, LtRoles<true>::THREADS, smem, s>>>(mB, mA, q, cx);
  } else {
    if (mode == EPI_RELAX) k_lt<EPI_RELAX, false><<<grid, LtRoles<false>::THREADS, smem, s>>>(mB, mA, q, cx);
    else if (mode == EPI_CONCRETIZE) k_lt<EPI_CONCRETIZE, false><<<grid, LtRoles<false>::THREADS, smem, s>>>(mB, mA, q, cx);
    else k_lt<EPI_FWD, false><<<grid, LtRoles<false>::THREADS, smem, s>>>(mB, mA, q, cx);
  }
  ++g_launches;
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

}  // namespace

// Per-row sizes of the workspace: the NHWC activation buffer (elements) and an upper bound of the
// partial-sum slots (one per position block and column group of every backward pass), and the
// rows per chunk for a 16 GB target.
static void plan_sizes(const bcrown_net* net, int R, long long* act, long long* S, long long* Rc) {
  long long a = 0, sl = 1;
  for (int l = 0; l < net->L; ++l) {
    const MapDims m = map_of(net, l);
    a = std::max(a, (long long)m.HW() * m.Cp);
  }
  for (int i = 1; i <= net->L - 1; ++i) {
    const MapDims mo = map_of(net, i - 1);
    sl += 2LL * mo.HW() * std::max(1, (mo.Cp + MAX_NP - 1) / MAX_NP) + 2LL * (((long long)mo.HW() * mo.Cp + MAX_NP - 1) / MAX_NP);
  }
  *act = (a + 63) / 64 * 64;
  *S = sl;
  const size_t per_row = (size_t)2 * *act * 2 + (size_t)sl * 4;
  const size_t target = size_t(16) << 30;
  *Rc = std::max<long long>(1, std::min<long long>(std::max(R, 1), (long long)(target / per_row)));
}

bool lt_supported(const bcrown_net* net) {
  if (net->L < 2) return false;
  for (int i = 1; i <= net->L - 1; ++i) {
    const LayerDev& l = net->ly[i - 1];
    const MapDims mi = map_of(net, i), mo = map_of(net, i - 1);
    if (l.kind == BCROWN_LAYER_CONV) {
      if (l.in_c > MAX_NP || l.out_c > MAX_NP) return false;
      const int T = (l.k + l.stride - 1) / l.stride;
      if (pad_to(T * T * mi.Cp, 64) > MAX_KP || pad_to(l.k * l.k * mo.Cp, 64) > MAX_KP) return false;
    } else {
      if (pad_to(mi.Cp, 64) > MAX_KP) return false;   // backward K
      if ((long long)mo.HW() * mo.Cp > 65536 || l.d_out > 65536) return false;
    }
    if ((long long)mi.HW() * mi.Cp > (1LL << 24)) return false;
  }
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaGetLastError();
  return major == 10 && minor == 3;
}

size_t lt_workspace_bytes(const bcrown_net* net, int R, int P, int64_t n_alpha, bool grad) {
  long long act, S, Rc;
  plan_sizes(net, R, &act, &S, &Rc);
  long long nh = 16;
  for (int l = 1; l <= net->L - 1; ++l) {
    const MapDims m = map_of(net, l);
    nh += (long long)m.HW() * m.Cp;
  }
  const size_t B = (size_t)R / std::max(net->K, 1);
  size_t bytes = align_up((size_t)Rc * act * 2) * 2 + align_up((size_t)Rc * S * 4);
  bytes += align_up((size_t)R * 16) + align_up(B * BCROWN_MAX_SPLITS * 4) + align_up(B * (net->L + 1) * 4);
  bytes += align_up((size_t)std::max(P, 1) * nh * 4) + align_up((size_t)std::max(P, 1) * std::max(net->H, 1) * 8);
  if (grad) bytes += align_up((size_t)std::max<int64_t>(n_alpha, 1) * 2);
  return bytes;
}

int lt_bound(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* bt, const Tables& tb, char* ws,
             size_t ws_bytes, bool grad, const float* alpha, const float* beta, float* lb, float* dalpha,
             float* dbeta, cudaStream_t s) {
  LtNet* t = lt_of(net);
  BC_CHECK(prepare(net, t));
  const int K = net->K, L = net->L;
  const int R = bt->B * K;
  if (R == 0) return BCROWN_OK;
  if (ws_bytes < lt_workspace_bytes(net, R, dom->n_props, bt->n_alpha, grad))
    return fail(BCROWN_ERR_OOM, "layer path: workspace");
  long long act_b, S_b, Rc;
  plan_sizes(net, R, &act_b, &S_b, &Rc);
  if (act_b != t->act_elems || S_b < t->S) return fail(BCROWN_ERR_ARG, "layer path: inconsistent plan");
  Arena ar{ws};
  __nv_bfloat16* act[2];
  act[0] = ar.take<__nv_bfloat16>((size_t)Rc * t->act_elems);
  act[1] = ar.take<__nv_bfloat16>((size_t)Rc * t->act_elems);
  float* cpart = ar.take<float>((size_t)Rc * S_b);
  int4* rowinfo = ar.take<int4>((size_t)R);
  uint32_t* ssplit = ar.take<uint32_t>((size_t)bt->B * BCROWN_MAX_SPLITS);
  int* slayer = ar.take<int>((size_t)bt->B * (L + 1));
  uint32_t* ntab = ar.take<uint32_t>((size_t)dom->n_props * t->NH);
  float2* chord = ar.take<float2>((size_t)dom->n_props * std::max(net->H, 1));
  __nv_bfloat16* stash = grad ? ar.take<__nv_bfloat16>((size_t)std::max<int64_t>(bt->n_alpha, 1)) : nullptr;
  if (ar.off > ws_bytes) return fail(BCROWN_ERR_OOM, "layer path: workspace plan");
  Ctx cx;
  cx.K = K;
  cx.P = dom->n_props;
  cx.H = net->H;
  cx.d0 = net->d[0];
  cx.S = t->S;
  cx.bt = BatchView{bt->B, bt->prop_of, bt->split_off, bt->split_cnt, bt->split_layer, bt->split_idx, bt->split_sign,
                    bt->alpha_off};
  cx.tb = tb;
  cx.x_lo = dom->x_lo;
  cx.x_hi = dom->x_hi;
  cx.alpha = alpha;
  cx.beta = beta;
  cx.n_alpha = bt->n_alpha;
  cx.n_beta = bt->n_beta;
  cx.dalpha = dalpha;
  cx.dbeta = dbeta;
  cx.stash = stash;
  cx.cpart = cpart;
  cx.status = net->status;
  cx.rowinfo = rowinfo;
  cx.ssplit = ssplit;
  cx.slayer = slayer;
  cx.L = L;
  cx.NH = t->NH;
  cx.chord = chord;
  // the properties' neurons in NHWC order and their chords by rank, once per call
  BC_CUDA(cudaMemsetAsync(ntab, 0, (size_t)dom->n_props * t->NH * 4, s));
  for (int l = 1; l <= L - 1; ++l) {
    const MapDims m = map_of(net, l);
    const long long n = (long long)dom->n_props * m.C * m.HW();
    k_lt_ntab<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dom->n_props, net->H, net->hoff[l - 1], m.C, m.HW(), m.Cp,
                                                         t->NH, t->nhwc_off[l], tb, ntab, chord);
    ++g_launches;
  }
  // the rows' alpha / beta offsets and the subdomains' splits sorted by layer, once per call
  k_lt_rowinfo<<<(R + 255) / 256, 256, 0, s>>>(R, K, dom->n_props, cx.bt, tb.U, bt->n_alpha, rowinfo, net->status);
  k_lt_splits<<<(bt->B * 32 + 255) / 256, 256, 0, s>>>(bt->B, L, t->width, cx.bt, ssplit, slayer, net->status);
  g_launches += 2;
  const long long stride = t->act_elems;
  for (long long r0 = 0; r0 < R; r0 += Rc) {
    cx.r0 = (int)r0;
    cx.R = (int)std::min<long long>(Rc, R - r0);
    // top: Lambda^(L-1) into act[0]
    {
      ProfScope pr(net, BCROWN_PROF_RELAX, s);
      const MapDims mt = map_of(net, L - 1);
      k_lt_top<<<(cx.R + 7) / 8, 256, 0, s>>>(cx, L - 1, net->hoff[L - 2], mt.C, mt.HW(), mt.Cp, net->Wbar,
                                              net->ly[L - 2].b, act[0], stride);
      ++g_launches;
    }
    int cur = 0;
    for (int i = L - 1; i >= 1; --i) {
      const LayerPrep& P = t->ly[i];
      for (const PassPrep& pp : P.bwd) {
        Pass q = pp.p;
        q.ntab = i >= 2 ? ntab + t->nhwc_off[i - 1] : nullptr;
        q.src = act[cur];
        q.src_stride = stride;
        q.dst = act[cur ^ 1];
        q.dst_stride = stride;
        BC_CHECK(launch_pass(net, P.mb, q, i == 1 ? EPI_CONCRETIZE : EPI_RELAX, cx, s));
      }
      cur ^= 1;
    }
    {
      ProfScope pr(net, BCROWN_PROF_CONCRETIZE, s);
      k_lt_lb<<<(cx.R + 7) / 8, 256, 0, s>>>(cx, net->bbar, lb);
      ++g_launches;
    }
    if (!grad) continue;
    // adjoint: x* is in act[cur]
    for (int i = 1; i <= L - 1; ++i) {
      const LayerPrep& P = t->ly[i];
      Pass q = P.fwd.p;
      q.ntab = ntab + t->nhwc_off[i];
      q.src = act[cur];
      q.src_stride = stride;
      q.dst = i < L - 1 ? act[cur ^ 1] : nullptr;
      q.dst_stride = stride;
      BC_CHECK(launch_pass(net, P.mf, q, EPI_FWD, cx, s));
      cur ^= 1;
    }
  }
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

void lt_release(const bcrown_net* net) {
  std::lock_guard<std::mutex> g(g_lt_mu);
  for (size_t i = 0; i < g_lt.size(); ++i)
    if (g_lt[i].first == net) {
      for (void* b : g_lt[i].second->bufs) cudaFree(b);
      delete g_lt[i].second;
      g_lt.erase(g_lt.begin() + i);
      return;
    }
}

}  // namespace bcrown
