// Fused tensor-core bound pass for fully connected ReLU networks (sm_103a: tcgen05 + TMA).
//
// One persistent CTA per SM walks tiles of TR = 64 rows (row = subdomain x spec).  For a
// tile, the whole backward recursion of Theorem 3.1 (Eq. definition_A) runs on chip:
//
//   A^(i-1)^T = W^(i)^T Lambda^(i)^T      (tcgen05.mma, M = 128 output neurons, N = TR rows,
//                                          K = 16; BF16 operands, FP32 accumulator in TMEM)
//
// The weight tile is the MMA's A operand (loaded by TMA, 128B swizzle, K-major) and the
// activations Lambda^T are its B operand (written to shared memory by the epilogue in the
// same swizzled layout).  Putting neurons on TMEM lanes makes every epilogue access to
// alpha, the per-neuron tables, the gradients and the stash coalesced across a warp.
//
// The epilogue (16 warps) reads the accumulator with tcgen05.ld, applies the relaxation of
// Lemma 2.1 / Eq. definition_D (split overriding stability), the beta shift and the bias
// sums (Lambda = A D + beta S; c += Lambda b + A lambda), and writes Lambda^(i-1) in BF16
// as the next contraction's operand.  The last contraction is concretised over the box
// (Eq. beta_crown_lp).  With a gradient requested the adjoint pass follows in the same
// launch: zhat^(i) = W^(i) h^(i-1) + b^(i) along h^(0) = x*, dalpha = A zhat, dbeta = S zhat,
// h = D zhat + lambda.  The kernel writes the gradients only: the projected Adam step
// (Appendix C.1) and the per-row best tracking run afterwards in a separate element-wise
// kernel over alpha and beta.
//
// Roles: warps 0-15 epilogue, warp 16 TMA producer, warp 17 MMA issuer (one lane each).
// Every mbarrier wait is bounded; on expiry the kernel records BCROWN_ERR_TIMEOUT, stops
// issuing work, waits (bounded) for its copies in flight, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstring>

#include "fused_tc.cuh"
#include "tc_ptx.cuh"

namespace bcrown {

extern std::atomic<long long> g_launches;

namespace tc {

constexpr int TR = 64;            // rows per tile = MMA N
constexpr int MCH = 128;          // neurons per M chunk = MMA M
constexpr int NSLOT = 8;          // activation (B operand) ring
constexpr int NSTAGE = 4;         // weight (A operand) ring
constexpr int NACC = 4;           // accumulator ring (TR columns each)
constexpr int SLOT_BYTES = TR * 128;     // 8 KB
constexpr int STAGE_BYTES = MCH * 128;   // 16 KB
constexpr int NEPI = 16;                 // epilogue warps
constexpr int TMA_WARP = 16, MMA_WARP = 17;
constexpr int NTHREADS = 18 * 32;
constexpr int MAXL = 9;
constexpr int MAX_D0 = 1024;
constexpr int SIGN_WORDS = MAX_D0 / 32;
constexpr int MAX_MASK_WORDS = 48;       // sum over hidden layers of ceil(d_i/32)
static_assert(MAX_MASK_WORDS % 8 == 0, "set-up step 3 splits the mask words over 8 threads per row");
constexpr int MAX_H = MAX_MASK_WORDS * 32;  // hidden neurons whose tables a tile stages
constexpr int MAX_HIDDEN = 256;

struct Smem {
  uint8_t act[NSLOT][SLOT_BYTES];        // 64 KB, 1024-aligned slots
  uint8_t w[NSTAGE][STAGE_BYTES];        // 64 KB
  uint32_t sign[TR][SIGN_WORDS];         // 8 KB: A^(0) >= 0 per (row, input)
  uint32_t smask[MAX_MASK_WORDS][TR];    // split present, [word][row]: a warp reads its 16 rows at once
  uint32_t sneg[MAX_MASK_WORDS][TR];     // split sign +1 (z < 0)
  unsigned long long wrows[MAX_MASK_WORDS];  // rows with any split in mask word w
  float part[4][TR];                     // lb partial sums per lane quadrant
  long long abase[TR];                   // first alpha of the row
  long long bbase[TR];                   // first beta of the row
  int rowid[TR];                         // global row of each tile slot (-1: empty)
  int spec[TR];
  int valid[TR];
  int scnt[TR];                          // the row's split count and first split entry
  int soff[TR];
  uint8_t sorig[TR][BCROWN_MAX_SPLITS];  // the row's splits in (mask word, bit) order: list position
  float sbeta[TR][BCROWN_MAX_SPLITS];    //   and beta (clamped at 0)
  uint8_t wfirst[MAX_MASK_WORDS][TR];    // splits of the row in mask words before w
  uint32_t tcode[MAX_H];                 // the tile's property: code << 16 | unstable rank, per hidden neuron
  float tslope[MAX_H];                   //   upper chord slope
  float ticpt[MAX_H];                    //   upper chord intercept
  float sxlo[MAX_D0];                    //   input box
  float sxhi[MAX_D0];
  float sbias[MAX_H];                    // hidden-layer biases, by global hidden index
  unsigned long long vrows;              // tile slots holding a valid row
  uint64_t act_full[NSLOT], act_empty[NSLOT];
  uint64_t w_full[NSTAGE], w_empty[NSTAGE];
  uint64_t acc_full[NACC], acc_empty[NACC];
  uint64_t epi;   // epilogue-wide barrier (NEPI warp arrivals per phase)
  uint64_t done;
  uint32_t tmem_base;
  int abort_flag;
};

static_assert(sizeof(Smem) + 1024 <= 232448, "shared memory plan exceeds 227 KB per CTA");

struct Args {
  int L, K, P, H, R;
  const int* n_tiles;                 // tiles to process (written by the row planner)
  const int* tile_prop;               // [tile] property of every row of the tile
  const int* rowmap;                  // [tile][TR] global row of each slot, -1 when empty
  int d[MAXL + 1];
  long long hoff[MAXL + 1];           // first global hidden index of layer i (1-based)
  int woff[MAXL + 1];                 // first mask word of layer i
  int mask_words;
  const float* bias[MAXL + 1];
  const float* Wbar;
  const float* bbar;
  BatchView bt;
  Tables tb;
  const float* x_lo;
  const float* x_hi;
  const float* alpha;
  const float* beta;
  int64_t n_alpha, n_beta;
  float* lb;
  float* dalpha;
  __nv_bfloat16* dalpha16;            // MODE 2: dlb/dalpha rounded to BF16 (optimiser input)
  float* dbeta;
  __nv_bfloat16* stash;               // [tile][H][TR]: A^(i) of the backward pass, per neuron
  int* status;
  int box_bwd[MAXL + 1];
  int box_fwd[MAXL + 1];
};

struct Maps {
  CUtensorMap bwd[MAXL + 1];   // Wt^(i): [d_{i-1}][Kp(d_i)] bf16, rows = output neurons of the backward
  CUtensorMap fwd[MAXL + 1];   // W^(i):  [d_i][Kp(d_{i-1})] bf16, rows = output neurons of the forward
};

// ------------------------------------------------------------------------------------------
// PTX helpers
// ------------------------------------------------------------------------------------------

// Bounded wait (about 2 s of SM clock); on expiry records a timeout and raises the abort flag.
// Inlined: as a called function it cost the single-thread MMA and TMA loops ~0.2 us per wait.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, Smem* sm, int* status) {
  if (mbar_try(b, parity)) return true;
  long long t0 = clock64();
  while (true) {
    if (mbar_try_sleep(b, parity, 20000u)) return true;
    if (*(volatile int*)&sm->abort_flag) return false;
    if (clock64() - t0 > 4000000000LL) {
      atomicCAS(status, 0, BCROWN_ERR_TIMEOUT);
      *(volatile int*)&sm->abort_flag = 1;
      return false;
    }
  }
}
// Wait by a whole warp: one lane polls the barrier (512 polling threads would flood the
// shared-memory pipe every other warp needs), then the warp reconverges.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* b, uint32_t parity, Smem* sm, int* status) {
  __syncwarp();
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(b, parity, sm, status) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}
__device__ __forceinline__ bool epi_sync(Smem* sm, uint32_t& seq, int* status) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(&sm->epi);
  const bool ok = mbar_wait_warp(&sm->epi, seq & 1, sm, status);
  ++seq;
  return ok;
}
// Barrier among the 16 epilogue warps built on an mbarrier, so that a warp that gives up
// after a timeout cannot leave the others blocked: every wait here is bounded.
__device__ __forceinline__ bool epi_sync(Smem* sm, uint32_t& seq, int* status);




// Loads issued where they are written (volatile asm keeps them ahead of the barrier waits that
// follow, instead of letting the compiler sink them to their first use); 0 when pred is false.
__device__ __forceinline__ float ldg_f32(const float* p, bool pred) {
  float v;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.f32 %0, 0f00000000;\n\t@q ld.global.f32 %0, [%1];\n\t}"
               : "=f"(v)
               : "l"(p), "r"((uint32_t)pred)
               : "memory");
  return v;
}
__device__ __forceinline__ float ldg_bf16(const __nv_bfloat16* p, bool pred) {
  uint16_t v;
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.u16 %0, 0;\n\t@q ld.global.u16 %0, [%1];\n\t}"
               : "=h"(v)
               : "l"(p), "r"((uint32_t)pred)
               : "memory");
  return __uint_as_float(((uint32_t)v) << 16);
}

// Sum of v[r] over the 32 lanes of a warp, for r = 0..15, scattered so that lanes 2r and 2r+1
// both hold the sum for r (16 shuffles instead of 80).
__device__ __forceinline__ float reduce16(float (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool hi = lane & 16;
    const float send = hi ? v[i] : v[i + 8];
    const float keep = hi ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool hi = lane & 8;
    const float send = hi ? v[i] : v[i + 4];
    const float keep = hi ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = lane & 4;
    const float send = hi ? v[i] : v[i + 2];
    const float keep = hi ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool hi = lane & 2;
    const float send = hi ? v[0] : v[1];
    const float keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Sum of v[r] over the 32 lanes, r = 0..7, scattered: lanes 4r..4r+3 hold the sum for r.
__device__ __forceinline__ float reduce8(float (&v)[8]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool hi = lane & 16;
    const float send = hi ? v[i] : v[i + 4];
    const float keep = hi ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = lane & 8;
    const float send = hi ? v[i] : v[i + 2];
    const float keep = hi ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const bool hi = lane & 4;
    const float send = hi ? v[0] : v[1];
    const float keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  float r = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 2);
  return r + __shfl_xor_sync(0xffffffffu, r, 1);
}

// 16-byte global load (zero when !pred) and store.
__device__ __forceinline__ uint4 ldg_v4(const void* p, bool pred) {
  uint4 v;
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\tmov.b32 %0, 0;\n\tmov.b32 %1, 0;\n\tmov.b32 %2, 0;\n\t"
      "mov.b32 %3, 0;\n\t@q ld.global.v4.b32 {%0, %1, %2, %3}, [%4];\n\t}"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "r"((uint32_t)pred)
      : "memory");
  return v;
}
__device__ __forceinline__ void stg_v4(void* p, uint4 v) {
  asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

// L2 prefetch of [p, p + bytes): only the 16-byte aligned interior, so it stays in bounds.
__device__ __forceinline__ void prefetch_l2(const void* p, long long bytes) {
  uintptr_t lo = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  uintptr_t hi = ((uintptr_t)p + (uintptr_t)bytes) & ~(uintptr_t)15;
  while (lo < hi) {
    uint32_t n = (uint32_t)min((uintptr_t)(1u << 20), hi - lo);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"(n) : "memory");
    lo += n;
  }
}

// Byte offset of element (row, k) inside one activation slot (TR rows x 64 bf16, 128B swizzle).
__device__ __forceinline__ uint32_t act_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ row) & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ int nkb_of(int K) { return (K + KBLK - 1) / KBLK; }
__device__ __forceinline__ int nmc_of(int N) { return (N + MCH - 1) / MCH; }

// Contraction ci of a tile: backward layers L-1..1, then (gradient modes) forward layers 1..L-1.
__device__ __forceinline__ void contraction(const Args& a, int ci, int& layer, int& N, int& K, bool& fwd) {
  int nb = a.L - 1;
  if (ci < nb) {
    layer = a.L - 1 - ci;
    N = a.d[layer - 1];
    K = a.d[layer];
    fwd = false;
  } else {
    layer = ci - nb + 1;
    N = a.d[layer];
    K = a.d[layer - 1];
    fwd = true;
  }
}

// Index into beta of split (layer i, neuron j) of a tile row, or -1 (scans the row's split list).
// Slot of the split at (mask word w, bit) of a tile row, in the row's sorted split order:
// the splits in earlier words plus those below `bit` in word w (O(1), no search).
__device__ __forceinline__ int split_slot(const Smem* sm, int row, int w, int bit) {
  return (int)sm->wfirst[w][row] + __popc(sm->smask[w][row] & ((1u << bit) - 1u));
}

// ------------------------------------------------------------------------------------------
// The kernel
// ------------------------------------------------------------------------------------------
// MODE 0: bound only; MODE 1: bound and gradient (adjoint pass); MODE 2: as MODE 1 with dlb/dalpha
// stored in BF16 (the optimiser's own gradient buffer).
template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 1) k_fused(const __grid_constant__ Maps maps, const Args a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // pointer arithmetic on the shared array (not through an integer) keeps the shared address
  // space visible to the compiler, so accesses through `sm` are shared loads/stores
  const uint32_t pad = (1024u - (su32(smem_raw) & 1023u)) & 1023u;
  Smem* sm = reinterpret_cast<Smem*>(smem_raw + pad);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_contr = (a.L - 1) * (MODE >= 1 ? 2 : 1);
  const int n_tiles = *a.n_tiles;

  if (threadIdx.x == 0) {
    for (int i = 0; i < NSLOT; ++i) {
      mbar_init(&sm->act_full[i], NEPI / 2);   // the 8 warps that write a K block
      mbar_init(&sm->act_empty[i], 1);
    }
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(&sm->w_full[i], 1);
      mbar_init(&sm->w_empty[i], 1);
    }
    for (int i = 0; i < NACC; ++i) {
      mbar_init(&sm->acc_full[i], 1);
      mbar_init(&sm->acc_empty[i], NEPI);
    }
    mbar_init(&sm->epi, NEPI);
    mbar_init(&sm->done, 1);
    sm->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sm->tmem_base)),
                 "r"(NACC * TR)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm->tmem_base;

  if (warp == TMA_WARP) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      uint32_t wseq = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x)
        for (int ci = 0; ci < n_contr && ok; ++ci) {
          int layer, N, K;
          bool fwd;
          contraction(a, ci, layer, N, K, fwd);
          const CUtensorMap* map = fwd ? &maps.fwd[layer] : &maps.bwd[layer];
          const uint32_t bytes = (uint32_t)(fwd ? a.box_fwd[layer] : a.box_bwd[layer]) * 128u;
          const int nmc = nmc_of(N), nkb = nkb_of(K);
          const bool stream = nkb > NSLOT / 2;   // same order as the MMA issuer
          const int n_outer = stream ? nkb : nmc, n_inner = stream ? nmc : nkb;
          for (int o = 0; o < n_outer && ok; ++o)
            for (int in = 0; in < n_inner && ok; ++in) {
              const int mc = stream ? in : o, kb = stream ? o : in;
              int st = wseq % NSTAGE;
              if (!mbar_wait(&sm->w_empty[st], ((wseq / NSTAGE) & 1) ^ 1, sm, a.status)) {
                ok = false;
                break;
              }
              mbar_expect_tx(&sm->w_full[st], bytes);
              tma_load_2d(sm->w[st], map, kb * KBLK, mc * MCH, &sm->w_full[st]);
              ++wseq;
            }
        }
      if (!ok) {
        // wait (bounded) for the copies still in flight before the CTA may exit
        for (uint32_t s = (wseq > NSTAGE ? wseq - NSTAGE : 0); s < wseq; ++s) {
          long long t0 = clock64();
          while (!mbar_try(&sm->w_full[s % NSTAGE], (s / NSTAGE) & 1) && clock64() - t0 < 200000000LL) {
          }
        }
      }
    }
  } else if (warp == MMA_WARP) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t wseq = 0, accseq = 0, aseq = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x)
        for (int ci = 0; ci < n_contr && ok; ++ci) {
          int layer, N, K;
          bool fwd;
          contraction(a, ci, layer, N, K, fwd);
          const int nmc = nmc_of(N), nkb = nkb_of(K);
          const uint32_t idesc = idesc_bf16(TR);
          if (nkb > NSLOT / 2) {
            // Streamed operand (more K blocks than stay resident): K blocks outer, all M
            // chunks accumulate at once (nmc <= NACC), each K block released after use.
            for (int mc = 0; mc < nmc && ok; ++mc) {
              const uint32_t sq = accseq + mc;
              if (!mbar_wait(&sm->acc_empty[sq % NACC], ((sq / NACC) & 1) ^ 1, sm, a.status)) ok = false;
            }
            tc_fence_after();
            for (int kb = 0; kb < nkb && ok; ++kb) {
              const uint32_t as = aseq + kb;
              const int slot = as % NSLOT;
              if (!mbar_wait(&sm->act_full[slot], (as / NSLOT) & 1, sm, a.status)) {
                ok = false;
                break;
              }
              for (int mc = 0; mc < nmc; ++mc) {
                const int st = wseq % NSTAGE;
                if (!mbar_wait(&sm->w_full[st], (wseq / NSTAGE) & 1, sm, a.status)) {
                  ok = false;
                  break;
                }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(((accseq + mc) % NACC) * TR);
                const uint32_t wa = su32(sm->w[st]);
                const uint32_t ba = su32(sm->act[slot]);
                umma_kblock(dt, sdesc(wa), sdesc(ba), idesc, kb != 0 ? 1u : 0u);
                umma_commit(&sm->w_empty[st]);
                ++wseq;
              }
              if (!ok) break;
              umma_commit(&sm->act_empty[slot]);
            }
            if (!ok) break;
            for (int mc = 0; mc < nmc; ++mc) umma_commit(&sm->acc_full[(accseq + mc) % NACC]);
            accseq += nmc;
            aseq += nkb;
            continue;
          }
          for (int mc = 0; mc < nmc && ok; ++mc) {
            const int buf = accseq % NACC;
            if (!mbar_wait(&sm->acc_empty[buf], ((accseq / NACC) & 1) ^ 1, sm, a.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t dt = tmem + (uint32_t)(buf * TR);
            for (int kb = 0; kb < nkb; ++kb) {
              const uint32_t as = aseq + kb;
              const int slot = as % NSLOT;
              if (mc == 0 && !mbar_wait(&sm->act_full[slot], (as / NSLOT) & 1, sm, a.status)) {
                ok = false;
                break;
              }
              const int st = wseq % NSTAGE;
              if (!mbar_wait(&sm->w_full[st], (wseq / NSTAGE) & 1, sm, a.status)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t wa = su32(sm->w[st]);
              const uint32_t ba = su32(sm->act[slot]);
              umma_kblock(dt, sdesc(wa), sdesc(ba), idesc, kb != 0 ? 1u : 0u);
              umma_commit(&sm->w_empty[st]);
              ++wseq;
              if (mc == nmc - 1) umma_commit(&sm->act_empty[slot]);
            }
            if (!ok) break;
            umma_commit(&sm->acc_full[buf]);
            ++accseq;
          }
          aseq += nkb;
        }
      umma_commit(&sm->done);
      mbar_wait(&sm->done, 0, sm, a.status);
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 0..15)
    const int q = warp & 3;          // TMEM lane quadrant: neurons 32q..32q+31 of an M chunk
    const int cg = warp >> 2;        // column group: tile rows 16cg..16cg+15
    const int r0 = 16 * cg;          // first tile row of this thread
    const int etid = threadIdx.x;    // 0..511
    const int pg = warp & 1;         // producer group: writes the K blocks kb with kb % 2 == pg
    const int gt = (warp >> 1) * 32 + lane;   // thread index within the producer group, 0..255
    const int prow = gt >> 2, pc16 = gt & 3;  // producer thread: tile row, 16 consecutive k
    uint32_t aseq = 0, accseq = 0, eseq = 0;
    bool ok = true;

    // hidden-layer biases, indexed by global hidden neuron, for the whole launch
    for (int i = 1; i < a.L; ++i)
      for (int j = etid; j < a.d[i]; j += NEPI * 32) sm->sbias[a.hoff[i] + j] = a.bias[i][j];

    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      // Every row of a tile belongs to one property (the rows are grouped by property before
      // the launch); slots past the property's last row are empty.
      const int p = a.tile_prop[tile];
      // ---------------- tile set-up, step 1: per-row scalars (one thread per row)
      if (etid < TR) {
        const int row = etid;
        const int r = a.rowmap[(size_t)tile * TR + row];
        int v = r >= 0 && r < a.R && p >= 0 && p < a.P;
        int k = 0, cnt = 0, off = 0;
        long long ab = 0, bb = 0;
        if (v) {
          const int b = r / a.K;
          k = r - b * a.K;
          cnt = a.bt.split_cnt[b];
          off = a.bt.split_off[b];
          const long long ao = a.bt.alpha_off[b];
          const int U = a.tb.U[p];
          ab = ao + (long long)k * U;
          bb = (long long)off * a.K + (long long)k * cnt;
          // every alpha of the row must lie in the array: then no per-element check is needed
          if (cnt < 0 || cnt > BCROWN_MAX_SPLITS || off < 0 || ab < 0 || ab + U > a.n_alpha) {
            atomicCAS(a.status, 0, BCROWN_ERR_ARG);
            v = 0;
          }
        }
        sm->valid[row] = v;
        sm->rowid[row] = v ? r : -1;
        sm->spec[row] = v ? k : 0;
        sm->scnt[row] = v ? cnt : 0;
        sm->soff[row] = off;
        sm->abase[row] = v ? ab : 0;
        sm->bbase[row] = v ? bb : 0;
        sm->part[0][row] = sm->part[1][row] = sm->part[2][row] = sm->part[3][row] = 0.f;
        const unsigned vb = __ballot_sync(0xffffffffu, v != 0);   // warps 0 and 1
        if (lane == 0) reinterpret_cast<uint32_t*>(&sm->vrows)[warp] = vb;
      }
      {
        // the property's per-neuron tables and input box
        const int pp = (p >= 0 && p < a.P) ? p : 0;
        // all loads first, then the stores (3 neurons and 2 inputs per thread at most)
        constexpr int NT = (MAX_H + NEPI * 32 - 1) / (NEPI * 32), NX = (MAX_D0 + NEPI * 32 - 1) / (NEPI * 32);
        int cd[NT], rk[NT];
        float sl[NT], ic[NT], xl[NX], xh[NX];
#pragma unroll
        for (int u = 0; u < NT; ++u) {
          const int nn = etid + u * NEPI * 32;
          const size_t g = (size_t)pp * a.H + nn;
          const bool in = nn < a.H;
          cd[u] = in ? a.tb.code[g] : 0;
          rk[u] = in ? a.tb.rank[g] : 0;
          sl[u] = in ? a.tb.slope[g] : 0.f;
          ic[u] = in ? a.tb.icpt[g] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < NX; ++u) {
          const int m = etid + u * NEPI * 32;
          const bool in = m < a.d[0];
          xl[u] = in ? a.x_lo[(size_t)pp * a.d[0] + m] : 0.f;
          xh[u] = in ? a.x_hi[(size_t)pp * a.d[0] + m] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < NT; ++u) {
          const int nn = etid + u * NEPI * 32;
          if (nn < a.H) {
            sm->tcode[nn] = ((uint32_t)cd[u] << 16) | (uint32_t)(rk[u] < 0 ? 0xFFFF : (rk[u] & 0xFFFF));
            sm->tslope[nn] = sl[u];
            sm->ticpt[nn] = ic[u];
          }
        }
#pragma unroll
        for (int u = 0; u < NX; ++u) {
          const int m = etid + u * NEPI * 32;
          if (m < a.d[0]) {
            sm->sxlo[m] = xl[u];
            sm->sxhi[m] = xh[u];
          }
        }
      }
      for (int x = etid; x < a.mask_words * TR; x += NEPI * 32) {
        (&sm->smask[0][0])[x] = 0u;
        (&sm->sneg[0][0])[x] = 0u;
      }
      if (etid < a.mask_words) sm->wrows[etid] = 0ull;
      if (!epi_sync(sm, eseq, a.status)) {
        ok = false;
        break;
      }
      // ---------------- step 2: split masks (8 threads per row) and the splits' beta
      int ent[BCROWN_MAX_SPLITS / 8];   // this thread's split entries: mask word << 5 | bit, or -1
      float bv[BCROWN_MAX_SPLITS / 8];  // and their beta (loaded now, stored in step 4)
      {
        const int row = etid >> 3, e0 = etid & 7;
        const int cnt = sm->scnt[row], off = sm->soff[row];
#pragma unroll
        for (int m = 0; m < BCROWN_MAX_SPLITS / 8; ++m) {
          const long long bi = sm->bbase[row] + e0 + 8 * m;
          bv[m] = ldg_f32(a.beta + bi, e0 + 8 * m < cnt && bi >= 0 && bi < a.n_beta);
        }
#pragma unroll
        for (int m = 0; m < BCROWN_MAX_SPLITS / 8; ++m) {
          const int e = e0 + 8 * m;
          ent[m] = -1;
          if (e < cnt) {
            const int ly = a.bt.split_layer[off + e];
            const int j = (int)a.bt.split_idx[off + e];
            const int s = a.bt.split_sign[off + e];
            if (ly < 1 || ly > a.L - 1 || j < 0 || j >= a.d[ly] || (s != 1 && s != -1)) {
              atomicCAS(a.status, 0, BCROWN_ERR_ARG);
            } else {
              const int wd = a.woff[ly] + (j >> 5);
              atomicOr(&sm->smask[wd][row], 1u << (j & 31));
              if (s == 1) atomicOr(&sm->sneg[wd][row], 1u << (j & 31));
              ent[m] = (wd << 5) | (j & 31);
            }
          }
        }
      }
      if (!epi_sync(sm, eseq, a.status)) {
        ok = false;
        break;
      }
      // ---------------- step 3: per-row split counts before each mask word (a prefix over the
      // row's 8 threads, 6 words each) and the rows with a split in each word (shared atomics)
      {
        const int row = etid >> 3, part = etid & 7;
        constexpr int WPT = MAX_MASK_WORDS / 8;
        int cw[WPT];
        int loc = 0;
#pragma unroll
        for (int u = 0; u < WPT; ++u) {
          const int w = part * WPT + u;
          const uint32_t m = w < a.mask_words ? sm->smask[w][row] : 0u;
          cw[u] = __popc(m);
          loc += cw[u];
          if (m) atomicOr(&sm->wrows[w], 1ull << row);
        }
        int incl = loc;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o, 8);
          if (part >= o) incl += y;
        }
        int run = incl - loc;
#pragma unroll
        for (int u = 0; u < WPT; ++u) {
          const int w = part * WPT + u;
          if (w < a.mask_words) sm->wfirst[w][row] = (uint8_t)run;
          run += cw[u];
        }
      }
      if (!epi_sync(sm, eseq, a.status)) {
        ok = false;
        break;
      }
      // ---------------- step 4: each split's slot in (word, bit) order, its list position and beta
      {
        const int row = etid >> 3, e0 = etid & 7;
#pragma unroll
        for (int m = 0; m < BCROWN_MAX_SPLITS / 8; ++m) {
          if (ent[m] >= 0) {
            const int ks = split_slot(sm, row, ent[m] >> 5, ent[m] & 31);
            sm->sorig[row][ks] = (uint8_t)(e0 + 8 * m);
            sm->sbeta[row][ks] = fmaxf(bv[m], 0.f);
          }
        }
      }
      if (!epi_sync(sm, eseq, a.status)) {
        ok = false;
        break;
      }
      // rows of this thread that take part (bit c: tile row r0 + c); empty rows have all-zero
      // operands, so they only need their global loads and stores masked
      const uint32_t vbits = (uint32_t)(sm->vrows >> r0) & 0xFFFFu;

      // per-thread lb partial sums of its 16 rows over the lanes' neurons (whole backward pass)
      float racc[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) racc[c] = 0.f;

      // ---------------- backward pass: A^(i-1) = Lambda^(i) W^(i) from the accumulator, relaxed
      // into the next operand Lambda^(i-1).  i = L is the top: A^(L-1) = Wbar (no contraction).
      for (int i = a.L; i >= 1 && ok; --i) {
        const bool top = (i == a.L);
        const int N = a.d[i - 1];
        const int nmc = nmc_of(N);
        const bool concretise = (i == 1);
        const int li = i - 1;
        const int nkb_next = concretise ? 0 : nkb_of(N);
        for (int mc = 0; mc < nmc && ok; ++mc) {
          const int buf = accseq % NACC;
          const int j = mc * MCH + 32 * q + lane;   // output neuron of this lane
          const bool jin = j < N;
          if (concretise) {
            // ---- lb += sum_m min(A_m x_lo_m, A_m x_hi_m) (Eq. beta_crown_lp); sign bits of A^(0) for x*
            const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * TR + r0);
            const float uxl = jin ? sm->sxlo[j] : 0.f, uxh = jin ? sm->sxhi[j] : 0.f;
            if (!mbar_wait_warp(&sm->acc_full[buf], (accseq / NACC) & 1, sm, a.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              float v[8];
              tmem_ld8(tbase + 8 * h, v);
              if (h == 1) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm->acc_empty[buf]);
                ++accseq;
              }
#pragma unroll
              for (int c8 = 0; c8 < 8; ++c8) {
                const int c = 8 * h + c8;
                const float av = v[c8];
                racc[c] += fminf(av * uxl, av * uxh);
                if constexpr (MODE >= 1) {
                  const unsigned bits = __ballot_sync(0xffffffffu, jin && av >= 0.f);
                  if (lane == 0 && mc * MCH + 32 * q < MAX_D0) sm->sign[r0 + c][(mc * MCH + 32 * q) >> 5] = bits;
                }
              }
            }
            continue;
          }
          // ---- relaxation of layer i-1 (Lemma 2.1 / Eq. definition_D, split override of Eq. 3)
          // D = 1 active, 0 inactive; unstable: alpha where A >= 0, the chord slope (+ intercept
          // lambda) where A < 0; a split neuron takes D = 1 or 0 and adds beta S.
          const long long n = a.hoff[li] + j;
          int code = CODE_INACTIVE, rank = 0;
          float dneg = 0.f, lneg = 0.f, bj = 0.f;
          if (jin) {
            bj = sm->sbias[n];
            const uint32_t t = sm->tcode[n];
            code = (int)(t >> 16);
            rank = (int)(t & 0xFFFF);
            dneg = code == CODE_ACTIVE ? 1.f : (code == CODE_UNSTABLE ? sm->tslope[n] : 0.f);
            lneg = code == CODE_UNSTABLE ? sm->ticpt[n] : 0.f;
          }
          const bool unst = code == CODE_UNSTABLE;
          const float apos = code == CODE_ACTIVE ? 1.f : 0.f;
          const int kb = (mc * MCH + 32 * q) / KBLK;   // this warp's K block of the next operand
          const bool writer = kb < nkb_next;
          const uint32_t as = aseq + kb;
          const int slot = as % NSLOT;
          // split bits of the warp's 32 neurons (none when they all lie past the layer's end)
          const int wd = a.woff[li] + ((mc * MCH + 32 * q) >> 5);
          const uint32_t bit = 1u << lane;
          const uint32_t rbits = mc * MCH + 32 * q < N ? (uint32_t)(sm->wrows[wd] >> r0) & 0xFFFFu : 0u;
          // alpha of the 16 rows, issued before waiting for the accumulator
          float al[16];
#pragma unroll
          for (int c = 0; c < 16; ++c) al[c] = ldg_f32(a.alpha + sm->abase[r0 + c] + rank, unst && ((vbits >> c) & 1u));
          // byte offset of (row r0 + 8h + c8, k = j % 64) in the slot: row & 7 == c8
          const int kk = j & (KBLK - 1);
          uint8_t* aslot = sm->act[slot] + r0 * 128 + ((kk & 7) << 1);
          const uint32_t kx = (uint32_t)(kk >> 3) << 4;
          // rows r0 + 8h .. r0 + 8h + 7 of A^(i-1)_j: relaxation, lb terms, operand and stash
          auto relax8 = [&](const int h, const float (&v)[8]) {
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) {
              const int c = 8 * h + c8;
              const int row = r0 + c;
              const float av = v[c8];
              const bool pos = av >= 0.f;
              float D = pos ? __saturatef(al[c] + apos) : dneg;
              float lm = pos ? 0.f : lneg;
              float bs = 0.f;
              if ((rbits >> c) & 1u) {
                if (sm->smask[wd][row] & bit) {
                  const int sg = (sm->sneg[wd][row] & bit) ? 1 : -1;
                  D = sg == -1 ? 1.f : 0.f;
                  lm = 0.f;
                  bs = sm->sbeta[row][split_slot(sm, row, wd, lane)] * (float)sg;
                }
              }
              const float L = fmaf(av, D, bs);
              racc[c] = fmaf(L, bj, fmaf(av, lm, racc[c]));
              if (writer)
                *reinterpret_cast<__nv_bfloat16*>(aslot + (8 * h + c8) * 128 + (kx ^ (uint32_t)(c8 << 4))) =
                    __float2bfloat16_rn(L);
            }
            if constexpr (MODE >= 1) {
              // A^(i-1) of the 8 rows for the adjoint pass: one 16-byte store per lane
              if (jin) {
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                  __nv_bfloat162 v2 = __floats2bfloat162_rn(v[e], v[e + 1]);
                  pk[e >> 1] = *reinterpret_cast<uint32_t*>(&v2);
                }
                stg_v4(a.stash + ((size_t)tile * a.H + n) * TR + r0 + 8 * h, make_uint4(pk[0], pk[1], pk[2], pk[3]));
              }
            }
          };
          if (!top) {
            if (!mbar_wait_warp(&sm->acc_full[buf], (accseq / NACC) & 1, sm, a.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          if (writer && !mbar_wait_warp(&sm->act_empty[slot], ((as / NSLOT) & 1) ^ 1, sm, a.status)) {
            ok = false;
            break;
          }
          const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * TR + r0);
          if (top) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              // A^(L-1) = Wbar rows of the rows' specifications
              float v[8];
#pragma unroll
              for (int c8 = 0; c8 < 8; ++c8) {
                const int c = 8 * h + c8;
                v[c8] = ldg_f32(a.Wbar + (size_t)sm->spec[r0 + c] * N + j, jin && ((vbits >> c) & 1u));
              }
              relax8(h, v);
            }
          } else {
            // rows r0..r0+7, then r0+8..r0+15: the second load runs under the first half's work
            uint32_t u0[8], u1[8];
            tmem_ld8_issue(tbase, u0);
            tmem_wait8(u0);
            tmem_ld8_issue(tbase + 8, u1);
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(u0[e]);
            relax8(0, v);
            tmem_wait8(u1);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm->acc_empty[buf]);
            ++accseq;
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(u1[e]);
            relax8(1, v);
          }
          // each K block is complete once its 8 writer warps arrived
          if (writer) {
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm->act_full[slot]);
          }
        }
        aseq += nkb_next;
      }
      if (!ok) break;

      // ---------------- lb of each row: reduce the lanes' partial sums, then the quadrants'
      {
        const float rs = reduce16(racc);
        if ((lane & 1) == 0) atomicAdd(&sm->part[q][r0 + (lane >> 1)], rs);
      }
      if (!epi_sync(sm, eseq, a.status)) {
        ok = false;
        break;
      }
      if (etid < TR && sm->valid[etid]) {
        const int row = etid;
        float lbv = a.bbar[sm->spec[row]] + ((sm->part[0][row] + sm->part[1][row]) + (sm->part[2][row] + sm->part[3][row]));
        if (!isfinite(lbv)) {
          atomicCAS(a.status, 0, BCROWN_ERR_NONFINITE);
          lbv = -INFINITY;
        }
        a.lb[sm->rowid[row]] = lbv;
      }
      if constexpr (MODE == 0) continue;

      // ---------------- adjoint: x* operand (K blocks of d0), then forward contractions
      {
        const int d0 = a.d[0];
        const int nkb = nkb_of(d0);
        const bool rv = sm->valid[prow] != 0;
        for (int kb = pg; kb < nkb && ok; kb += 2) {
          const uint32_t as = aseq + kb;
          const int slot = as % NSLOT;
          if (!mbar_wait_warp(&sm->act_empty[slot], ((as / NSLOT) & 1) ^ 1, sm, a.status)) {
            ok = false;
            break;
          }
          uint32_t pk[8];
#pragma unroll
          for (int e = 0; e < 16; e += 2) {
            float xv[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int m = kb * KBLK + pc16 * 16 + e + h;
              float x = 0.f;
              if (m < d0 && rv) {
                // x* minimises A^(0) x over the box: x_lo where A^(0) >= 0, else x_hi
                const bool pos = (sm->sign[prow][m >> 5] >> (m & 31)) & 1u;
                x = pos ? sm->sxlo[m] : sm->sxhi[m];
              }
              xv[h] = x;
            }
            __nv_bfloat162 v2 = __floats2bfloat162_rn(xv[0], xv[1]);
            pk[e >> 1] = *reinterpret_cast<uint32_t*>(&v2);
          }
          *reinterpret_cast<uint4*>(sm->act[slot] + act_off(prow, pc16 * 16)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          *reinterpret_cast<uint4*>(sm->act[slot] + act_off(prow, pc16 * 16 + 8)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sm->act_full[slot]);
        }
        aseq += nkb;
      }
      // zhat^(i) = W^(i) h^(i-1) + b^(i); dalpha = A zhat (unstable, unsplit, A >= 0), dbeta = S zhat;
      // h^(i) = D zhat + lambda is the next forward operand
      for (int i = 1; i <= a.L - 1 && ok; ++i) {
        const int N = a.d[i];
        const int nmc = nmc_of(N);
        const int nkb_next = (i + 1 <= a.L - 1) ? nkb_of(N) : 0;
        for (int mc = 0; mc < nmc && ok; ++mc) {
          const int buf = accseq % NACC;
          const int j = mc * MCH + 32 * q + lane;
          const bool jin = j < N;
          const long long n = a.hoff[i] + j;
          int code = CODE_INACTIVE, rank = 0;
          float dneg = 0.f, lneg = 0.f, bj = 0.f;
          if (jin) {
            bj = sm->sbias[n];
            const uint32_t t = sm->tcode[n];
            code = (int)(t >> 16);
            rank = (int)(t & 0xFFFF);
            dneg = code == CODE_ACTIVE ? 1.f : (code == CODE_UNSTABLE ? sm->tslope[n] : 0.f);
            lneg = code == CODE_UNSTABLE ? sm->ticpt[n] : 0.f;
          }
          const bool unst = code == CODE_UNSTABLE;
          const float apos = code == CODE_ACTIVE ? 1.f : 0.f;
          const int kb = (mc * MCH + 32 * q) / KBLK;
          const bool writer = kb < nkb_next;
          const uint32_t as = aseq + kb;
          const int slot = as % NSLOT;
          const int wd = a.woff[i] + ((mc * MCH + 32 * q) >> 5);
          const uint32_t bit = 1u << lane;
          const uint32_t rbits = mc * MCH + 32 * q < N ? (uint32_t)(sm->wrows[wd] >> r0) & 0xFFFFu : 0u;
          // A^(i) of the 16 rows (two 16-byte loads) and alpha, issued before the accumulator wait
          const __nv_bfloat16* sp = a.stash + ((size_t)tile * a.H + n) * TR + r0;
          const uint4 s0 = ldg_v4(sp, jin), s1 = ldg_v4(sp + 8, jin);
          float al[16];
#pragma unroll
          for (int c = 0; c < 16; ++c) al[c] = ldg_f32(a.alpha + sm->abase[r0 + c] + rank, unst && ((vbits >> c) & 1u));
          if (!mbar_wait_warp(&sm->acc_full[buf], (accseq / NACC) & 1, sm, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (writer && !mbar_wait_warp(&sm->act_empty[slot], ((as / NSLOT) & 1) ^ 1, sm, a.status)) {
            ok = false;
            break;
          }
          const int kk = j & (KBLK - 1);
          uint8_t* aslot = sm->act[slot] + r0 * 128 + ((kk & 7) << 1);
          const uint32_t kx = (uint32_t)(kk >> 3) << 4;
          const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * TR + r0);
          // rows r0 + 8h .. r0 + 8h + 7: zhat, gradients, next operand
          auto fwd8 = [&](const int h, const uint32_t (&u)[8]) {
            const uint4 sw = h == 0 ? s0 : s1;
            const uint32_t swv[4] = {sw.x, sw.y, sw.z, sw.w};
#pragma unroll
            for (int c8 = 0; c8 < 8; ++c8) {
              const int c = 8 * h + c8;
              const int row = r0 + c;
              const bool rin = (vbits >> c) & 1u;
              const float A = __uint_as_float((c8 & 1) ? (swv[c8 >> 1] & 0xFFFF0000u) : (swv[c8 >> 1] << 16));
              const float z = __uint_as_float(u[c8]) + bj;
              const bool pos = A >= 0.f;
              float D = pos ? __saturatef(al[c] + apos) : dneg;
              float lm = pos ? 0.f : lneg;
              float g = pos ? A * z : 0.f;
              if ((rbits >> c) & 1u) {
                if (sm->smask[wd][row] & bit) {
                  const int sg = (sm->sneg[wd][row] & bit) ? 1 : -1;
                  D = sg == -1 ? 1.f : 0.f;
                  lm = 0.f;
                  g = 0.f;
                  const long long bi = sm->bbase[row] + sm->sorig[row][split_slot(sm, row, wd, lane)];
                  if (bi < a.n_beta) a.dbeta[bi] = (float)sg * z;
                }
              }
              if (unst && rin) {
                if constexpr (MODE == 2) a.dalpha16[sm->abase[row] + rank] = __float2bfloat16_rn(g);
                else a.dalpha[sm->abase[row] + rank] = g;
              }
              const float hv = rin ? fmaf(D, z, lm) : 0.f;
              if (writer)
                *reinterpret_cast<__nv_bfloat16*>(aslot + (8 * h + c8) * 128 + (kx ^ (uint32_t)(c8 << 4))) =
                    __float2bfloat16_rn(hv);
            }
          };
          uint32_t u0[8], u1[8];
          tmem_ld8_issue(tbase, u0);
          tmem_wait8(u0);
          tmem_ld8_issue(tbase + 8, u1);
          fwd8(0, u0);
          tmem_wait8(u1);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sm->acc_empty[buf]);
          ++accseq;
          fwd8(1, u1);
          if (writer) {
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm->act_full[slot]);
          }
        }
        aseq += nkb_next;
      }
      if (ok && !epi_sync(sm, eseq, a.status)) ok = false;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NACC * TR) : "memory");
  }
}

// ------------------------------------------------------------------------------------------
// Row planner: group the rows (subdomain, spec) by property into tiles of TR rows, so that the
// fused kernel stages one property's tables per tile.  Row results do not depend on the tile a
// row lands in (each row is one column of every contraction), so the order inside a property
// is free; it is taken from atomic counters.
// ------------------------------------------------------------------------------------------
__global__ void k_plan_count(int B, int P, const int32_t* __restrict__ prop_of, int* __restrict__ cnt, int* status) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    const int p = prop_of[b];
    if (p < 0 || p >= P) {
      atomicCAS(status, 0, BCROWN_ERR_ARG);
      continue;
    }
    atomicAdd(&cnt[p], 1);
  }
}

// Exclusive prefix sums over the properties of their subdomains and of their tiles (one block).
__global__ void __launch_bounds__(1024) k_plan_scan(int P, int K, const int* __restrict__ cnt, int* __restrict__ cursor,
                                                    int* __restrict__ sub_base, int* __restrict__ tile_base,
                                                    int* __restrict__ n_tiles) {
  __shared__ int ws[32], wt[32];
  __shared__ int run_s, run_t;
  if (threadIdx.x == 0) run_s = run_t = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < P; base += blockDim.x) {
    const int p = base + threadIdx.x;
    const int c = p < P ? cnt[p] : 0;
    const int t = (int)(((long long)c * K + TR - 1) / TR);
    int is = c, it = t;   // inclusive scans within the warp
    for (int o = 1; o < 32; o <<= 1) {
      const int xs = __shfl_up_sync(0xffffffffu, is, o), xt = __shfl_up_sync(0xffffffffu, it, o);
      if (lane >= o) {
        is += xs;
        it += xt;
      }
    }
    if (lane == 31) {
      ws[w] = is;
      wt[w] = it;
    }
    __syncthreads();
    int os = run_s, ot = run_t;
    for (int q = 0; q < w; ++q) {
      os += ws[q];
      ot += wt[q];
    }
    if (p < P) {
      sub_base[p] = os + is - c;
      tile_base[p] = ot + it - t;
      cursor[p] = 0;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) {
      run_s = os + is;
      run_t = ot + it;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sub_base[P] = run_s;
    tile_base[P] = run_t;
    *n_tiles = run_t;
  }
}

__global__ void k_plan_scatter(int B, int P, const int32_t* __restrict__ prop_of, const int* __restrict__ sub_base,
                               int* __restrict__ cursor, int* __restrict__ perm) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    const int p = prop_of[b];
    if (p < 0 || p >= P) continue;
    perm[sub_base[p] + atomicAdd(&cursor[p], 1)] = b;
  }
}

// Slot s of tile t: the property whose tiles contain t, and the global row in that slot.
__global__ void k_plan_rows(int max_tiles, int K, int P, const int* __restrict__ n_tiles,
                            const int* __restrict__ tile_base, const int* __restrict__ sub_base,
                            const int* __restrict__ perm, int* __restrict__ tile_prop, int* __restrict__ rowmap) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)max_tiles * TR) return;
  const int t = (int)(id / TR), sl = (int)(id - (long long)t * TR);
  if (t >= *n_tiles) {
    rowmap[id] = -1;
    if (sl == 0) tile_prop[t] = -1;
    return;
  }
  int lo = 0, hi = P - 1;   // smallest p with tile_base[p + 1] > t
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (tile_base[mid + 1] > t) hi = mid;
    else lo = mid + 1;
  }
  const int p = lo;
  const long long i = (long long)(t - tile_base[p]) * TR + sl;
  const long long rows_p = (long long)(sub_base[p + 1] - sub_base[p]) * K;
  rowmap[id] = i < rows_p ? (int)((long long)perm[sub_base[p] + i / K] * K + i % K) : -1;
  if (sl == 0) tile_prop[t] = p;
}

// ------------------------------------------------------------------------------------------
}  // namespace tc

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------
using namespace tc;

struct TcNet {
  bool ready = false;
  std::vector<__nv_bfloat16*> bufs;
  Maps maps;
  int box_bwd[MAXL + 1] = {0};
  int box_fwd[MAXL + 1] = {0};
  int woff[MAXL + 1] = {0};
  int mask_words = 0;
  // conv layers on the tensor cores: BF16 weight matrices [Np][Kp] for the backward (rows =
  // input channels) and the forward (rows = output channels), with their TMA maps
  bool conv_ready = false;
};

static std::mutex g_tc_mu;
static std::vector<std::pair<const bcrown_net*, TcNet*>> g_tc;

static TcNet* tc_of(const bcrown_net* net) {
  std::lock_guard<std::mutex> g(g_tc_mu);
  for (auto& e : g_tc)
    if (e.first == net) return e.second;
  TcNet* t = new TcNet();
  g_tc.push_back({net, t});
  return t;
}

bool tc_supported(const bcrown_net* net) {
  if (net->L < 2 || net->L > MAXL) return false;
  if (net->d[0] > MAX_D0) return false;
  int words = 0;
  for (int i = 0; i < net->L; ++i)
    if (net->ly[i].kind != BCROWN_LAYER_FC) return false;
  for (int i = 1; i < net->L; ++i) {
    if (net->d[i] > MAX_HIDDEN) return false;
    words += (net->d[i] + 31) / 32;
  }
  if (words > MAX_MASK_WORDS || net->H > MAX_H) return false;
  // the forward contraction of layer 1 streams d0 in K blocks: its M chunks must fit the
  // accumulator ring (hidden widths <= 256 give at most 2)
  if ((net->d[1] + MCH - 1) / MCH > NACC) return false;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaGetLastError();
  return major == 10 && minor == 3;
}

// Tiles the planner can produce: every property may end in one partly filled tile.
static long long max_tiles_of(int B, int K, int P) { return ((long long)B * K + TR - 1) / TR + P; }

// Workspace: the row plan (counters, prefix sums, permutation, tile -> property, row map), then,
// for the gradient, the BF16 stash [tile][H][TR].
struct TcPlan {
  int *cnt, *cursor, *sub_base, *tile_base, *n_tiles, *perm, *tile_prop, *rowmap;
  __nv_bfloat16* stash;
};
static size_t carve(char* base, int B, int K, int P, int H, bool grad, TcPlan* out) {
  const long long T = max_tiles_of(B, K, P);
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  TcPlan pl;
  pl.cnt = (int*)take((size_t)(P + 1) * 4);
  pl.cursor = (int*)take((size_t)(P + 1) * 4);
  pl.sub_base = (int*)take((size_t)(P + 1) * 4);
  pl.tile_base = (int*)take((size_t)(P + 1) * 4);
  pl.n_tiles = (int*)take(4);
  pl.perm = (int*)take((size_t)std::max(B, 1) * 4);
  pl.tile_prop = (int*)take((size_t)T * 4);
  pl.rowmap = (int*)take((size_t)T * TR * 4);
  pl.stash = grad ? (__nv_bfloat16*)take((size_t)T * TR * std::max(H, 1) * sizeof(__nv_bfloat16)) : nullptr;
  if (out) *out = pl;
  return off;
}

size_t tc_workspace_bytes(const bcrown_net* net, int B, int P, bool grad) {
  return carve(nullptr, B, net->K, P, net->H, grad, nullptr);
}


// BF16 copy of a [rows][cols] FP32 matrix with the row length padded to a multiple of 64.
static int padded_bf16(const float* src_dev, int rows, int cols, __nv_bfloat16** out, int* kp) {
  *kp = (cols + KBLK - 1) / KBLK * KBLK;
  std::vector<float> h((size_t)rows * cols);
  if (cudaMemcpy(h.data(), src_dev, h.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(BCROWN_ERR_CUDA, "copy of weights");
  std::vector<__nv_bfloat16> p((size_t)rows * *kp, __float2bfloat16_rn(0.f));
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) p[(size_t)r * *kp + c] = __float2bfloat16_rn(h[(size_t)r * cols + c]);
  if (cudaMalloc(out, p.size() * 2) != cudaSuccess) return fail(BCROWN_ERR_OOM, "bf16 weights");
  if (cudaMemcpy(*out, p.data(), p.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(BCROWN_ERR_CUDA, "bf16 weights upload");
  return BCROWN_OK;
}

static int tc_prepare(bcrown_net* net, TcNet* t) {
  if (t->ready) return BCROWN_OK;
  memset(&t->maps, 0, sizeof(t->maps));
  int w = 0;
  for (int i = 1; i < net->L; ++i) {
    t->woff[i] = w;
    w += (net->d[i] + 31) / 32;
  }
  t->mask_words = w;
  for (int i = 1; i < net->L; ++i) {
    const LayerDev& l = net->ly[i - 1];
    // backward: rows = d_{i-1} output neurons, K = d_i
    __nv_bfloat16* wt = nullptr;
    int kp = 0;
    BC_CHECK(padded_bf16(l.Wt, l.d_in, l.d_out, &wt, &kp));
    t->bufs.push_back(wt);
    t->box_bwd[i] = MCH;
    BC_CHECK(encode_map(&t->maps.bwd[i], wt, l.d_in, kp, t->box_bwd[i]));
    // forward: rows = d_i output neurons, K = d_{i-1}
    __nv_bfloat16* wf = nullptr;
    BC_CHECK(padded_bf16(l.W, l.d_out, l.d_in, &wf, &kp));
    t->bufs.push_back(wf);
    t->box_fwd[i] = MCH;
    BC_CHECK(encode_map(&t->maps.fwd[i], wf, l.d_out, kp, t->box_fwd[i]));
  }
  BC_CUDA(cudaFuncSetAttribute(k_fused<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem) + 1024));
  BC_CUDA(cudaFuncSetAttribute(k_fused<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem) + 1024));
  BC_CUDA(cudaFuncSetAttribute(k_fused<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem) + 1024));
  t->ready = true;
  return BCROWN_OK;
}

static int tc_launch(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* bt, const Tables& tb, Args& A,
                     char* ws, size_t ws_bytes, int mode, bool plan, cudaStream_t s) {
  const bool grad = mode >= 1;
  TcNet* t = tc_of(net);
  BC_CHECK(tc_prepare(net, t));
  const int B = bt->B, K = net->K, P = dom->n_props;
  const int R = B * K;
  if (R == 0) return BCROWN_OK;
  if (!ws || ws_bytes < tc_workspace_bytes(net, B, P, grad))
    return fail(BCROWN_ERR_OOM, "tensor-core workspace too small");
  TcPlan pl;
  carve(ws, B, K, P, net->H, grad, &pl);
  const long long T = max_tiles_of(B, K, P);
  if (plan) {
    BC_CUDA(cudaMemsetAsync(pl.cnt, 0, (size_t)(P + 1) * 4, s));
    const int gb = (int)std::min<long long>((B + 255) / 256, 4096);
    k_plan_count<<<gb, 256, 0, s>>>(B, P, bt->prop_of, pl.cnt, net->status);
    k_plan_scan<<<1, 1024, 0, s>>>(P, K, pl.cnt, pl.cursor, pl.sub_base, pl.tile_base, pl.n_tiles);
    k_plan_scatter<<<gb, 256, 0, s>>>(B, P, bt->prop_of, pl.sub_base, pl.cursor, pl.perm);
    k_plan_rows<<<(int)((T * TR + 255) / 256), 256, 0, s>>>((int)T, K, P, pl.n_tiles, pl.tile_base, pl.sub_base,
                                                           pl.perm, pl.tile_prop, pl.rowmap);
    g_launches += 4;
  }
  A.L = net->L;
  A.K = K;
  A.P = P;
  A.H = net->H;
  A.R = R;
  A.n_tiles = pl.n_tiles;
  A.tile_prop = pl.tile_prop;
  A.rowmap = pl.rowmap;
  A.stash = pl.stash;
  for (int i = 0; i <= net->L && i <= MAXL; ++i) A.d[i] = net->d[i];
  for (int i = 1; i < net->L; ++i) {
    A.hoff[i] = net->hoff[i - 1];
    A.woff[i] = t->woff[i];
    A.bias[i] = net->ly[i - 1].b;
    A.box_bwd[i] = t->box_bwd[i];
    A.box_fwd[i] = t->box_fwd[i];
  }
  A.mask_words = t->mask_words;
  A.Wbar = net->Wbar;
  A.bbar = net->bbar;
  A.bt = BatchView{bt->B, bt->prop_of, bt->split_off, bt->split_cnt, bt->split_layer, bt->split_idx, bt->split_sign,
                   bt->alpha_off};
  A.tb = tb;
  A.x_lo = dom->x_lo;
  A.x_hi = dom->x_hi;
  A.n_alpha = bt->n_alpha;
  A.n_beta = bt->n_beta;
  A.status = net->status;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one CTA per SM at most; the planned tile count (at most T) is read on the device
  const int grid = (int)std::min<long long>(T, sms);
  {
    ProfScope ps(net, BCROWN_PROF_FUSED, s);
    if (mode == 2)
      k_fused<2><<<grid, NTHREADS, sizeof(Smem) + 1024, s>>>(t->maps, A);
    else if (mode == 1)
      k_fused<1><<<grid, NTHREADS, sizeof(Smem) + 1024, s>>>(t->maps, A);
    else
      k_fused<0><<<grid, NTHREADS, sizeof(Smem) + 1024, s>>>(t->maps, A);
    ++g_launches;
  }
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

int tc_bound(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* bt, const Tables& tb, char* ws,
             size_t ws_bytes, bool grad, bool plan, const float* alpha, const float* beta, float* lb, float* dalpha,
             float* dbeta, cudaStream_t s, __nv_bfloat16* dalpha16) {
  Args A;
  memset(&A, 0, sizeof(A));
  A.alpha = alpha;
  A.beta = beta;
  A.lb = lb;
  A.dalpha = dalpha;
  A.dalpha16 = dalpha16;
  A.dbeta = dbeta;
  return tc_launch(net, dom, bt, tb, A, ws, ws_bytes, !grad ? 0 : (dalpha16 ? 2 : 1), plan, s);
}

void tc_release(const bcrown_net* net) {
  std::lock_guard<std::mutex> g(g_tc_mu);
  for (size_t i = 0; i < g_tc.size(); ++i)
    if (g_tc[i].first == net) {
      for (auto* b : g_tc[i].second->bufs) cudaFree(b);
      delete g_tc[i].second;
      g_tc.erase(g_tc.begin() + i);
      return;
    }
}

}  // namespace bcrown
