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
// alpha, the per-neuron tables, Adam state and the stash coalesced across a warp.
//
// The epilogue (16 warps) reads the accumulator with tcgen05.ld, applies the relaxation of
// Lemma 2.1 / Eq. definition_D (split overriding stability), the beta shift and the bias
// sums (Lambda = A D + beta S; c += Lambda b + A lambda), and writes Lambda^(i-1) in BF16
// as the next contraction's operand.  The last contraction is concretised over the box
// (Eq. beta_crown_lp).  With a gradient requested the adjoint pass follows in the same
// launch: zhat^(i) = W^(i) h^(i-1) + b^(i) along h^(0) = x*, dalpha = A zhat, dbeta = S zhat,
// h = D zhat + lambda; in optimiser mode the projected Adam step (Appendix C.1) and the
// per-row best tracking are applied to alpha and beta in that epilogue.
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

namespace bcrown {

extern std::atomic<long long> g_launches;

namespace tc {

constexpr int TR = 64;            // rows per tile = MMA N
constexpr int MCH = 128;          // neurons per M chunk = MMA M
constexpr int KBLK = 64;          // bf16 per K block (128 bytes, one swizzle row)
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
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// As mbar_try, but a thread whose phase is not complete yet is suspended (for at most about
// `ns` nanoseconds) until it completes, instead of returning at once: waiting threads then
// leave the issue slots and the shared-memory pipe to the warps doing work.
__device__ __forceinline__ bool mbar_try_sleep(uint64_t* b, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
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
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          su32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Barrier among the 16 epilogue warps built on an mbarrier, so that a warp that gives up
// after a timeout cannot leave the others blocked: every wait here is bounded.
__device__ __forceinline__ bool epi_sync(Smem* sm, uint32_t& seq, int* status);

// Shared-memory matrix descriptor, K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
  return d;
}
// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(MCH >> 4) << 24);
}
// One 64-wide K block: four MMAs of K = 16.  Descriptors of consecutive 16-element K steps
// differ by 32 bytes in the start address (field unit 16 bytes: +2); `acc` = 0 starts the
// accumulator with the first MMA.
__device__ __forceinline__ void umma_kblock(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %4, 0;\n\tsetp.eq.b32 q, 0, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %5, %6, %3, q;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %7, %8, %3, q;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %9, %10, %3, q;\n\t}" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc), "l"(ad + 2), "l"(bd + 2), "l"(ad + 4), "l"(bd + 4), "l"(ad + 6),
      "l"(bd + 6)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Split form of tmem_ld8: the load, then the wait.  The wait names the registers as in-out
// operands, so no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_ld8_issue(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait8(uint32_t (&r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
}

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
// Col is gathered into BF16 by k_im2col from a per-K table (source channel offset, signed tap
// offsets: no divisions in the inner loop); k_tcg multiplies it with the BF16 weights:
// M = rows x positions (tiles of 128 on the TMEM lanes), N = channels (padded to 16), K in
// blocks of 64 streamed by TMA.
// ------------------------------------------------------------------------------------------
constexpr int TCG_NS = 4;         // pipeline stages (A: 128 x 64, B: Np x 64)
constexpr int TCG_THREADS = 192;  // warps 0-3 epilogue, 4 TMA, 5 MMA

// One gather: row m = (r, pp), pp = i * nJ + j; source position (y0 + dy_K, x0 + dx_K) with
// y0 = i * ms + cy, x0 = j * ms + cx, in a [C][Hs][Ws] map of row r (d_src floats per row).
struct Im2colPass {
  long long M;
  int Pm, nJ, ms, cy, cx, Hs, Ws, d_src, Kp;
  const int2* tab;  // [Kp]: {channel offset C * Hs * Ws, or -1 for a zero column; (dy & 0xffff) | dx << 16}
};

// 32 consecutive rows m per block.  Lanes walk the 32 rows for one pair of K at a time (K
// uniform per warp: coalesced source reads) into a shared tile [32][Kp + 8], whose rows then
// leave in 16-byte stores.
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
  const int y0 = i * q.ms + q.cy, x0 = j * q.ms + q.cx;
  const float* sr = src + (size_t)r * q.d_src;
  __syncthreads();
  for (int K = 2 * w; K < Kp; K += 16) {
    float v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int2 t = tab[K + e];
      const int y = y0 + (int)(short)(t.y & 0xffff), x = x0 + (t.y >> 16);
      v[e] = (mv && t.x >= 0 && (unsigned)y < (unsigned)q.Hs && (unsigned)x < (unsigned)q.Ws)
                 ? sr[t.x + y * q.Ws + x]
                 : 0.f;
    }
    *reinterpret_cast<__nv_bfloat162*>(tile + lane * S + K) = __floats2bfloat162_rn(v[0], v[1]);
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

// Where k_tcg writes: row m = (r, pp), pp = i * nJ + j, goes to position
// p = (a + so * i) * Wo + (b + so * j) of out[r * stride + n * P + p] (+ bias[n * P + p]).
struct TcgOut {
  long long M;
  int N, Np, nkb, brow;  // brow: first row of the weight operand's tile in its tensor map
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

// out[r * stride + n * P + p] = (Col x W^T)[m = r * P + p][n] (+ bias[n * P + p]) for n < N.
__global__ void __launch_bounds__(TCG_THREADS, 1) k_tcg(const __grid_constant__ CUtensorMap mapA,
                                                        const __grid_constant__ CUtensorMap mapB, TcgOut o,
                                                        float* __restrict__ out, const float* __restrict__ bias,
                                                        int* status) {
  const long long M = o.M;
  const int N = o.N, Np = o.Np, nkb = o.nkb;
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
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long ntiles = (M + 127) / 128;
  // two accumulators of Np columns, allocated as a power of two >= 32
  const uint32_t tcols = Np <= 16 ? 32u : (Np <= 32 ? 64u : (Np <= 64 ? 128u : (Np <= 128 ? 256u : 512u)));
  if (threadIdx.x == 0) {
    for (int i = 0; i < TCG_NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tbase_sm)), "r"(tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tbase_sm;
  if (warp == 4) {
    if (lane == 0) {
      uint32_t seq = 0;
      bool ok = true;
      for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
        for (int kb = 0; kb < nkb; ++kb, ++seq) {
          const int st = seq % TCG_NS;
          if (!tcg_wait(&empty[st], ((seq / TCG_NS) & 1) ^ 1, abort, status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[st], 16384u + (uint32_t)bbytes);
          tma_load_2d(sA + st * 16384, &mapA, kb * 64, (int)(tile * 128), &full[st]);
          tma_load_2d(sB + st * bbytes, &mapB, kb * 64, o.brow, &full[st]);
        }
      if (!ok) {
        for (uint32_t q = (seq > TCG_NS ? seq - TCG_NS : 0); q < seq; ++q) {
          long long t0 = clock64();
          while (!mbar_try(&full[q % TCG_NS], (q / TCG_NS) & 1) && clock64() - t0 < 200000000LL) {
          }
        }
      }
    }
  } else if (warp == 5) {
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
  } else {
    // epilogue: warp w owns TMEM lanes (tile rows) 32w..32w+31
    uint32_t accseq = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++accseq) {
      const int buf = accseq & 1;
      int okw = 1;
      if (lane == 0) okw = tcg_wait(&acc_full[buf], (accseq >> 1) & 1, abort, status) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      tc_fence_after();
      const long long m = tile * 128 + 32 * warp + lane;
      const bool min_ = m < M;
      const long long r = min_ ? m / o.Pm : 0;
      const int pp = min_ ? (int)(m - r * o.Pm) : 0;
      const int i = pp / o.nJ, j = pp - (pp / o.nJ) * o.nJ;
      const int p = (o.a + o.so * i) * o.Wo + o.b + o.so * j;
      float* orow = out + r * o.stride + p;
      for (int n0 = 0; n0 < Np; n0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(buf * Np + n0), v);
        if (min_) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int n = n0 + e;
            if (n < N) orow[(size_t)n * o.P] = v[e] + (bias ? bias[(size_t)n * o.P + p] : 0.f);
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
  if (warp == 5) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
  }
}

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
  struct ConvW {
    int Np_b = 0, Kp_b = 0, Np_f = 0, Kp_f = 0;
    CUtensorMap mb, mf;              // mb: the s * s phase matrices stacked, Np_b rows each
    int2 *tab_b = nullptr, *tab_f = nullptr;  // gather tables: [s * s][Kp_b], [Kp_f]
  } conv[MAXL + 1];
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

static int encode_map(CUtensorMap* m, void* base, int rows, int kp, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        !p)
      return fail(BCROWN_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)KBLK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(BCROWN_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return BCROWN_OK;
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

// ---------------------------------------------------------------- conv layers on tensor cores
static int pad_to(int x, int m) { return (x + m - 1) / m * m; }

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
static int2 tab_entry(int chan_off, int dy, int dx) {
  return make_int2(chan_off, (int)(((uint32_t)dy & 0xffffu) | ((uint32_t)dx << 16)));
}

bool tcg_supported(const bcrown_net* net) {
  bool conv = false;
  for (int i = 0; i < net->L; ++i) {
    const LayerDev& l = net->ly[i];
    if (l.kind != BCROWN_LAYER_CONV) continue;
    conv = true;
    if (pad_to(l.in_c, 16) > 256 || pad_to(l.out_c, 16) > 256) return false;
    if (kp_bwd(l) > IM2COL_MAX_KP || kp_fwd(l) > IM2COL_MAX_KP) return false;
  }
  if (!conv) return false;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaGetLastError();
  return major == 10 && minor == 3;
}

size_t tcg_col_bytes_per_row(const bcrown_net* net) {
  size_t b = 0;
  for (int i = 0; i < net->L; ++i) {
    const LayerDev& l = net->ly[i];
    if (l.kind != BCROWN_LAYER_CONV) continue;
    const size_t ph = (size_t)((l.in_h + l.stride - 1) / l.stride) * ((l.in_w + l.stride - 1) / l.stride);
    const size_t bwd = ph * kp_bwd(l);
    const size_t fwd = (size_t)l.out_h * l.out_w * kp_fwd(l);
    b = std::max(b, std::max(bwd, fwd) * sizeof(__nv_bfloat16));
  }
  return b;
}

static int tcg_prepare(bcrown_net* net, TcNet* t) {
  if (t->conv_ready) return BCROWN_OK;
  for (int i = 1; i <= net->L; ++i) {
    const LayerDev& l = net->ly[i - 1];
    if (l.kind != BCROWN_LAYER_CONV) continue;
    const int kk = l.k * l.k, s = l.stride, T = taps_per_axis(l);
    std::vector<float> w((size_t)l.out_c * l.in_c * kk);
    if (cudaMemcpy(w.data(), l.W, w.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(BCROWN_ERR_CUDA, "copy of conv weights");
    TcNet::ConvW& c = t->conv[i];
    c.Np_b = pad_to(l.in_c, 16);
    c.Kp_b = kp_bwd(l);
    c.Np_f = pad_to(l.out_c, 16);
    c.Kp_f = kp_fwd(l);
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    std::vector<__nv_bfloat16> wb((size_t)s * s * c.Np_b * c.Kp_b, zero);
    std::vector<__nv_bfloat16> wf((size_t)c.Np_f * c.Kp_f, zero);
    std::vector<int2> tb((size_t)s * s * c.Kp_b, make_int2(-1, 0)), tf((size_t)c.Kp_f, make_int2(-1, 0));
    // forward: K = (ci, ky, kx), source (oy * s - pad + ky, ox * s - pad + kx) of channel ci
    for (int co = 0; co < l.out_c; ++co)
      for (int ci = 0; ci < l.in_c; ++ci)
        for (int q = 0; q < kk; ++q)
          wf[(size_t)co * c.Kp_f + ci * kk + q] = __float2bfloat16_rn(w[((size_t)co * l.in_c + ci) * kk + q]);
    for (int ci = 0; ci < l.in_c; ++ci)
      for (int q = 0; q < kk; ++q) tf[ci * kk + q] = tab_entry(ci * l.in_h * l.in_w, q / l.k, q % l.k);
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
              tb[ph * c.Kp_b + K] = tab_entry(co * l.out_h * l.out_w, -dy, -dx);
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
    t->bufs.push_back(reinterpret_cast<__nv_bfloat16*>(c.tab_b));
    t->bufs.push_back(reinterpret_cast<__nv_bfloat16*>(c.tab_f));
    if (cudaMemcpy(db, wb.data(), wb.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(df, wf.data(), wf.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c.tab_b, tb.data(), tb.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c.tab_f, tf.data(), tf.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(BCROWN_ERR_CUDA, "bf16 conv weights upload");
    BC_CHECK(encode_map(&c.mb, db, s * s * c.Np_b, c.Kp_b, c.Np_b));
    BC_CHECK(encode_map(&c.mf, df, c.Np_f, c.Kp_f, c.Np_f));
  }
  const int smem = 1024 + TCG_NS * (16384 + 256 * 128) + 256;
  BC_CUDA(cudaFuncSetAttribute(k_tcg, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  BC_CUDA(cudaFuncSetAttribute(k_im2col, cudaFuncAttributeMaxDynamicSharedMemorySize, im2col_smem(IM2COL_MAX_KP)));
  t->conv_ready = true;
  return BCROWN_OK;
}

// One im2col + GEMM pass (a phase of a backward layer, or the forward layer).
static int tcg_pass(bcrown_net* net, const Im2colPass& q, const CUtensorMap& mB, const TcgOut& o, const float* src,
                    float* dst, const float* bias, char* col, size_t col_bytes, cudaStream_t s) {
  if (q.M <= 0) return BCROWN_OK;
  if ((size_t)q.M * q.Kp * sizeof(__nv_bfloat16) > col_bytes) return fail(BCROWN_ERR_OOM, "im2col workspace too small");
  __nv_bfloat16* cb = reinterpret_cast<__nv_bfloat16*>(col);
  k_im2col<<<(unsigned)((q.M + IM2COL_ROWS - 1) / IM2COL_ROWS), 256, im2col_smem(q.Kp), s>>>(q, src, cb);
  ++g_launches;
  CUtensorMap mA;
  BC_CHECK(encode_map(&mA, cb, (int)q.M, q.Kp, 128));
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (q.M + 127) / 128;
  const int grid = (int)std::min<long long>(ntiles, 2LL * sms);
  const int smem = 1024 + TCG_NS * (16384 + o.Np * 128) + 256;
  k_tcg<<<grid, TCG_THREADS, smem, s>>>(mA, mB, o, dst, bias, net->status);
  ++g_launches;
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

int tcg_conv(bcrown_net* net, int i, bool fwd, int R, const float* src, float* dst, const float* bias, char* col,
             size_t col_bytes, cudaStream_t s) {
  TcNet* t = tc_of(net);
  BC_CHECK(tcg_prepare(net, t));
  const LayerDev& l = net->ly[i - 1];
  const TcNet::ConvW& c = t->conv[i];
  if (R <= 0) return BCROWN_OK;
  if (fwd) {
    const int P = l.out_h * l.out_w;
    const Im2colPass q{(long long)R * P, P, l.out_w, l.stride, -l.pad, -l.pad, l.in_h, l.in_w, l.d_in, c.Kp_f, c.tab_f};
    const TcgOut o{q.M, l.out_c, c.Np_f, c.Kp_f / 64, 0, P, l.out_w, 0, 0, 1, l.out_w, P, (long long)l.d_out};
    return tcg_pass(net, q, c.mf, o, src, dst, bias, col, col_bytes, s);
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
      const TcgOut o{q.M, l.in_c, c.Np_b, c.Kp_b / 64, ph * c.Np_b, Pm, px.n, a, b, st, l.in_w,
                     l.in_h * l.in_w, (long long)l.d_in};
      BC_CHECK(tcg_pass(net, q, c.mb, o, src, dst, nullptr, col, col_bytes, s));
    }
  return BCROWN_OK;
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
