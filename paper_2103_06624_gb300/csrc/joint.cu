// Joint optimisation of intermediate-layer bounds (Section 3.3, Eq. opt_non_convex) for fully
// connected ReLU networks, FP32 on the CUDA cores.
//
// Per subdomain the bounds l^(T), u^(T) of every hidden layer T >= 2 are recomputed by
// beta-CROWN (Theorem 3.1 with the objective +-z^(T)_j) from the subdomain's bounds of the
// layers below, its split constraints, and free variables alpha', beta' shared by all target
// neurons of one layer (one vector per subdomain, target layer and direction: the section's
// O(L^2 d) variant).  Layer 1 keeps the root's interval bounds; the recomputed bounds are
// intersected with the root's.  The final bound of the K specs then uses these bounds.
//
// Layout (per subdomain b of property p; first[p][T] = root-unstable neurons of p in layers
// 1..T-1, rank = a neuron's rank among them in layer-major order):
//   alpha' block of (b, T, dir) at ap_off[b] + sum_{t=2}^{T-1} 2 first[p][t] + dir first[p][T],
//   first[p][T] entries indexed by rank; ap_off[b] = the sum of the earlier subdomains' sizes
//   (2 sum_{T=2}^{L-1} first[p][T] each).  beta' block of (b, T, dir) at
//   2 (L-2) split_off[b] + (2 (T-2) + dir) split_cnt[b], indexed by the split's list position
//   (entries of splits in layers >= T unused).  dir 0 bounds z^(T) from below, dir 1 bounds
//   -z^(T) (u = -bound).
//
// Gradient of g = sum of all rows' bounds (the adjoint of each pass as in the plain bound:
// dlb/dD_j = A_j zhat_j, dlb/dlambda_j = A_j, along the primal path from x*), plus the chain
// through the recomputed bounds: an unstable neuron's upper chord u/(u-l), -u l/(u-l) moves
// with l, u, which are the bounds of target passes (where they beat the root's) -- so the
// reverse sweep visits the final pass, then target layers L-1 .. 2, each target row weighted
// by dg/dl (dir 0) or -dg/du (dir 1) of its neuron, accumulated by the passes visited before.
//
// Every reduction over rows is done by one thread in a fixed order (no atomics): the results
// are deterministic.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include "simt.cuh"

namespace bcrown {

extern std::atomic<long long> g_launches;

namespace jt {

constexpr int MAXL = 32;   // layers (the hidden offsets travel by value)
struct Hoff {
  long long v[MAXL];
  __host__ __device__ long long operator[](int i) const { return v[i]; }
};

struct View {
  int B, K, H, P, L, d0;
  const int32_t* prop_of;
  const int32_t* split_off;
  const int32_t* split_cnt;
  const int64_t* alpha_off;
  const int32_t* rank;     // [P][H] root rank among the property's unstable neurons, -1 if stable
  const int32_t* U;        // [P]
  const int32_t* first;    // [P][L]: root-unstable neurons of p in layers 1..T-1 (index T)
  const int64_t* jblk;     // [P][L]: offset of target layer T's block pair in the subdomain's block
  const int64_t* ap_off;   // [B + 1]
  const float* l_root;     // [P][H]
  const float* u_root;
  float* lsub;             // [B][H] the subdomain's bounds
  float* usub;
  uint8_t* from_pass;      // [B][H] bit 0: l from its target pass, bit 1: u from its target pass
  const int8_t* ssign;     // [B][H] split sign of the neuron in the subdomain (0: not split)
  const int8_t* sslot;     // [B][H] its position in the split list
  const float* x_lo;       // [P][d0]
  const float* x_hi;
  int* status;
};

struct Pass {
  int target;        // 1: target layer T (rows (b, dir, j)), 0: the specs (rows (b, k))
  int T;             // top layer: the target layer, or L
  int dT;            // target neurons d_T (target), K (specs)
  int b0, Bc;        // the chunk's subdomains
  int rpb;           // rows per subdomain: 2 d_T or K
  const float* va;   // alpha' (target) or alpha (specs)
  int64_t na;
  const float* vb;   // beta' or beta
  int64_t nb;
};

__device__ __forceinline__ void jflag(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Row r of the chunk: subdomain, property, direction (target) or spec, and the bases of the
// row's alpha / beta vectors with the alpha vector's length.
struct RowRef {
  int b, p, dir, j;
  long long ab, bb;
  int alim;
};

__device__ __forceinline__ RowRef row_ref(const View& v, const Pass& q, int r) {
  RowRef o;
  const int bl = r / q.rpb, rr = r - bl * q.rpb;
  o.b = q.b0 + bl;
  o.p = v.prop_of[o.b];
  if (o.p < 0 || o.p >= v.P) {
    jflag(v.status, BCROWN_ERR_ARG);
    o.p = 0;
  }
  const int cnt = v.split_cnt[o.b];
  if (q.target) {
    o.dir = rr / q.dT;
    o.j = rr - o.dir * q.dT;
    const int f = v.first[(size_t)o.p * v.L + q.T];
    o.ab = v.ap_off[o.b] + v.jblk[(size_t)o.p * v.L + q.T] + (long long)o.dir * f;
    o.alim = f;
    o.bb = 2LL * (v.L - 2) * v.split_off[o.b] + (long long)(2 * (q.T - 2) + o.dir) * cnt;
  } else {
    o.dir = 0;
    o.j = rr;
    const int Up = v.U[o.p];
    o.ab = v.alpha_off[o.b] + (long long)rr * Up;
    o.alim = Up;
    o.bb = (long long)v.split_off[o.b] * v.K + (long long)rr * cnt;
  }
  return o;
}

// Relaxation of neuron n (Lemma 2.1 / Eq. definition_D) in a subdomain: D, lambda, and which
// case applies (1: alpha slope, 2: upper chord, 0 otherwise).
struct Rel {
  float D, lam;
  int kind;
  int s, t;
};

__device__ __forceinline__ Rel relax_of(const View& v, int b, int n, float a, float alpha_val) {
  Rel o{0.f, 0.f, 0, 0, -1};
  const size_t bn = (size_t)b * v.H + n;
  o.s = v.ssign[bn];
  o.t = v.sslot[bn];
  if (o.s == -1) {
    o.D = 1.f;
    return o;
  }
  if (o.s == 1) return o;
  const float lo = v.lsub[bn], hi = v.usub[bn];
  if (lo >= 0.f) {
    o.D = 1.f;
  } else if (hi <= 0.f) {
    o.D = 0.f;
  } else if (a >= 0.f) {
    o.D = fminf(fmaxf(alpha_val, 0.f), 1.f);
    o.kind = 1;
  } else {
    const float den = hi - lo;
    o.D = hi / den;
    o.lam = -hi * lo / den;
    o.kind = 2;
  }
  return o;
}

__device__ __forceinline__ float warp_sum(float x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// ---- setup kernels ------------------------------------------------------------------------

// first[p][T] and jblk[p][T] from the root ranks (one thread per property)
__global__ void k_layout(int P, int H, int L, Hoff hoff, const int32_t* rank, int32_t* first,
                         int64_t* jblk) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  long long blk = 0;
  for (int T = 0; T < L; ++T) {
    int f = 0;
    if (T >= 1) {
      // unstable neurons of layers 1..T-1: one past the rank of the last unstable neuron
      // before layer T's first (ranks are layer-major)
      const long long end = hoff[T - 1];
      for (long long n = end - 1; n >= 0; --n)
        if (rank[(size_t)p * H + n] >= 0) {
          f = rank[(size_t)p * H + n] + 1;
          break;
        }
    }
    first[(size_t)p * L + T] = f;
    jblk[(size_t)p * L + T] = blk;
    if (T >= 2) blk += 2LL * f;
  }
}

// ap_off over the subdomains (one thread: a sequential scan); a subdomain's block holds the
// pairs of target layers 2..L-1: jblk[p][L-1] + 2 first[p][L-1] entries (none for L = 2)
__global__ void k_ap_off(int B, int L, const int32_t* prop_of, const int32_t* first, const int64_t* jblk, int P,
                         int64_t* ap_off, int* status) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  long long run = 0;
  for (int b = 0; b < B; ++b) {
    ap_off[b] = run;
    int p = prop_of[b];
    if (p < 0 || p >= P) {
      jflag(status, BCROWN_ERR_ARG);
      p = 0;
    }
    if (L >= 3) run += jblk[(size_t)p * L + (L - 1)] + 2LL * first[(size_t)p * L + (L - 1)];
  }
  ap_off[B] = run;
}

// the per-subdomain state: bounds from the root, no split (k_splitmap then marks the splits)
__global__ void k_init(View v) {
  const int b = blockIdx.y;
  if (b >= v.B) return;
  int p = v.prop_of[b];
  if (p < 0 || p >= v.P) p = 0;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < v.H; n += gridDim.x * blockDim.x) {
    const size_t bn = (size_t)b * v.H + n;
    v.lsub[bn] = v.l_root[(size_t)p * v.H + n];
    v.usub[bn] = v.u_root[(size_t)p * v.H + n];
    v.from_pass[bn] = 0;
    const_cast<int8_t*>(v.ssign)[bn] = 0;
    const_cast<int8_t*>(v.sslot)[bn] = -1;
  }
}

__global__ void k_splitmap(View v, const uint8_t* split_layer, const uint32_t* split_idx, const int8_t* split_sign,
                           Hoff hoff) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= v.B) return;
  const int cnt = v.split_cnt[b], off = v.split_off[b];
  if (cnt < 0 || cnt > BCROWN_MAX_SPLITS) {
    jflag(v.status, BCROWN_ERR_ARG);
    return;
  }
  for (int t = 0; t < cnt; ++t) {
    const int ly = split_layer[off + t];
    const int s = split_sign[off + t];
    if (ly < 1 || ly > v.L - 1 || (s != -1 && s != 1)) {
      jflag(v.status, BCROWN_ERR_ARG);
      continue;
    }
    const long long n = hoff[ly - 1] + (long long)split_idx[off + t];
    if (split_idx[off + t] >= (uint32_t)(hoff[ly] - hoff[ly - 1])) {
      jflag(v.status, BCROWN_ERR_ARG);
      continue;
    }
    const_cast<int8_t*>(v.ssign)[(size_t)b * v.H + n] = (int8_t)s;
    const_cast<int8_t*>(v.sslot)[(size_t)b * v.H + n] = (int8_t)t;
  }
}

// alpha' at the root's adaptive rule (1 where u >= -l, else 0) for every (b, T, dir) block
__global__ void k_init_alpha_p(View v, Hoff hoff, float* alpha_p, int64_t n_alpha_p) {
  const int b = blockIdx.y;
  if (b >= v.B) return;
  int p = v.prop_of[b];
  if (p < 0 || p >= v.P) p = 0;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < v.H; n += gridDim.x * blockDim.x) {
    const int rk = v.rank[(size_t)p * v.H + n];
    if (rk < 0) continue;
    const float lo = v.l_root[(size_t)p * v.H + n], hi = v.u_root[(size_t)p * v.H + n];
    const float val = hi >= -lo ? 1.f : 0.f;
    int layer = 1;
    while (layer < v.L - 1 && n >= hoff[layer]) ++layer;
    for (int T = layer + 1; T <= v.L - 1; ++T) {
      const int f = v.first[(size_t)p * v.L + T];
      for (int dir = 0; dir < 2; ++dir) {
        const long long i = v.ap_off[b] + v.jblk[(size_t)p * v.L + T] + (long long)dir * f + rk;
        if (i >= 0 && i < n_alpha_p) alpha_p[i] = val;
        else jflag(v.status, BCROWN_ERR_ARG);
      }
    }
  }
}

// ---- the bound passes ---------------------------------------------------------------------

// top of a pass: A^(T-1) rows and the constants
__global__ void k_top(View v, Pass q, int dprev, const float* __restrict__ W, const float* __restrict__ bias,
                      float* __restrict__ A, float* __restrict__ cf) {
  const int r = blockIdx.x;
  const RowRef rr = row_ref(v, q, r);
  const float sg = (q.target && rr.dir == 1) ? -1.f : 1.f;
  const float* w = W + (size_t)rr.j * dprev;
  for (int m = threadIdx.x; m < dprev; m += blockDim.x) A[(size_t)r * dprev + m] = sg * w[m];
  if (threadIdx.x == 0) cf[r] = sg * bias[rr.j];
}

// relaxation of layer m for every row (one warp per row):
//   Lambda = A D + beta S;  c += Lambda b^(m) + A lambda
constexpr int RW = 8;   // warps (rows) per block
__global__ void __launch_bounds__(32 * RW) k_relax(View v, Pass q, int R, int d, long long hoff,
                                                   const float* __restrict__ bias, const float* __restrict__ A,
                                                   float* __restrict__ Lam, float* __restrict__ cf) {
  const int r = blockIdx.x * RW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= R) return;
  const RowRef rr = row_ref(v, q, r);
  float acc = 0.f;
  for (int j = lane; j < d; j += 32) {
    const int n = (int)(hoff + j);
    const float a = A[(size_t)r * d + j];
    const int rk = v.rank[(size_t)rr.p * v.H + n];
    float al = 0.f;
    if (rk >= 0 && a >= 0.f) {
      if (rk < rr.alim && rr.ab + rk < q.na) al = q.va[rr.ab + rk];
      else jflag(v.status, BCROWN_ERR_ARG);
    }
    const Rel re = relax_of(v, rr.b, n, a, al);
    if (re.kind == 1 && rk < 0) jflag(v.status, BCROWN_ERR_ARG);   // unstable in a subdomain only: impossible
    float bs = 0.f;
    if (re.s != 0) {
      const long long bi = rr.bb + re.t;
      if (re.t >= 0 && bi < q.nb) bs = fmaxf(q.vb[bi], 0.f) * (float)re.s;
      else jflag(v.status, BCROWN_ERR_ARG);
    }
    const float L = fmaf(a, re.D, bs);
    Lam[(size_t)r * d + j] = L;
    acc = fmaf(L, bias[j], fmaf(a, re.lam, acc));
  }
  acc = warp_sum(acc);
  if (lane == 0) cf[r] += acc;
}

// concretisation over the property's box (Eq. beta_crown_lp, Hoelder for a box)
__global__ void __launch_bounds__(32 * RW) k_conc(View v, Pass q, int R, const float* __restrict__ A0,
                                                  const float* __restrict__ cf, float* __restrict__ lb) {
  const int r = blockIdx.x * RW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= R) return;
  const RowRef rr = row_ref(v, q, r);
  const float* xl = v.x_lo + (size_t)rr.p * v.d0;
  const float* xh = v.x_hi + (size_t)rr.p * v.d0;
  float s = 0.f;
  for (int m = lane; m < v.d0; m += 32) {
    const float a = A0[(size_t)r * v.d0 + m];
    s += fminf(a * xl[m], a * xh[m]);
  }
  s = warp_sum(s);
  if (lane == 0) {
    float out = cf[r] + s;
    if (!isfinite(out)) {
      jflag(v.status, BCROWN_ERR_NONFINITE);
      out = -INFINITY;
    }
    lb[r] = out;
  }
}

// the chunk's recomputed bounds of target layer T, intersected with the root's
__global__ void k_update(View v, Pass q, long long hoffT, const float* __restrict__ tlb) {
  const int bl = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= q.dT) return;
  const int b = q.b0 + bl;
  int p = v.prop_of[b];
  if (p < 0 || p >= v.P) p = 0;
  const long long n = hoffT + j;
  const size_t bn = (size_t)b * v.H + n;
  const float lnew = tlb[(size_t)bl * q.rpb + j];
  const float unew = -tlb[(size_t)bl * q.rpb + q.dT + j];
  const float lr = v.l_root[(size_t)p * v.H + n], ur = v.u_root[(size_t)p * v.H + n];
  uint8_t f = 0;
  float lo = lr, hi = ur;
  if (lnew > lr) {
    lo = lnew;
    f |= 1;
  }
  if (unew < ur) {
    hi = unew;
    f |= 2;
  }
  v.lsub[bn] = lo;
  v.usub[bn] = hi;
  v.from_pass[bn] = f;
}

// x*: the box corner minimising A^(0) x
__global__ void k_xstar(View v, Pass q, int R, const float* __restrict__ A0, float* __restrict__ h0) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)R * v.d0) return;
  const int r = (int)(id / v.d0), m = (int)(id - (long long)r * v.d0);
  const RowRef rr = row_ref(v, q, r);
  h0[id] = A0[id] >= 0.f ? v.x_lo[(size_t)rr.p * v.d0 + m] : v.x_hi[(size_t)rr.p * v.d0 + m];
}

// Adjoint of layer m along the primal path (zhat = Z, bias added by the GEMM): h = D zhat +
// lambda for every row, and the gradients.  One thread per (subdomain, neuron), looping over
// the subdomain's rows in order.  Spec rows write dalpha / dbeta per row; target rows (weighted
// by dg/dl or -dg/du of their neuron) sum into the subdomain's dalpha' / dbeta'.  Both add
// their chord terms to dg/dl, dg/du of the neuron.
__global__ void __launch_bounds__(256) k_adj(View v, Pass q, int d, long long hoff, long long hoffT,
                                             const float* __restrict__ Z, const float* __restrict__ A,
                                             float* __restrict__ Hout, float* __restrict__ ga, float* __restrict__ gb,
                                             float* __restrict__ gl, float* __restrict__ gu) {
  const int bl = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  const int b = q.b0 + bl;
  int p = v.prop_of[b];
  if (p < 0 || p >= v.P) p = 0;
  const int n = (int)(hoff + j);
  const size_t bn = (size_t)b * v.H + n;
  const int rk = v.rank[(size_t)p * v.H + n];
  float sa[2] = {0.f, 0.f}, sb[2] = {0.f, 0.f}, sl = 0.f, su = 0.f;
  const float lo = v.lsub[bn], hi = v.usub[bn];
  for (int rr_ = 0; rr_ < q.rpb; ++rr_) {
    const int r = bl * q.rpb + rr_;
    const RowRef rr = row_ref(v, q, r);
    float w = 1.f;
    if (q.target) {
      const size_t bt = (size_t)b * v.H + hoffT + rr.j;
      const uint8_t f = v.from_pass[bt];
      w = rr.dir == 0 ? ((f & 1) ? gl[bt] : 0.f) : ((f & 2) ? -gu[bt] : 0.f);
    }
    const float z = Z[(size_t)r * d + j];
    const float a = A[(size_t)r * d + j];
    float al = 0.f;
    if (rk >= 0 && a >= 0.f && rk < rr.alim && rr.ab + rk < q.na) al = q.va[rr.ab + rk];
    const Rel re = relax_of(v, b, n, a, al);
    Hout[(size_t)r * d + j] = fmaf(re.D, z, re.lam);
    const float gal = re.kind == 1 ? a * z : 0.f;
    if (!q.target && rk >= 0) {
      const long long ai = rr.ab + rk;
      if (rk < rr.alim && ai < q.na) ga[ai] = gal;
      else jflag(v.status, BCROWN_ERR_ARG);
    }
    if (re.s != 0) {
      if (q.target) {
        sb[rr.dir] += w * (float)re.s * z;
      } else {
        const long long bi = rr.bb + re.t;
        if (re.t >= 0 && bi < q.nb) gb[bi] = (float)re.s * z;
        else jflag(v.status, BCROWN_ERR_ARG);
      }
    }
    if (q.target) sa[rr.dir] += w * gal;
    if (re.kind == 2) {
      // d/dl and d/du of a (zhat s + t), s = u / (u - l), t = -u l / (u - l)
      const float den = hi - lo, i2 = 1.f / (den * den);
      const float dsdl = hi * i2, dsdu = -lo * i2, dtdl = -hi * hi * i2, dtdu = lo * lo * i2;
      sl += w * a * fmaf(z, dsdl, dtdl);
      su += w * a * fmaf(z, dsdu, dtdu);
    }
  }
  gl[bn] += sl;
  gu[bn] += su;
  if (q.target) {
    if (rk >= 0) {
      const int f = v.first[(size_t)p * v.L + q.T];
      for (int dir = 0; dir < 2; ++dir) {
        const long long ai = v.ap_off[b] + v.jblk[(size_t)p * v.L + q.T] + (long long)dir * f + rk;
        if (rk < f && ai < q.na) ga[ai] = sa[dir];
        else jflag(v.status, BCROWN_ERR_ARG);
      }
    }
    const int s = v.ssign[bn], t = v.sslot[bn];
    if (s != 0) {
      const int cnt = v.split_cnt[b];
      for (int dir = 0; dir < 2; ++dir) {
        const long long bi = 2LL * (v.L - 2) * v.split_off[b] + (long long)(2 * (q.T - 2) + dir) * cnt + t;
        if (t >= 0 && bi < q.nb) gb[bi] = sb[dir];
        else jflag(v.status, BCROWN_ERR_ARG);
      }
    }
  }
}

// ---- optimiser ------------------------------------------------------------------------------

// projected Adam step taken uphill (Appendix C.1), t counted from 0 via the bias corrections
__global__ void k_adam(long long n, float* __restrict__ th, float* __restrict__ m, float* __restrict__ vv,
                       const float* __restrict__ g, float lr, float b1, float b2, float eps, float bc1, float bc2,
                       float lo, float hi) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * vv[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  vv[i] = vi;
  const float step = (mi / bc1) / (sqrtf(vi / bc2) + eps);
  th[i] = fminf(fmaxf(fmaf(lr, step, th[i]), lo), hi);
}

// per subdomain: the sum of its spec bounds against the best so far
__global__ void k_score(int B, int K, const float* __restrict__ lb, float* __restrict__ best,
                        uint8_t* __restrict__ improved) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float s = 0.f;
  for (int k = 0; k < K; ++k) s += lb[(size_t)b * K + k];
  const bool up = s > best[b];
  improved[b] = up ? 1 : 0;
  if (up) best[b] = s;
}

__global__ void k_keep(long long n, const int32_t* __restrict__ owner, const uint8_t* __restrict__ improved,
                       const float* __restrict__ th, float* __restrict__ kept) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (improved[owner[i]]) kept[i] = th[i];
}

// owning subdomain of every entry of alpha, beta, alpha', beta'
__global__ void k_owner(View v, int32_t* oa, int64_t na, int32_t* ob, int64_t nb, int32_t* oap, int64_t nap,
                        int32_t* obp, int64_t nbp) {
  const int b = blockIdx.x;
  if (b >= v.B) return;
  int p = v.prop_of[b];
  if (p < 0 || p >= v.P) p = 0;
  const long long a0 = v.alpha_off[b], a1 = a0 + (long long)v.K * v.U[p];
  for (long long i = a0 + threadIdx.x; i < a1 && i < na; i += blockDim.x) oa[i] = b;
  const long long b0 = (long long)v.split_off[b] * v.K, b1 = b0 + (long long)v.K * v.split_cnt[b];
  for (long long i = b0 + threadIdx.x; i < b1 && i < nb; i += blockDim.x) ob[i] = b;
  for (long long i = v.ap_off[b] + threadIdx.x; i < v.ap_off[b + 1] && i < nap; i += blockDim.x) oap[i] = b;
  const long long c0 = 2LL * (v.L - 2) * v.split_off[b], c1 = c0 + 2LL * (v.L - 2) * v.split_cnt[b];
  for (long long i = c0 + threadIdx.x; i < c1 && i < nbp; i += blockDim.x) obp[i] = b;
}

// ---- host side ------------------------------------------------------------------------------

struct Work {
  View v;
  Hoff hoff;
  // chunk buffers
  int Bc, rows_max;
  std::vector<float*> A;     // [L]: A^(m) [rows][d_m]
  float *Lam, *Z, *Hb, *cf, *tlb;
  float *gl, *gu;
};

static int fc_only(const bcrown_net* net) {
  for (int i = 0; i < net->L; ++i)
    if (net->ly[i].kind != BCROWN_LAYER_FC) return 0;
  return 1;
}

static int rows_per_b(const bcrown_net* net) {
  int m = net->K;
  for (int T = 2; T <= net->L - 1; ++T) m = std::max(m, 2 * net->d[T]);
  return m;
}

// Carves the workspace and computes the layout and per-subdomain state.
static int setup(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* bt, bool grad, Work& w,
                 cudaStream_t s) {
  const int P = dom->n_props, H = net->H, L = net->L, B = bt->B;
  const int rpb = rows_per_b(net);
  size_t per_row = 0;
  for (int m = 0; m < L; ++m) per_row += (size_t)net->d[m];
  per_row += (size_t)net->max_hidden + 2 * (size_t)net->max_width + 2;
  const size_t budget = size_t(4) << 30;
  w.Bc = (int)std::max<long long>(1, std::min<long long>(B, (long long)(budget / ((size_t)rpb * per_row * 4))));
  w.rows_max = w.Bc * rpb;
  const size_t PH = (size_t)P * H, BH = (size_t)B * H;
  size_t bytes = 0;
  auto add = [&](size_t n) { bytes += align_up(n); };
  add(PH), add(PH * 4), add(PH * 4), add(PH * 4), add((size_t)P * 4);           // tables
  add((size_t)P * L * 4), add((size_t)P * L * 8), add((size_t)(B + 1) * 8);      // layout
  add(BH * 4), add(BH * 4), add(BH), add(BH), add(BH);                             // state
  if (grad) add(BH * 4), add(BH * 4);
  for (int m = 0; m < L; ++m) add((size_t)w.rows_max * net->d[m] * 4);
  add((size_t)w.rows_max * net->max_hidden * 4);
  add((size_t)w.rows_max * net->max_width * 4), add((size_t)w.rows_max * net->max_width * 4);
  add((size_t)w.rows_max * 4), add((size_t)w.rows_max * 4);
  int st = 0;
  void* base = ws_get(net, bytes, &st);
  if (!base) return st;
  Arena ar{(char*)base};
  uint8_t* code = ar.take<uint8_t>(PH);
  int32_t* rank = ar.take<int32_t>(PH);
  float* slope = ar.take<float>(PH);
  float* icpt = ar.take<float>(PH);
  int32_t* U = ar.take<int32_t>(P);
  Tables tb;
  launch_tables(P, H, dom->l, dom->u, tb, code, rank, slope, icpt, U, s);
  View& v = w.v;
  v.B = B, v.K = net->K, v.H = H, v.P = P, v.L = L, v.d0 = net->d[0];
  v.prop_of = bt->prop_of, v.split_off = bt->split_off, v.split_cnt = bt->split_cnt, v.alpha_off = bt->alpha_off;
  v.rank = rank, v.U = U;
  int32_t* first = ar.take<int32_t>((size_t)P * L);
  int64_t* jblk = ar.take<int64_t>((size_t)P * L);
  int64_t* ap_off = ar.take<int64_t>((size_t)B + 1);
  v.first = first, v.jblk = jblk, v.ap_off = ap_off;
  v.l_root = dom->l, v.u_root = dom->u;
  v.lsub = ar.take<float>(BH);
  v.usub = ar.take<float>(BH);
  v.from_pass = ar.take<uint8_t>(BH);
  int8_t* ssign = ar.take<int8_t>(BH);
  int8_t* sslot = ar.take<int8_t>(BH);
  v.ssign = ssign, v.sslot = sslot;
  v.x_lo = dom->x_lo, v.x_hi = dom->x_hi;
  v.status = net->status;
  for (int i = 0; i < MAXL; ++i) w.hoff.v[i] = i < L ? net->hoff[i] : 0;
  if (grad) {
    w.gl = ar.take<float>(BH);
    w.gu = ar.take<float>(BH);
  } else {
    w.gl = w.gu = nullptr;
  }
  w.A.assign(L, nullptr);
  for (int m = 0; m < L; ++m) w.A[m] = ar.take<float>((size_t)w.rows_max * net->d[m]);
  w.Lam = ar.take<float>((size_t)w.rows_max * net->max_hidden);
  w.Z = ar.take<float>((size_t)w.rows_max * net->max_width);
  w.Hb = ar.take<float>((size_t)w.rows_max * net->max_width);
  w.cf = ar.take<float>(w.rows_max);
  w.tlb = ar.take<float>(w.rows_max);
  if (ar.off > net->ws.size) return fail(BCROWN_ERR_OOM, "joint: workspace plan overflow");
  k_layout<<<(P + 127) / 128, 128, 0, s>>>(P, H, L, w.hoff, rank, first, jblk);
  k_ap_off<<<1, 1, 0, s>>>(B, L, bt->prop_of, first, jblk, P, ap_off, net->status);
  k_init<<<dim3((H + 255) / 256, B), 256, 0, s>>>(v);
  k_splitmap<<<(B + 127) / 128, 128, 0, s>>>(v, bt->split_layer, bt->split_idx, bt->split_sign, w.hoff);
  g_launches += 4;
  if (grad) {
    BC_CUDA(cudaMemsetAsync(w.gl, 0, BH * 4, s));
    BC_CUDA(cudaMemsetAsync(w.gu, 0, BH * 4, s));
  }
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

// The backward recursion of one pass over the chunk (top, relaxation and contraction down to
// the input, concretisation into out): A^(m) of every layer stays in w.A for the adjoint.
static int backward(bcrown_net* net, Work& w, const Pass& q, float* out, cudaStream_t s) {
  const int R = q.Bc * q.rpb;
  const int T = q.T;
  const LayerDev& top = net->ly[T - 1];
  if (q.target)
    k_top<<<R, 128, 0, s>>>(w.v, q, net->d[T - 1], top.W, top.b, w.A[T - 1], w.cf);
  else
    k_top<<<R, 128, 0, s>>>(w.v, q, net->d[T - 1], net->Wbar, net->bbar, w.A[T - 1], w.cf);
  ++g_launches;
  for (int m = T - 1; m >= 1; --m) {
    const LayerDev& l = net->ly[m - 1];
    k_relax<<<(R + RW - 1) / RW, 32 * RW, 0, s>>>(w.v, q, R, net->d[m], net->hoff[m - 1], l.b, w.A[m], w.Lam,
                                                  w.cf);
    ++g_launches;
    // A^(m-1) = Lambda^(m) W^(m)
    launch_sgemm(R, l.d_in, l.d_out, w.Lam, l.d_out, l.W, l.d_in, w.A[m - 1], l.d_in, nullptr, s);
  }
  k_conc<<<(R + RW - 1) / RW, 32 * RW, 0, s>>>(w.v, q, R, w.A[0], w.cf, out);
  ++g_launches;
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

// The adjoint of the pass just run by backward(): h^(0) = x*, then for m = 1..T-1
// zhat = W^(m) h + b^(m) and the layer's gradients.
static int adjoint(bcrown_net* net, Work& w, const Pass& q, float* ga, float* gb, cudaStream_t s) {
  const int R = q.Bc * q.rpb;
  const int d0 = net->d[0];
  k_xstar<<<grid1d((long long)R * d0, 256), 256, 0, s>>>(w.v, q, R, w.A[0], w.Hb);
  ++g_launches;
  const long long hoffT = q.target ? net->hoff[q.T - 1] : 0;
  for (int m = 1; m <= q.T - 1; ++m) {
    const LayerDev& l = net->ly[m - 1];
    launch_sgemm(R, l.d_out, l.d_in, w.Hb, l.d_in, l.Wt, l.d_out, w.Z, l.d_out, l.b, s);
    k_adj<<<dim3((l.d_out + 255) / 256, q.Bc), 256, 0, s>>>(w.v, q, l.d_out, net->hoff[m - 1], hoffT, w.Z,
                                                            w.A[m], w.Hb, ga, gb, w.gl, w.gu);
    ++g_launches;
  }
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

static Pass make_pass(const bcrown_net* net, bool target, int T, int b0, int Bc, const float* va, int64_t na,
                      const float* vb, int64_t nb) {
  Pass q;
  q.target = target ? 1 : 0;
  q.T = T;
  q.dT = target ? net->d[T] : net->K;
  q.rpb = target ? 2 * net->d[T] : net->K;
  q.b0 = b0;
  q.Bc = Bc;
  q.va = va;
  q.na = na;
  q.vb = vb;
  q.nb = nb;
  return q;
}

// The joint bound (and with grad, its gradient) of every row of the batch.
static int run(bcrown_net* net, Work& w, const bcrown_batch* bt, const float* alpha, const float* beta,
               const float* alpha_p, int64_t n_alpha_p, const float* beta_p, int64_t n_beta_p, float* lb, bool grad,
               float* dalpha, float* dbeta, float* dalpha_p, float* dbeta_p, cudaStream_t s) {
  const int L = net->L, B = bt->B, K = net->K;
  if (grad) {
    if (bt->n_alpha) BC_CUDA(cudaMemsetAsync(dalpha, 0, bt->n_alpha * 4, s));
    if (bt->n_beta) BC_CUDA(cudaMemsetAsync(dbeta, 0, bt->n_beta * 4, s));
    if (n_alpha_p) BC_CUDA(cudaMemsetAsync(dalpha_p, 0, n_alpha_p * 4, s));
    if (n_beta_p) BC_CUDA(cudaMemsetAsync(dbeta_p, 0, n_beta_p * 4, s));
  }
  for (int b0 = 0; b0 < B; b0 += w.Bc) {
    const int Bc = std::min(w.Bc, B - b0);
    for (int T = 2; T <= L - 1; ++T) {
      Pass q = make_pass(net, true, T, b0, Bc, alpha_p, n_alpha_p, beta_p, n_beta_p);
      BC_CHECK(backward(net, w, q, w.tlb, s));
      k_update<<<dim3((net->d[T] + 127) / 128, Bc), 128, 0, s>>>(w.v, q, net->hoff[T - 1], w.tlb);
      ++g_launches;
    }
    Pass f = make_pass(net, false, L, b0, Bc, alpha, bt->n_alpha, beta, bt->n_beta);
    BC_CHECK(backward(net, w, f, lb + (size_t)b0 * K, s));
    if (!grad) continue;
    BC_CHECK(adjoint(net, w, f, dalpha, dbeta, s));
    for (int T = L - 1; T >= 2; --T) {
      Pass q = make_pass(net, true, T, b0, Bc, alpha_p, n_alpha_p, beta_p, n_beta_p);
      BC_CHECK(backward(net, w, q, w.tlb, s));   // recomputed: A^(m) of this pass for its adjoint
      BC_CHECK(adjoint(net, w, q, dalpha_p, dbeta_p, s));
    }
  }
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

static int check(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* bt) {
  if (!net || !dom || !bt) return fail(BCROWN_ERR_ARG, "joint: null argument");
  if (dom->n_props < 1 || !dom->x_lo || !dom->x_hi || !dom->l || !dom->u)
    return fail(BCROWN_ERR_ARG, "joint: domain arrays missing");
  if (bt->B < 0 || (bt->B > 0 && (!bt->prop_of || !bt->split_off || !bt->split_cnt || !bt->alpha_off)))
    return fail(BCROWN_ERR_ARG, "joint: batch arrays missing");
  if (!fc_only(net)) return fail(BCROWN_ERR_UNIMPLEMENTED, "joint: fully connected networks only");
  if (net->L < 2 || net->L > MAXL) return fail(BCROWN_ERR_ARG, "joint: 2 to 32 layers");
  return BCROWN_OK;
}

static int copy_bounds(Work& w, const bcrown_batch* bt, int H, float* l_out, float* u_out, cudaStream_t s) {
  const size_t n = (size_t)bt->B * H * 4;
  if (l_out) BC_CUDA(cudaMemcpyAsync(l_out, w.v.lsub, n, cudaMemcpyDeviceToDevice, s));
  if (u_out) BC_CUDA(cudaMemcpyAsync(u_out, w.v.usub, n, cudaMemcpyDeviceToDevice, s));
  return BCROWN_OK;
}

}  // namespace jt
}  // namespace bcrown

using namespace bcrown;
using namespace bcrown::jt;

extern "C" int bcrown_joint_sizes(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                                  int64_t* n_alpha_p, int64_t* n_beta_p, void* stream) {
  BC_CHECK(jt::check(net, dom, batch));
  if (!n_alpha_p || !n_beta_p) return fail(BCROWN_ERR_ARG, "joint_sizes: null output");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  if (batch->B == 0) {
    *n_alpha_p = *n_beta_p = 0;
    return BCROWN_OK;
  }
  Work w;
  BC_CHECK(setup(net, dom, batch, false, w, s));
  int64_t na = 0;
  int32_t off = 0, cnt = 0;
  BC_CUDA(cudaMemcpyAsync(&na, w.v.ap_off + batch->B, 8, cudaMemcpyDeviceToHost, s));
  BC_CUDA(cudaMemcpyAsync(&off, batch->split_off + batch->B - 1, 4, cudaMemcpyDeviceToHost, s));
  BC_CUDA(cudaMemcpyAsync(&cnt, batch->split_cnt + batch->B - 1, 4, cudaMemcpyDeviceToHost, s));
  BC_CUDA(cudaStreamSynchronize(s));
  *n_alpha_p = na;
  *n_beta_p = 2LL * (net->L - 2) * ((int64_t)off + cnt);
  return BCROWN_OK;
}

extern "C" int bcrown_joint_init_alpha(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                                       float* alpha_p, int64_t n_alpha_p, void* stream) {
  BC_CHECK(jt::check(net, dom, batch));
  if (batch->B == 0) return BCROWN_OK;
  if (!alpha_p && n_alpha_p) return fail(BCROWN_ERR_ARG, "joint_init_alpha: null alpha'");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  Work w;
  BC_CHECK(setup(net, dom, batch, false, w, s));
  if (n_alpha_p) BC_CUDA(cudaMemsetAsync(alpha_p, 0, n_alpha_p * 4, s));
  k_init_alpha_p<<<dim3((net->H + 255) / 256, batch->B), 256, 0, s>>>(w.v, w.hoff, alpha_p, n_alpha_p);
  ++g_launches;
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

extern "C" int bcrown_bound_joint(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                                  const float* alpha, const float* beta, const float* alpha_p, int64_t n_alpha_p,
                                  const float* beta_p, int64_t n_beta_p, float* lb, float* l_out, float* u_out,
                                  void* stream) {
  BC_CHECK(jt::check(net, dom, batch));
  if (batch->B == 0) return BCROWN_OK;
  if (!lb) return fail(BCROWN_ERR_ARG, "bound_joint: null lb");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  Work w;
  BC_CHECK(setup(net, dom, batch, false, w, s));
  BC_CHECK(run(net, w, batch, alpha, beta, alpha_p, n_alpha_p, beta_p, n_beta_p, lb, false, nullptr, nullptr,
               nullptr, nullptr, s));
  return copy_bounds(w, batch, net->H, l_out, u_out, s);
}

extern "C" int bcrown_bound_joint_grad(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                                       const float* alpha, const float* beta, const float* alpha_p,
                                       int64_t n_alpha_p, const float* beta_p, int64_t n_beta_p, float* lb,
                                       float* dalpha, float* dbeta, float* dalpha_p, float* dbeta_p, void* stream) {
  BC_CHECK(jt::check(net, dom, batch));
  if (batch->B == 0) return BCROWN_OK;
  if (!lb || (batch->n_alpha && !dalpha) || (batch->n_beta && !dbeta) || (n_alpha_p && !dalpha_p) ||
      (n_beta_p && !dbeta_p))
    return fail(BCROWN_ERR_ARG, "bound_joint_grad: null output");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  Work w;
  BC_CHECK(setup(net, dom, batch, true, w, s));
  return run(net, w, batch, alpha, beta, alpha_p, n_alpha_p, beta_p, n_beta_p, lb, true, dalpha, dbeta, dalpha_p,
             dbeta_p, s);
}

extern "C" int bcrown_optimize_joint(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                                     const bcrown_opt_cfg* cfg, float* alpha, float* beta, float* alpha_p,
                                     int64_t n_alpha_p, float* beta_p, int64_t n_beta_p, float* lb_out, float* l_out,
                                     float* u_out, void* stream) {
  BC_CHECK(jt::check(net, dom, batch));
  if (!cfg || cfg->iters < 0) return fail(BCROWN_ERR_ARG, "optimize_joint: null cfg or negative iterations");
  if (cfg->precision != BCROWN_FP32 || cfg->certify)
    return fail(BCROWN_ERR_UNIMPLEMENTED, "optimize_joint: FP32 iterations and an FP32 final pass only");
  if (batch->B == 0) return BCROWN_OK;
  if (!lb_out) return fail(BCROWN_ERR_ARG, "optimize_joint: null lb");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  // optimiser buffers first (a separate allocation: the workspace below is the library's)
  const int64_t n[4] = {batch->n_alpha, batch->n_beta, n_alpha_p, n_beta_p};
  float* theta[4] = {alpha, beta, alpha_p, beta_p};   // in: theta_0; out: the kept iterate
  const int B = batch->B, K = net->K, R = B * K;
  size_t bytes = 0;
  for (int q = 0; q < 4; ++q) bytes += align_up((size_t)std::max<int64_t>(n[q], 1) * 4) * 4;  // cur, m, v, g
  for (int q = 0; q < 4; ++q) bytes += align_up((size_t)std::max<int64_t>(n[q], 1) * 4);      // owners
  bytes += align_up((size_t)B * 4) + align_up((size_t)B) + align_up((size_t)R * 4);
  char* opt = nullptr;
  BC_CUDA(cudaMalloc(reinterpret_cast<void**>(&opt), bytes));
  Arena ar{opt};
  float *cur[4], *mm[4], *vv[4], *gg[4];
  int32_t* own[4];
  for (int q = 0; q < 4; ++q) {
    cur[q] = ar.take<float>(std::max<int64_t>(n[q], 1));
    mm[q] = ar.take<float>(std::max<int64_t>(n[q], 1));
    vv[q] = ar.take<float>(std::max<int64_t>(n[q], 1));
    gg[q] = ar.take<float>(std::max<int64_t>(n[q], 1));
  }
  for (int q = 0; q < 4; ++q) own[q] = ar.take<int32_t>(std::max<int64_t>(n[q], 1));
  float* best = ar.take<float>(B);
  uint8_t* improved = ar.take<uint8_t>(B);
  float* lbt = ar.take<float>(R);
  int rc = BCROWN_OK;
  {
    Work w;
    rc = setup(net, dom, batch, true, w, s);
    if (rc == BCROWN_OK) {
      for (int q = 0; q < 4; ++q)
        if (n[q]) {
          cudaMemcpyAsync(cur[q], theta[q], n[q] * 4, cudaMemcpyDeviceToDevice, s);
          cudaMemsetAsync(mm[q], 0, n[q] * 4, s);
          cudaMemsetAsync(vv[q], 0, n[q] * 4, s);
        }
      launch_fill(best, B, -INFINITY, s);
      // entries no subdomain owns (gaps the caller's alpha_off may leave) read subdomain 0
      for (int q = 0; q < 4; ++q) cudaMemsetAsync(own[q], 0, std::max<int64_t>(n[q], 1) * 4, s);
      k_owner<<<B, 256, 0, s>>>(w.v, own[0], n[0], own[1], n[1], own[2], n[2], own[3], n[3]);
      ++g_launches;
      const bool frozen[4] = {(cfg->freeze & BCROWN_FREEZE_ALPHA) != 0, (cfg->freeze & BCROWN_FREEZE_BETA) != 0,
                              (cfg->freeze & BCROWN_FREEZE_ALPHA) != 0, (cfg->freeze & BCROWN_FREEZE_BETA) != 0};
      const float lr0[4] = {cfg->lr_alpha, cfg->lr_beta, cfg->lr_alpha, cfg->lr_beta};
      const float hi[4] = {1.f, INFINITY, 1.f, INFINITY};
      for (int it = 0; it < cfg->iters && rc == BCROWN_OK; ++it) {
        // gradient at theta_t (the workspace state is rebuilt by the pass itself)
        rc = setup(net, dom, batch, true, w, s);
        if (rc != BCROWN_OK) break;
        rc = run(net, w, batch, cur[0], cur[1], cur[2], n[2], cur[3], n[3], lbt, true, gg[0], gg[1], gg[2], gg[3],
                 s);
        if (rc != BCROWN_OK) break;
        k_score<<<(B + 127) / 128, 128, 0, s>>>(B, K, lbt, best, improved);
        ++g_launches;
        for (int q = 0; q < 4; ++q)
          if (n[q]) {
            k_keep<<<grid1d(n[q], 256), 256, 0, s>>>(n[q], own[q], improved, cur[q], theta[q]);
            ++g_launches;
          }
        const float fac = std::pow(cfg->decay, (float)it);
        const float bc1 = 1.f - std::pow(cfg->adam_beta1, (float)(it + 1));
        const float bc2 = 1.f - std::pow(cfg->adam_beta2, (float)(it + 1));
        for (int q = 0; q < 4; ++q)
          if (n[q] && !frozen[q]) {
            k_adam<<<grid1d(n[q], 256), 256, 0, s>>>(n[q], cur[q], mm[q], vv[q], gg[q], lr0[q] * fac,
                                                     cfg->adam_beta1, cfg->adam_beta2, cfg->adam_eps, bc1, bc2, 0.f,
                                                     hi[q]);
            ++g_launches;
          }
      }
      if (rc == BCROWN_OK) {
        // the bound at the kept iterate
        rc = setup(net, dom, batch, false, w, s);
        if (rc == BCROWN_OK)
          rc = run(net, w, batch, alpha, beta, alpha_p, n[2], beta_p, n[3], lb_out, false, nullptr, nullptr,
                   nullptr, nullptr, s);
        if (rc == BCROWN_OK) rc = copy_bounds(w, batch, net->H, l_out, u_out, s);
      }
    }
  }
  cudaStreamSynchronize(s);
  cudaFree(opt);
  if (rc == BCROWN_OK) BC_CUDA(cudaGetLastError());
  return rc;
}
