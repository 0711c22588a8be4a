// FP32 convolutions of the SIMT path (the plain FP32 form and the certifying pass) as implicit
// GEMMs: rows M = (subdomain row, output position), columns N = output channels, and K = (input
// channel, tap), the operand gathered from the channel-major FP32 activations while it is staged
// in shared memory.  The transposed convolution of the backward pass (Eq. definition_A) is split
// into its stride phases, as on the tensor-core path: input positions p = (a + s i, b + s j)
// receive only the taps ky = ky0(a) + s dy from source rows i + off(a) - dy, so no work is spent
// on the zeros of the stride and no thread diverges on a divisibility test.
//
// Each output is one sequential FMA chain over its K terms (K tile by K tile, in K order), at
// most the layer's terms_bwd / terms_fwd of them, so the certifying pass's a priori bound
// gamma_n sum |x_i y_i| (Higham, Accuracy and Stability of Numerical Algorithms, 3.1) holds.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "simt.cuh"

namespace bcrown {

extern std::atomic<long long> g_launches;

bool sconv_supported(const bcrown_net* net, int i);

namespace {

struct SconvPass {
  long long M;     // rows: R * Pm
  int Pm, nJ;      // positions per row in this pass, and the pass grid's width
  int N, K;        // output channels; terms per output
  int Hs, Ws;      // source map (one channel)
  long long HWs;
  int ms, cy, cx;  // base source position of (i, j): (i ms + cy, j ms + cx)
  int oa, ob, os, Wo;
  long long HWo;   // output position (oa + os i) Wo + ob + os j, channel stride HWo
  const int4* tab; // [K]: {source offset c HWs + dy Ws + dx, dy, dx, 0}
  const float* B;  // [K][N] weights
};

constexpr int SC_BM = 128, SC_BK = 16, SC_THREADS = 256;

template <int BN>
__global__ void __launch_bounds__(SC_THREADS) k_sconv(SconvPass q, const float* __restrict__ src, long long sstride,
                                                      float* __restrict__ out, long long ostride,
                                                      const float* __restrict__ bias) {
  constexpr int TN = BN / 16;          // output channels per thread
  extern __shared__ __align__(16) uint8_t sc_raw[];
  float(*As)[SC_BK][SC_BM + 4] = reinterpret_cast<float(*)[SC_BK][SC_BM + 4]>(sc_raw);
  float(*Bs)[SC_BK][BN + 4] = reinterpret_cast<float(*)[SC_BK][BN + 4]>(sc_raw + 2 * SC_BK * (SC_BM + 4) * 4);
  int4* stab = reinterpret_cast<int4*>(sc_raw + 2 * SC_BK * (SC_BM + 4) * 4 + 2 * SC_BK * (BN + 4) * 4);
  const int tid = threadIdx.x;
  const int tm = tid & 15, tn = tid >> 4;
  const long long m0 = (long long)blockIdx.x * SC_BM;
  const int n0 = blockIdx.y * BN;
  for (int k = tid; k < q.K; k += SC_THREADS) stab[k] = q.tab[k];
  // the row this thread gathers (fixed across K tiles) and its base source position
  const long long mg = m0 + (tid & 127);
  const bool mv = mg < q.M;
  const long long r = mv ? mg / q.Pm : 0;
  const int pp = mv ? (int)(mg - r * q.Pm) : 0;
  const int pi = pp / q.nJ, pj = pp - (pp / q.nJ) * q.nJ;
  const int y0 = mv ? pi * q.ms + q.cy : -32768, x0 = pj * q.ms + q.cx;
  const float* srow = src + r * sstride + (mv ? (long long)y0 * q.Ws + x0 : 0);
  float acc[8][TN];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  float ra[8], rb[TN];
  __syncthreads();
  auto load = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int kk = (tid >> 7) + 2 * u;
      const int k = k0 + kk;
      float v = 0.f;
      if (k < q.K) {
        const int4 t = stab[k];
        if ((unsigned)(y0 + t.y) < (unsigned)q.Hs && (unsigned)(x0 + t.z) < (unsigned)q.Ws) v = srow[t.x];
      }
      ra[u] = v;
    }
#pragma unroll
    for (int u = 0; u < TN; ++u) {
      const int e = tid + SC_THREADS * u;
      const int kk = e / BN, n = e - (e / BN) * BN;
      const int k = k0 + kk;
      rb[u] = (k < q.K && n0 + n < q.N) ? q.B[(size_t)k * q.N + n0 + n] : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 8; ++u) As[buf][(tid >> 7) + 2 * u][tid & 127] = ra[u];
#pragma unroll
    for (int u = 0; u < TN; ++u) {
      const int e = tid + SC_THREADS * u;
      Bs[buf][e / BN][e - (e / BN) * BN] = rb[u];
    }
  };
  const int nk = (q.K + SC_BK - 1) / SC_BK;
  load(0);
  store(0);
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int buf = t & 1;
    if (t + 1 < nk) load((t + 1) * SC_BK);
#pragma unroll
    for (int kk = 0; kk < SC_BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * tm]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + 4 * tm]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      float bv[TN];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[buf][kk][tn * TN + j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (t + 1 < nk) store(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long m = m0 + (i < 4 ? 4 * tm + i : 64 + 4 * tm + i - 4);
    if (m >= q.M) continue;
    const long long rr = m / q.Pm;
    const int p2 = (int)(m - rr * q.Pm);
    const int ii = p2 / q.nJ, jj = p2 - (p2 / q.nJ) * q.nJ;
    const long long p = (long long)(q.oa + q.os * ii) * q.Wo + q.ob + q.os * jj;
    float* orow = out + rr * ostride + p;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tn * TN + j;
      if (n < q.N) orow[(size_t)n * q.HWo] = acc[i][j] + (bias ? bias[(size_t)n * q.HWo + p] : 0.f);
    }
  }
}

// Passes with at most 4 output channels (the backward pass of a first layer over 1-4 input
// channels): a 128 x 16 tile would spend most of its FMAs on padding and its shared-memory reads
// would outnumber them, and no operand value is reused across output channels anyway.  Each
// thread computes 4 rows (m, m + 256, m + 512, m + 768 of its block, so every load of a warp is
// one contiguous run of positions) times the N channels, loading its operand straight from
// global memory; the K loop reads the tap table and the N weights of each term from shared
// memory (one broadcast load each).  Each output is the same sequential FMA chain in K order as
// in k_sconv, so the result is the same bit for bit and the same a priori error bound holds.
constexpr int SN_THREADS = 256, SN_TM = 4;

template <int N>
__global__ void __launch_bounds__(SN_THREADS) k_sconv_narrow(SconvPass q, const float* __restrict__ src,
                                                            long long sstride, float* __restrict__ out,
                                                            long long ostride, const float* __restrict__ bias) {
  extern __shared__ __align__(16) uint8_t sn_raw[];
  int4* stab = reinterpret_cast<int4*>(sn_raw);
  float4* sB = reinterpret_cast<float4*>(sn_raw + (size_t)q.K * sizeof(int4));
  const int tid = threadIdx.x;
  for (int k = tid; k < q.K; k += SN_THREADS) {
    stab[k] = q.tab[k];
    const float* b = q.B + (size_t)k * N;
    sB[k] = make_float4(b[0], N > 1 ? b[1] : 0.f, N > 2 ? b[2] : 0.f, N > 3 ? b[3] : 0.f);
  }
  const float* srow[SN_TM];
  int y0[SN_TM], x0[SN_TM];
  long long mrow[SN_TM];
#pragma unroll
  for (int i = 0; i < SN_TM; ++i) {
    const long long m = (long long)blockIdx.x * (SN_THREADS * SN_TM) + i * SN_THREADS + tid;
    const bool mv = m < q.M;
    const long long r = mv ? m / q.Pm : 0;
    const int pp = mv ? (int)(m - r * q.Pm) : 0;
    const int pi = pp / q.nJ, pj = pp - (pp / q.nJ) * q.nJ;
    y0[i] = mv ? pi * q.ms + q.cy : -32768;
    x0[i] = pj * q.ms + q.cx;
    srow[i] = src + r * sstride + (mv ? (long long)y0[i] * q.Ws + x0[i] : 0);
    mrow[i] = mv ? m : -1;
  }
  __syncthreads();
  float acc[SN_TM][N];
#pragma unroll
  for (int i = 0; i < SN_TM; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) acc[i][j] = 0.f;
#pragma unroll 2
  for (int k = 0; k < q.K; ++k) {
    const int4 t = stab[k];
    const float4 b4 = sB[k];
    const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
    for (int i = 0; i < SN_TM; ++i) {
      const bool in = (unsigned)(y0[i] + t.y) < (unsigned)q.Hs && (unsigned)(x0[i] + t.z) < (unsigned)q.Ws;
      const float v = in ? srow[i][t.x] : 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) acc[i][j] = fmaf(v, bv[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < SN_TM; ++i) {
    const long long m = mrow[i];
    if (m < 0) continue;
    const long long rr = m / q.Pm;
    const int p2 = (int)(m - rr * q.Pm);
    const int ii = p2 / q.nJ, jj = p2 - (p2 / q.nJ) * q.nJ;
    const long long p = (long long)(q.oa + q.os * ii) * q.Wo + q.ob + q.os * jj;
    float* orow = out + rr * ostride + p;
#pragma unroll
    for (int j = 0; j < N; ++j) orow[(size_t)j * q.HWo] = acc[i][j] + (bias ? bias[(size_t)j * q.HWo + p] : 0.f);
  }
}

int sconv_narrow_smem(int K) { return K * (int)(sizeof(int4) + sizeof(float4)); }

int sconv_smem(int BN, int K) { return 2 * SC_BK * (SC_BM + 4) * 4 + 2 * SC_BK * (BN + 4) * 4 + K * (int)sizeof(int4); }

struct LayerF32 {
  std::vector<SconvPass> bwd;   // one per stride phase with positions
  SconvPass fwd;
};
struct SconvNet {
  bool ready = false;
  std::vector<LayerF32> ly;     // ly[i]: paper layer i (conv layers only)
  std::vector<void*> bufs;
};

std::mutex g_sc_mu;
std::vector<std::pair<const bcrown_net*, SconvNet*>> g_sc;

SconvNet* sc_of(const bcrown_net* net) {
  std::lock_guard<std::mutex> g(g_sc_mu);
  for (auto& e : g_sc)
    if (e.first == net) return e.second;
  SconvNet* t = new SconvNet();
  g_sc.push_back({net, t});
  return t;
}

int sc_upload(SconvNet* t, const void* host, size_t bytes, void** dev) {
  if (cudaMalloc(dev, bytes) != cudaSuccess) return fail(BCROWN_ERR_OOM, "FP32 conv: device tables");
  t->bufs.push_back(*dev);
  if (cudaMemcpy(*dev, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(BCROWN_ERR_CUDA, "FP32 conv: table upload");
  return BCROWN_OK;
}

// Phase a of one spatial axis of a stride-s transposed convolution: the taps k0 + s d (d < nk)
// reach input rows a + s i (i < n), whose source row is i + off - d.
void sc_phase(int a, int k, int s, int pad, int in, int* k0, int* nk, int* off, int* n) {
  *k0 = (a + pad) % s;
  *nk = *k0 < k ? (k - *k0 + s - 1) / s : 0;
  *off = (a + pad - *k0) / s;
  *n = a < in ? (in - a + s - 1) / s : 0;
}

int sc_prepare(bcrown_net* net, SconvNet* t) {
  if (t->ready) return BCROWN_OK;
  t->ly.assign(net->L, LayerF32());
  for (int i = 1; i <= net->L - 1; ++i) {
    const LayerDev& l = net->ly[i - 1];
    if (!sconv_supported(net, i)) continue;
    const int k = l.k, s = l.stride, kk = k * k;
    std::vector<float> w((size_t)l.out_c * l.in_c * kk);
    if (cudaMemcpy(w.data(), l.W, w.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(BCROWN_ERR_CUDA, "FP32 conv: copy of weights");
    LayerF32& P = t->ly[i];
    // backward phases: source Lambda^(i) (out_c x out_h x out_w), output the input map
    for (int a = 0; a < s; ++a)
      for (int b = 0; b < s; ++b) {
        int ky0, nky, offy, ny, kx0, nkx, offx, nx;
        sc_phase(a, k, s, l.pad, l.in_h, &ky0, &nky, &offy, &ny);
        sc_phase(b, k, s, l.pad, l.in_w, &kx0, &nkx, &offx, &nx);
        if (ny * nx == 0) continue;
        SconvPass q{};
        q.Pm = ny * nx;
        q.nJ = nx;
        q.N = l.in_c;
        q.K = std::max(1, l.out_c * nky * nkx);
        q.Hs = l.out_h;
        q.Ws = l.out_w;
        q.HWs = (long long)l.out_h * l.out_w;
        q.ms = 1;
        q.cy = offy;
        q.cx = offx;
        q.oa = a;
        q.ob = b;
        q.os = s;
        q.Wo = l.in_w;
        q.HWo = (long long)l.in_h * l.in_w;
        std::vector<int4> tab((size_t)q.K, make_int4(0, -32768, 0, 0));
        std::vector<float> B((size_t)q.K * q.N, 0.f);
        for (int co = 0; co < l.out_c; ++co)
          for (int dy = 0; dy < nky; ++dy)
            for (int dx = 0; dx < nkx; ++dx) {
              const int kq = (co * nky + dy) * nkx + dx;
              tab[kq] = make_int4((int)(co * q.HWs - dy * l.out_w - dx), -dy, -dx, 0);
              const int ky = ky0 + s * dy, kx = kx0 + s * dx;
              for (int ci = 0; ci < l.in_c; ++ci)
                B[(size_t)kq * q.N + ci] = w[(((size_t)co * l.in_c + ci) * k + ky) * k + kx];
            }
        void *dt = nullptr, *dB = nullptr;
        BC_CHECK(sc_upload(t, tab.data(), tab.size() * sizeof(int4), &dt));
        BC_CHECK(sc_upload(t, B.data(), B.size() * 4, &dB));
        q.tab = reinterpret_cast<const int4*>(dt);
        q.B = reinterpret_cast<const float*>(dB);
        P.bwd.push_back(q);
      }
    // forward: source h^(i-1) (in_c x in_h x in_w), output the layer's map
    SconvPass f{};
    f.Pm = l.out_h * l.out_w;
    f.nJ = l.out_w;
    f.N = l.out_c;
    f.K = l.in_c * kk;
    f.Hs = l.in_h;
    f.Ws = l.in_w;
    f.HWs = (long long)l.in_h * l.in_w;
    f.ms = s;
    f.cy = -l.pad;
    f.cx = -l.pad;
    f.oa = 0;
    f.ob = 0;
    f.os = 1;
    f.Wo = l.out_w;
    f.HWo = (long long)l.out_h * l.out_w;
    std::vector<int4> tab((size_t)f.K);
    std::vector<float> B((size_t)f.K * f.N);
    for (int ci = 0; ci < l.in_c; ++ci)
      for (int ky = 0; ky < k; ++ky)
        for (int kx = 0; kx < k; ++kx) {
          const int kq = (ci * k + ky) * k + kx;
          tab[kq] = make_int4((int)(ci * f.HWs + ky * l.in_w + kx), ky, kx, 0);
          for (int co = 0; co < l.out_c; ++co) B[(size_t)kq * f.N + co] = w[(((size_t)co * l.in_c + ci) * k + ky) * k + kx];
        }
    void *dt = nullptr, *dB = nullptr;
    BC_CHECK(sc_upload(t, tab.data(), tab.size() * sizeof(int4), &dt));
    BC_CHECK(sc_upload(t, B.data(), B.size() * 4, &dB));
    f.tab = reinterpret_cast<const int4*>(dt);
    f.B = reinterpret_cast<const float*>(dB);
    P.fwd = f;
  }
  {
    const int smem = sconv_narrow_smem(SCONV_MAX_K);
    for (cudaError_t e : {cudaFuncSetAttribute(k_sconv_narrow<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                          cudaFuncSetAttribute(k_sconv_narrow<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                          cudaFuncSetAttribute(k_sconv_narrow<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                          cudaFuncSetAttribute(k_sconv_narrow<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)})
      if (e != cudaSuccess)
        return fail(BCROWN_ERR_CUDA, std::string("FP32 conv: smem attribute: ") + cudaGetErrorString(e));
  }
  for (int BN : {16, 32, 64, 128}) {
    const int smem = sconv_smem(BN, SCONV_MAX_K);
    cudaError_t e = BN == 16    ? cudaFuncSetAttribute(k_sconv<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                    : BN == 32  ? cudaFuncSetAttribute(k_sconv<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                    : BN == 64  ? cudaFuncSetAttribute(k_sconv<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
                                : cudaFuncSetAttribute(k_sconv<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return fail(BCROWN_ERR_CUDA, std::string("FP32 conv: smem attribute: ") + cudaGetErrorString(e));
  }
  t->ready = true;
  return BCROWN_OK;
}

int sc_launch(const SconvPass& q0, int R, const float* src, long long sstride, float* out, long long ostride,
              const float* bias, cudaStream_t s) {
  SconvPass q = q0;
  q.M = (long long)R * q.Pm;
  if (q.M <= 0) return BCROWN_OK;
  if (q.N <= 4) {
    const unsigned nb = (unsigned)((q.M + SN_THREADS * SN_TM - 1) / (SN_THREADS * SN_TM));
    const int smem = sconv_narrow_smem(q.K);
    if (q.N == 1) k_sconv_narrow<1><<<nb, SN_THREADS, smem, s>>>(q, src, sstride, out, ostride, bias);
    else if (q.N == 2) k_sconv_narrow<2><<<nb, SN_THREADS, smem, s>>>(q, src, sstride, out, ostride, bias);
    else if (q.N == 3) k_sconv_narrow<3><<<nb, SN_THREADS, smem, s>>>(q, src, sstride, out, ostride, bias);
    else k_sconv_narrow<4><<<nb, SN_THREADS, smem, s>>>(q, src, sstride, out, ostride, bias);
    ++g_launches;
    return BCROWN_OK;
  }
  const int BN = q.N <= 16 ? 16 : q.N <= 32 ? 32 : q.N <= 64 ? 64 : 128;
  const dim3 grid((unsigned)((q.M + SC_BM - 1) / SC_BM), (unsigned)((q.N + BN - 1) / BN));
  const int smem = sconv_smem(BN, q.K);
  if (BN == 16) k_sconv<16><<<grid, SC_THREADS, smem, s>>>(q, src, sstride, out, ostride, bias);
  else if (BN == 32) k_sconv<32><<<grid, SC_THREADS, smem, s>>>(q, src, sstride, out, ostride, bias);
  else if (BN == 64) k_sconv<64><<<grid, SC_THREADS, smem, s>>>(q, src, sstride, out, ostride, bias);
  else k_sconv<128><<<grid, SC_THREADS, smem, s>>>(q, src, sstride, out, ostride, bias);
  ++g_launches;
  return BCROWN_OK;
}

}  // namespace

bool sconv_supported(const bcrown_net* net, int i) {
  const LayerDev& l = net->ly[i - 1];
  if (l.kind != BCROWN_LAYER_CONV) return false;
  const int T = (l.k + l.stride - 1) / l.stride;
  return (long long)l.out_c * T * T <= SCONV_MAX_K && (long long)l.in_c * l.k * l.k <= SCONV_MAX_K &&
         (long long)l.out_c * l.out_h * l.out_w < (1LL << 31) && (long long)l.in_c * l.in_h * l.in_w < (1LL << 31);
}

int sconv_load(bcrown_net* net) { return sc_prepare(net, sc_of(net)); }

int sconv_bwd(bcrown_net* net, int i, int R, const float* Lam, float* Ain, cudaStream_t s) {
  SconvNet* t = sc_of(net);
  if (!t->ready) return fail(BCROWN_ERR_ARG, "FP32 conv: tables not built");
  const LayerDev& l = net->ly[i - 1];
  for (const SconvPass& q : t->ly[i].bwd) BC_CHECK(sc_launch(q, R, Lam, l.d_out, Ain, l.d_in, nullptr, s));
  return BCROWN_OK;
}

int sconv_fwd(bcrown_net* net, int i, int R, const float* h, float* Z, const float* bias, cudaStream_t s) {
  SconvNet* t = sc_of(net);
  if (!t->ready) return fail(BCROWN_ERR_ARG, "FP32 conv: tables not built");
  const LayerDev& l = net->ly[i - 1];
  return sc_launch(t->ly[i].fwd, R, h, l.d_in, Z, l.d_out, bias, s);
}

void sconv_release(const bcrown_net* net) {
  std::lock_guard<std::mutex> g(g_sc_mu);
  for (size_t i = 0; i < g_sc.size(); ++i)
    if (g_sc[i].first == net) {
      for (void* b : g_sc[i].second->bufs) cudaFree(b);
      delete g_sc[i].second;
      g_sc.erase(g_sc.begin() + i);
      return;
    }
}

}  // namespace bcrown
