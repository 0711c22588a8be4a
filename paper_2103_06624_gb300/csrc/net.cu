// Network loading and layout (paper Section 2.1, Eq. 1; spec merged into the last layer),
// the device status word, the error message and the workspace.
#include <atomic>
#include <cfenv>
#include <cmath>
#include <cstring>

#include "bcrown_internal.cuh"
#include "conv_tc.cuh"
#include "fused_tc.cuh"
#include "layer_tc.cuh"
#include "simt.cuh"

namespace bcrown {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

void* ws_get(bcrown_net* net, size_t bytes, int* status) {
  *status = BCROWN_OK;
  if (bytes <= net->ws.size) return net->ws.ptr;
  if (net->ws.ptr) {
    cudaDeviceSynchronize();
    cudaFree(net->ws.ptr);
    net->ws.ptr = nullptr;
    net->ws.size = 0;
  }
  size_t want = align_up(bytes + bytes / 8, 1 << 20);
  cudaError_t e = cudaMalloc(&net->ws.ptr, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    net->ws.ptr = nullptr;
    *status = fail(BCROWN_ERR_OOM, std::string("workspace of ") + std::to_string(want) +
                                       " bytes: " + cudaGetErrorString(e));
    return nullptr;
  }
  net->ws.size = want;
  return net->ws.ptr;
}

static cudaEvent_t pool_event(bcrown_net* net) {
  if (!net->evpool.empty()) {
    cudaEvent_t e = net->evpool.back();
    net->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Under stream capture an ordinary record only orders the captured work; an external record
// becomes an event node of the graph, recorded at every replay (so that a scope captured into
// a graph times the kernels of the latest replay).
static void prof_record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

ProfScope::ProfScope(bcrown_net* n, int cls, cudaStream_t st) : net(n), s(st) {
  if (!net->prof_on) return;
  bcrown_net::ProfRec r{cls, pool_event(net), pool_event(net)};
  prof_record(r.a, s);
  net->prof.push_back(r);
  idx = (int)net->prof.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx >= 0) prof_record(net->prof[idx].b, s);
}

static void prof_clear(bcrown_net* net) {
  for (auto& r : net->prof) {
    net->evpool.push_back(r.a);
    net->evpool.push_back(r.b);
  }
  net->prof.clear();
}

extern std::atomic<long long> g_launches;

template <class T>
static int upload(T** dst, const T* src, size_t n) {
  if (n == 0) {
    *dst = nullptr;
    return BCROWN_OK;
  }
  cudaError_t e = cudaMalloc(dst, n * sizeof(T));
  if (e != cudaSuccess) return fail(BCROWN_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(BCROWN_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
  return BCROWN_OK;
}

static std::vector<__nv_bfloat16> to_bf16(const std::vector<float>& v) {
  std::vector<__nv_bfloat16> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = __float2bfloat16_rn(v[i]);
  return o;
}

}  // namespace bcrown

using namespace bcrown;

extern "C" const char* bcrown_last_error(void) { return g_last_error.c_str(); }

extern "C" void bcrown_free_net(bcrown_net* net) {
  if (!net) return;
  cudaDeviceSynchronize();
  tc_release(net);
  tcg_release(net);
  lt_release(net);
  sconv_release(net);
  for (auto& l : net->ly) {
    cudaFree(l.W);
    cudaFree(l.Wt);
    cudaFree(l.b);
    cudaFree(l.Wbf);
    cudaFree(l.Wtbf);
  }
  cudaFree(net->Wbar);
  cudaFree(net->bbar);
  cudaFree(net->bbar_rd);
  cudaFree(net->Wbar_err);
  cudaFree(net->Wbar_bf);
  cudaFree(net->status);
  cudaFree(net->ws.ptr);
  prof_clear(net);
  for (auto e : net->evpool) cudaEventDestroy(e);
  delete net;
}

extern "C" int bcrown_load_net(const bcrown_layer* layers, int n_layers, const float* C, int K,
                               bcrown_net** out) {
  if (!layers || n_layers < 1 || !C || K < 1 || !out) return fail(BCROWN_ERR_ARG, "load_net: null or empty argument");
  if (layers[n_layers - 1].kind != BCROWN_LAYER_FC)
    return fail(BCROWN_ERR_ARG, "load_net: the last layer must be fully connected");
  bcrown_net* net = new bcrown_net();
  net->L = n_layers;
  net->K = K;
  int prev = -1;
  for (int i = 0; i < n_layers; ++i) {
    const bcrown_layer& s = layers[i];
    LayerDev l;
    l.kind = s.kind;
    l.in_c = s.in_c; l.in_h = s.in_h; l.in_w = s.in_w;
    l.out_c = s.out_c; l.out_h = s.out_h; l.out_w = s.out_w;
    l.k = s.k; l.stride = s.stride; l.pad = s.pad;
    if (s.kind == BCROWN_LAYER_FC) {
      l.in_h = l.in_w = l.out_h = l.out_w = 1;
      l.k = 1; l.stride = 1; l.pad = 0;
    } else if (s.kind == BCROWN_LAYER_CONV) {
      if (s.k < 1 || s.stride < 1 || s.pad < 0 ||
          s.out_h != (s.in_h + 2 * s.pad - s.k) / s.stride + 1 ||
          s.out_w != (s.in_w + 2 * s.pad - s.k) / s.stride + 1) {
        delete net;
        return fail(BCROWN_ERR_ARG, "load_net: inconsistent convolution shape at layer " + std::to_string(i + 1));
      }
    } else {
      delete net;
      return fail(BCROWN_ERR_ARG, "load_net: unknown layer kind");
    }
    l.d_in = l.in_c * l.in_h * l.in_w;
    l.d_out = l.out_c * l.out_h * l.out_w;
    if (l.d_in <= 0 || l.d_out <= 0 || !s.W || !s.b || (prev >= 0 && prev != l.d_in)) {
      delete net;
      return fail(BCROWN_ERR_ARG, "load_net: layer " + std::to_string(i + 1) + " does not chain");
    }
    prev = l.d_out;
    net->ly.push_back(l);
  }
  net->d.push_back(net->ly[0].d_in);
  for (auto& l : net->ly) net->d.push_back(l.d_out);
  long long off = 0;
  for (int i = 1; i < n_layers; ++i) {
    net->hoff.push_back(off);
    off += net->d[i];
    net->max_hidden = std::max(net->max_hidden, net->d[i]);
  }
  net->hoff.push_back(off);
  net->H = (int)off;
  for (int i = 0; i < n_layers; ++i) net->max_width = std::max(net->max_width, net->d[i]);

  int st = BCROWN_OK;
  for (int i = 0; i < n_layers && st == BCROWN_OK; ++i) {
    const bcrown_layer& s = layers[i];
    LayerDev& l = net->ly[i];
    if (i == n_layers - 1) break;  // last layer only through Wbar
    if (l.kind == BCROWN_LAYER_FC) {
      std::vector<float> W(s.W, s.W + (size_t)l.d_out * l.d_in), Wt((size_t)l.d_in * l.d_out);
      for (int o = 0; o < l.d_out; ++o)
        for (int q = 0; q < l.d_in; ++q) Wt[(size_t)q * l.d_out + o] = W[(size_t)o * l.d_in + q];
      st = upload(&l.W, W.data(), W.size());
      if (st == BCROWN_OK) st = upload(&l.Wt, Wt.data(), Wt.size());
      auto Wb = to_bf16(W), Wtb = to_bf16(Wt);
      if (st == BCROWN_OK) st = upload(&l.Wbf, Wb.data(), Wb.size());
      if (st == BCROWN_OK) st = upload(&l.Wtbf, Wtb.data(), Wtb.size());
      std::vector<float> b(s.b, s.b + l.d_out);
      if (st == BCROWN_OK) st = upload(&l.b, b.data(), b.size());
      l.terms_bwd = l.d_out;
      l.terms_fwd = l.d_in;
    } else {
      size_t nw = (size_t)l.out_c * l.in_c * l.k * l.k;
      st = upload(&l.W, s.W, nw);
      std::vector<float> b((size_t)l.d_out);
      for (int c = 0; c < l.out_c; ++c)
        for (int p = 0; p < l.out_h * l.out_w; ++p) b[(size_t)c * l.out_h * l.out_w + p] = s.b[c];
      if (st == BCROWN_OK) st = upload(&l.b, b.data(), b.size());
      int taps = (l.k + l.stride - 1) / l.stride;
      l.terms_bwd = l.out_c * taps * taps;
      l.terms_fwd = l.in_c * l.k * l.k;
    }
  }
  if (st == BCROWN_OK) {
    // Wbar = C W^(L), bbar = C b^(L), in FP64 (Section 2.1: the spec is the output layer).
    const bcrown_layer& s = layers[n_layers - 1];
    const LayerDev& l = net->ly[n_layers - 1];
    int dL = l.d_out, dp = l.d_in;
    std::vector<float> Wbar((size_t)K * dp), bbar(K), Wbar_err((size_t)K * dp);
    std::vector<double> bbar_rd(K);
    const double u64 = std::ldexp(1.0, -53), u32 = std::ldexp(1.0, -24);
    for (int k = 0; k < K; ++k) {
      double bb = 0.0, ab = 0.0;
      for (int o = 0; o < dL; ++o) {
        double t = (double)C[(size_t)k * dL + o] * (double)s.b[o];  // exact: 24-bit x 24-bit
        bb += t;
        ab += std::fabs(t);
      }
      bbar[k] = (float)bb;
      // a priori bound of a recursive FP64 sum of dL exact terms: gamma_dL * sum |t|
      bbar_rd[k] = bb - 2.0 * (dL + 1) * u64 * ab - 1e-300;
      for (int q = 0; q < dp; ++q) {
        double w = 0.0, aw = 0.0;
        for (int o = 0; o < dL; ++o) {
          double t = (double)C[(size_t)k * dL + o] * (double)s.W[(size_t)o * dp + q];
          w += t;
          aw += std::fabs(t);
        }
        float wf = (float)w;
        Wbar[(size_t)k * dp + q] = wf;
        // |fl32(w) - exact| <= |fl32(w) - w| + |w - exact|; stored rounded up generously
        double err = std::fabs((double)wf - w) + 2.0 * (dL + 1) * u64 * aw;
        Wbar_err[(size_t)k * dp + q] = (float)(err * (1.0 + 4 * u32)) + 1e-38f;
      }
    }
    st = upload(&net->Wbar, Wbar.data(), Wbar.size());
    if (st == BCROWN_OK) st = upload(&net->bbar, bbar.data(), bbar.size());
    if (st == BCROWN_OK) st = upload(&net->bbar_rd, bbar_rd.data(), bbar_rd.size());
    if (st == BCROWN_OK) st = upload(&net->Wbar_err, Wbar_err.data(), Wbar_err.size());
    auto Wbb = to_bf16(Wbar);
    if (st == BCROWN_OK) st = upload(&net->Wbar_bf, Wbb.data(), Wbb.size());
  }
  if (st == BCROWN_OK) {
    cudaError_t e = cudaMalloc(&net->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(net->status, 0, sizeof(int));
    if (e != cudaSuccess) st = fail(BCROWN_ERR_CUDA, std::string("status word: ") + cudaGetErrorString(e));
  }
  // the FP32 convolutions' phase weights and gather tables, built here so that no later call
  // (the allocation-free bound included) allocates them
  if (st == BCROWN_OK) st = sconv_load(net);
  if (st != BCROWN_OK) {
    bcrown_free_net(net);
    return st;
  }
  *out = net;
  return BCROWN_OK;
}

extern "C" int bcrown_net_info(const bcrown_net* net, int* n_layers, int* widths, int* K) {
  if (!net) return fail(BCROWN_ERR_ARG, "net_info: null net");
  if (n_layers) *n_layers = net->L;
  if (widths)
    for (int i = 0; i <= net->L; ++i) widths[i] = net->d[i];
  if (K) *K = net->K;
  return BCROWN_OK;
}

extern "C" int bcrown_status(bcrown_net* net, void* stream) {
  if (!net) return fail(BCROWN_ERR_ARG, "status: null net");
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  BC_CUDA(cudaMemcpyAsync(&h, net->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  BC_CUDA(cudaStreamSynchronize(s));
  BC_CUDA(cudaMemsetAsync(net->status, 0, sizeof(int), s));
  BC_CUDA(cudaStreamSynchronize(s));
  if (h != BCROWN_OK) set_error("device status " + std::to_string(h));
  return h;
}

extern "C" int bcrown_profile(bcrown_net* net, int enable) {
  if (!net) return fail(BCROWN_ERR_ARG, "profile: null net");
  std::lock_guard<std::mutex> g(net->mu);
  BC_CUDA(cudaDeviceSynchronize());
  prof_clear(net);
  net->prof_on = enable != 0;
  return BCROWN_OK;
}

extern "C" int bcrown_profile_read(bcrown_net* net, int cls, double* total_ms, long long* launches) {
  if (!net || cls < 0 || cls >= BCROWN_PROF_NCLASS) return fail(BCROWN_ERR_ARG, "profile_read: bad argument");
  std::lock_guard<std::mutex> g(net->mu);
  double t = 0.0;
  long long n = 0;
  for (auto& r : net->prof) {
    if (r.cls != cls) continue;
    BC_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    BC_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    t += ms;
    ++n;
  }
  if (total_ms) *total_ms = t;
  if (launches) *launches = n;
  return BCROWN_OK;
}

extern "C" long long bcrown_kernel_launches(void) { return g_launches.load(); }

extern "C" int bcrown_workspace(bcrown_net* net, int64_t reserve_bytes, void** ptr, int64_t* bytes) {
  if (!net || reserve_bytes < 0) return fail(BCROWN_ERR_ARG, "workspace: bad argument");
  std::lock_guard<std::mutex> g(net->mu);
  if (reserve_bytes > 0) {
    int st = BCROWN_OK;
    if (!ws_get(net, (size_t)reserve_bytes, &st)) return st;
  }
  if (ptr) *ptr = net->ws.ptr;
  if (bytes) *bytes = (int64_t)net->ws.size;
  return BCROWN_OK;
}
