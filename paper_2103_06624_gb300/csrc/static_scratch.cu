// bcrown_bound_static: the FP32 bound pass of bcrown_bound for callers that cannot allocate
// device memory.  Its scratch (per-neuron tables and the row-chunk buffers) lives in one
// file-scope device array of fixed size instead of the net's cudaMalloc'd workspace.
//
// Who needs this: a host that must not call cudaMalloc while it runs this pass -- for example
// a real-time loop that cannot afford cudaMalloc's implicit device synchronisation and
// latency, or an embedding process that runs under a fixed device-memory budget handed out by
// its own allocator and may not grow it behind that allocator's back.  They pass inputs and
// outputs as usual; this entry point allocates nothing.
#include <algorithm>
#include <mutex>

#include "simt.cuh"

namespace bcrown {

// The array is part of the loaded module: every GPU that loads the library holds it until
// the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[BCROWN_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of the array on the current device.  Host code only sees a host-side
// stand-in for the symbol, so the address is looked up once per device (with that device
// current) and cached; the lookup is the only runtime call this set-up makes.
int static_scratch_address(void** out) {
  int dev = 0;
  BC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(BCROWN_ERR_ARG, "bound_static: device index out of range");
  std::lock_guard<std::mutex> g(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return fail(BCROWN_ERR_CUDA, std::string("bound_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return BCROWN_OK;
}

}  // namespace
}  // namespace bcrown

using namespace bcrown;

extern "C" int bcrown_bound_static(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                                   const float* alpha, const float* beta, float* lb, void* stream) {
  if (!net) return fail(BCROWN_ERR_ARG, "bound_static: null net");
  if (!dom || dom->n_props < 1 || !dom->x_lo || !dom->x_hi || (net->H > 0 && (!dom->l || !dom->u)))
    return fail(BCROWN_ERR_ARG, "bound_static: missing domain arrays");
  if (!batch || batch->B < 0 || batch->n_alpha < 0 || batch->n_beta < 0)
    return fail(BCROWN_ERR_ARG, "bound_static: bad batch");
  if (batch->B == 0) return BCROWN_OK;
  if (!lb || !batch->prop_of || !batch->split_off || !batch->split_cnt || !batch->alpha_off)
    return fail(BCROWN_ERR_ARG, "bound_static: null array");

  // Carve the fixed array: per-property tables first, then as many rows per chunk as fit.
  const size_t P = (size_t)dom->n_props;
  const size_t PH = P * (size_t)std::max(net->H, 1);
  const size_t table_bytes = align_up(PH) + 3 * align_up(PH * 4) + align_up(P * 4);
  size_t row_floats = 0;
  for (int i = 0; i < net->L; ++i) row_floats += (size_t)net->d[i];
  row_floats += (size_t)net->max_hidden;
  const size_t row_bytes = row_floats * 4 + 4;
  const size_t slack = (size_t)(net->L + 8) * 256;
  if (table_bytes + slack + row_bytes > (size_t)BCROWN_STATIC_SCRATCH_BYTES)
    return fail(BCROWN_ERR_ARG, "bound_static: " + std::to_string(P) + " properties x " + std::to_string(net->H) +
                                    " neurons exceed the static scratch of " +
                                    std::to_string((long long)BCROWN_STATIC_SCRATCH_BYTES) + " bytes");
  const long long R = (long long)batch->B * net->K;
  const long long Rc =
      std::min<long long>(R, (long long)((BCROWN_STATIC_SCRATCH_BYTES - table_bytes - slack) / row_bytes));

  void* base = nullptr;
  BC_CHECK(static_scratch_address(&base));
  // the net's lock, as every other entry point takes it: calls on one net are serialised on
  // the host (the net's status word is shared); the static array itself is shared by all nets
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  Arena ar{(char*)base};
  uint8_t* code = ar.take<uint8_t>(PH);
  int32_t* rank = ar.take<int32_t>(PH);
  float* slope = ar.take<float>(PH);
  float* icpt = ar.take<float>(PH);
  int32_t* U = ar.take<int32_t>(P);
  std::vector<float*> A(net->L);
  for (int i = 0; i < net->L; ++i) A[i] = ar.take<float>((size_t)Rc * net->d[i]);
  float* Lam = ar.take<float>((size_t)Rc * net->max_hidden);
  float* cf = ar.take<float>((size_t)Rc);
  if (ar.off > (size_t)BCROWN_STATIC_SCRATCH_BYTES) return fail(BCROWN_ERR_ARG, "bound_static: scratch plan overflow");

  // Every buffer below is fully written before it is read, so nothing needs clearing.  The
  // kernels are not timed by bcrown_profile: its event pairs may have to be created.
  Tables tb;
  launch_tables(dom->n_props, net->H, dom->l, dom->u, tb, code, rank, slope, icpt, U, s);
  RowsCtx c;
  c.K = net->K;
  c.P = dom->n_props;
  c.bt = BatchView{batch->B, batch->prop_of, batch->split_off, batch->split_cnt, batch->split_layer,
                   batch->split_idx, batch->split_sign, batch->alpha_off};
  c.tb = tb;
  c.x_lo = dom->x_lo;
  c.x_hi = dom->x_hi;
  c.l = dom->l;
  c.u = dom->u;
  c.status = net->status;
  const int L = net->L;
  const long long hoff_top = L >= 2 ? net->hoff[L - 2] : -1;
  for (long long r0 = 0; r0 < R; r0 += Rc) {
    c.r0 = (int)r0;
    c.R = (int)std::min<long long>(Rc, R - r0);
    launch_init_top(false, c, net->d[L - 1], net, hoff_top, A[L - 1], cf, nullptr, nullptr, s);
    for (int i = L - 1; i >= 1; --i) {
      const LayerDev& ly = net->ly[i - 1];
      launch_relax(false, c, i, net->d[i], net->hoff[i - 1], A[i], Lam, ly.b, alpha, batch->n_alpha, beta,
                   batch->n_beta, cf, nullptr, nullptr, nullptr, 0.0, s);
      if (ly.kind == BCROWN_LAYER_FC)
        launch_sgemm(c.R, ly.d_in, ly.d_out, Lam, ly.d_out, ly.W, ly.d_in, A[i - 1], ly.d_in, nullptr, s);
      else if (sconv_supported(net, i))
        BC_CHECK(sconv_bwd(net, i, c.R, Lam, A[i - 1], s));   // tables built at load: no allocation
      else
        launch_conv_bwd(c.R, geom_of(ly), Lam, ly.W, A[i - 1], s);
    }
    launch_concretize(false, c, net->d[0], A[0], cf, nullptr, nullptr, lb, s);
  }
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}
