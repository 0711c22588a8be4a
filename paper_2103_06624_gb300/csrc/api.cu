// C-ABI entry points: root bounds, bound, bound + gradient, projected Adam, batch_split,
// neuron codes.  Orchestrates the kernels of simt.cu (and the tensor-core path of
// fused_tc.cu for BCROWN_BF16) on the caller's stream.
#include <algorithm>
#include <cmath>

#include "conv_tc.cuh"
#include "fused_tc.cuh"
#include "layer_tc.cuh"
#include "simt.cuh"

using namespace bcrown;

namespace bcrown {

static const size_t kChunkBytes = size_t(8) << 30;  // per-chunk workspace target

static int check_domain(const bcrown_net* net, const bcrown_domain* dom) {
  if (!dom || dom->n_props < 1 || !dom->x_lo || !dom->x_hi || (net->H > 0 && (!dom->l || !dom->u)))
    return fail(BCROWN_ERR_ARG, "domain: missing arrays or n_props < 1");
  return BCROWN_OK;
}

static int check_batch(const bcrown_batch* bt) {
  if (!bt || bt->B < 0) return fail(BCROWN_ERR_ARG, "batch: null or negative B");
  if (bt->B > 0 && (!bt->prop_of || !bt->split_off || !bt->split_cnt || !bt->alpha_off))
    return fail(BCROWN_ERR_ARG, "batch: missing arrays");
  if (bt->n_alpha < 0 || bt->n_beta < 0) return fail(BCROWN_ERR_ARG, "batch: negative n_alpha/n_beta");
  return BCROWN_OK;
}

static BatchView view_of(const bcrown_batch* bt) {
  return BatchView{bt->B, bt->prop_of, bt->split_off, bt->split_cnt, bt->split_layer, bt->split_idx,
                   bt->split_sign, bt->alpha_off};
}

static double gamma_n(long long n) {
  const double u = std::ldexp(1.0, -24);
  double nu = (double)n * u;
  return nu / (1.0 - nu) * (1.0 + 1e-6);
}

// Workspace carve-up for one call.
struct Plan {
  int P, H, R, Rc;
  // tables
  uint8_t* code;
  int32_t* rank;
  float* slope;
  float* icpt;
  int32_t* U;
  float* wm;
  Tables tb;
  // chunk buffers
  std::vector<float*> Abuf;  // [L] : Abuf[i] for hidden i (1..L-1), Abuf[0] = A^(0)
  float* Lam;
  float* Z0;
  float* Z1;
  float* cf;
  double* cd;
  double* E;
  // optimiser state (optional)
  float *a_cur, *ma, *va, *ga, *b_cur, *mb, *vb, *gb, *best_lb, *lb_t;
  char* tc_ws;
  size_t tc_ws_bytes;
  // BF16 layer-by-layer path (null when unused)
  char* lt_ws = nullptr;
  size_t lt_ws_bytes = 0;
  // BF16 conv layers on the tensor cores: the im2col operand of one chunk (null when unused)
  char* col = nullptr;
  size_t col_bytes = 0;
};

static size_t row_bytes(const bcrown_net* net) {
  size_t f = 0;
  for (int i = 0; i < net->L; ++i) f += (size_t)net->d[i];  // A^(0..L-1)
  f += (size_t)net->max_hidden + 2 * (size_t)net->max_width;
  return f * 4 + 4 + 16 + 3 * 256;
}

static int make_plan(bcrown_net* net, int P, int R, bool cert, bool opt, int64_t n_alpha, int64_t n_beta,
                     size_t tc_bytes, Plan& pl, size_t col_per_row = 0, size_t lt_bytes = 0) {
  pl.P = P;
  pl.H = net->H;
  pl.R = R;
  size_t rb = row_bytes(net) + col_per_row;
  long long rc = std::max<long long>(1, (long long)(kChunkBytes / rb));
  pl.Rc = (int)std::min<long long>(std::max(R, 1), rc);
  size_t PH = (size_t)P * std::max(net->H, 1);
  size_t bytes = 0;
  bytes += align_up(PH) + align_up(PH * 4) * 3 + align_up((size_t)P * 4);
  if (cert) bytes += align_up(PH * 4);
  bytes += (size_t)pl.Rc * rb + 16 * 256;
  if (opt) bytes += align_up((size_t)n_alpha * 4) * 4 + align_up((size_t)n_beta * 4) * 4 + align_up((size_t)R * 4) * 2;
  bytes += align_up(tc_bytes) + align_up(lt_bytes);
  int st;
  void* base = ws_get(net, bytes, &st);
  if (!base) return st;
  Arena ar{(char*)base};
  pl.code = ar.take<uint8_t>(PH);
  pl.rank = ar.take<int32_t>(PH);
  pl.slope = ar.take<float>(PH);
  pl.icpt = ar.take<float>(PH);
  pl.U = ar.take<int32_t>(P);
  pl.wm = cert ? ar.take<float>(PH) : nullptr;
  pl.Abuf.assign(net->L, nullptr);
  for (int i = 0; i < net->L; ++i) pl.Abuf[i] = ar.take<float>((size_t)pl.Rc * net->d[i]);
  pl.Lam = ar.take<float>((size_t)pl.Rc * net->max_hidden);
  pl.Z0 = ar.take<float>((size_t)pl.Rc * net->max_width);
  pl.Z1 = ar.take<float>((size_t)pl.Rc * net->max_width);
  pl.cf = ar.take<float>(pl.Rc);
  pl.cd = ar.take<double>(pl.Rc);
  pl.E = ar.take<double>(pl.Rc);
  if (col_per_row) {
    pl.col_bytes = (size_t)pl.Rc * col_per_row;
    pl.col = ar.take<char>(pl.col_bytes);
  }
  if (opt) {
    pl.a_cur = ar.take<float>(n_alpha);
    pl.ma = ar.take<float>(n_alpha);
    pl.va = ar.take<float>(n_alpha);
    pl.ga = ar.take<float>(n_alpha);
    pl.b_cur = ar.take<float>(n_beta);
    pl.mb = ar.take<float>(n_beta);
    pl.vb = ar.take<float>(n_beta);
    pl.gb = ar.take<float>(n_beta);
    pl.best_lb = ar.take<float>(R);
    pl.lb_t = ar.take<float>(R);
  }
  pl.tc_ws = tc_bytes ? ar.take<char>(tc_bytes) : nullptr;
  pl.tc_ws_bytes = tc_bytes;
  pl.lt_ws = lt_bytes ? ar.take<char>(lt_bytes) : nullptr;
  pl.lt_ws_bytes = lt_bytes;
  if (ar.off > net->ws.size) return fail(BCROWN_ERR_OOM, "workspace plan overflow");
  return BCROWN_OK;
}

// ---- BF16 launch configuration (bcrown_set_launch, bcrown_autotune) ----
static bool path_ok(const bcrown_net* net, int path) {
  switch (path) {
    case BCROWN_PATH_FUSED: return tc_supported(net);
    case BCROWN_PATH_LAYER_EPI: return lt_supported(net);
    case BCROWN_PATH_LAYER_GATHER:
    case BCROWN_PATH_LAYER_IM2COL: return tcg_supported(net);
    default: return false;
  }
}

static int bucket_of(long long rows) {
  int b = 0;
  while ((1LL << b) < rows) ++b;
  return b;
}

// The configuration a BF16 call with `rows` rows takes (path 0: the net takes none).
static bcrown_net::Launch resolve_launch(const bcrown_net* net, long long rows) {
  const int bk = bucket_of(rows);
  for (const auto& t : net->tuned)
    if (t.first == bk && path_ok(net, t.second.path)) return t.second;
  if (net->launch_set.path && path_ok(net, net->launch_set.path)) return net->launch_set;
  bcrown_net::Launch l;
  l.grid_per_sm = net->launch_set.grid_per_sm;
  for (int p : {BCROWN_PATH_FUSED, BCROWN_PATH_LAYER_EPI, BCROWN_PATH_LAYER_GATHER, BCROWN_PATH_LAYER_IM2COL})
    if (path_ok(net, p)) {
      l.path = p;
      return l;
    }
  l.path = 0;
  return l;
}

static int bf16_path(const bcrown_net* net, int precision, long long rows) {
  return precision == BCROWN_BF16 ? resolve_launch(net, rows).path : 0;
}

static void build_tables(bcrown_net* net, const bcrown_domain* dom, Plan& pl, cudaStream_t s) {
  launch_tables(dom->n_props, net->H, dom->l, dom->u, pl.tb, pl.code, pl.rank, pl.slope, pl.icpt, pl.U, s);
}

static void build_wm(bcrown_net* net, const bcrown_domain* dom, Plan& pl, cudaStream_t s) {
  for (int i = 1; i < net->L; ++i) {
    long long hprev = i >= 2 ? net->hoff[i - 2] : -1;
    launch_absw_m(geom_of(net->ly[i - 1]), net->ly[i - 1].W, dom->n_props, net->H, net->hoff[i - 1], hprev, dom->u,
                  dom->x_lo, dom->x_hi, net->d[0], pl.wm, s);
  }
}

static RowsCtx ctx_of(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* bt, const Plan& pl, int r0,
                      int Rc) {
  RowsCtx c;
  c.r0 = r0;
  c.R = Rc;
  c.K = net->K;
  c.P = dom->n_props;
  c.bt = view_of(bt);
  c.tb = pl.tb;
  c.x_lo = dom->x_lo;
  c.x_hi = dom->x_hi;
  c.l = dom->l;
  c.u = dom->u;
  c.status = net->status;
  return c;
}

// Backward contraction of layer i: Aout = Lam W^(i) (fc) or transposed convolution.
// tc: BF16 tensor-core GEMMs (over an im2col operand for conv layers) with the operand in pl.col.
static int contract_bwd(bcrown_net* net, int i, int Rc, const float* Lam, float* Aout, cudaStream_t s,
                        const Plan* tc = nullptr) {
  ProfScope ps(net, tc ? BCROWN_PROF_LAYER_GEMM : BCROWN_PROF_CONTRACT, s);
  const LayerDev& l = net->ly[i - 1];
  if (tc)
    return tcg_conv(net, i, false, Rc, Lam, Aout, nullptr, tc->col, tc->col_bytes, s);
  if (l.kind == BCROWN_LAYER_FC)
    launch_sgemm(Rc, l.d_in, l.d_out, Lam, l.d_out, l.W, l.d_in, Aout, l.d_in, nullptr, s);
  else if (sconv_supported(net, i))
    return sconv_bwd(net, i, Rc, Lam, Aout, s);
  else
    launch_conv_bwd(Rc, geom_of(l), Lam, l.W, Aout, s);
  return BCROWN_OK;
}

// Forward contraction of layer i: Z = h W^(i)^T + b^(i).
static int contract_fwd(bcrown_net* net, int i, int Rc, const float* h, float* Z, cudaStream_t s,
                        const Plan* tc = nullptr) {
  ProfScope ps(net, tc ? BCROWN_PROF_LAYER_GEMM : BCROWN_PROF_CONTRACT, s);
  const LayerDev& l = net->ly[i - 1];
  if (tc)
    return tcg_conv(net, i, true, Rc, h, Z, l.b, tc->col, tc->col_bytes, s);
  if (l.kind == BCROWN_LAYER_FC)
    launch_sgemm(Rc, l.d_out, l.d_in, h, l.d_in, l.Wt, l.d_out, Z, l.d_out, l.b, s);
  else if (sconv_supported(net, i))
    return sconv_fwd(net, i, Rc, h, Z, l.b, s);
  else
    launch_conv_fwd(Rc, geom_of(l), h, l.W, l.b, Z, s);
  return BCROWN_OK;
}

// One chunk of rows: bound (and optionally the gradient) with the SIMT path.
static int chunk_simt(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* bt, Plan& pl, int r0, int Rc,
                      bool cert, bool grad, const float* alpha, const float* beta, float* lb, float* dalpha,
                      float* dbeta, cudaStream_t s, bool tc_layers = false, float* xstar = nullptr) {
  const Plan* tc = tc_layers ? &pl : nullptr;
  RowsCtx c = ctx_of(net, dom, bt, pl, r0, Rc);
  const int L = net->L;
  long long hoff_top = L >= 2 ? net->hoff[L - 2] : -1;
  launch_init_top(cert, c, net->d[L - 1], net, hoff_top, pl.Abuf[L - 1], pl.cf, pl.cd, pl.E, s);
  for (int i = L - 1; i >= 1; --i) {
    const LayerDev& ly = net->ly[i - 1];
    {
      ProfScope ps(net, BCROWN_PROF_RELAX, s);
      launch_relax(cert, c, i, net->d[i], net->hoff[i - 1], pl.Abuf[i], pl.Lam, ly.b, alpha, bt->n_alpha, beta, bt->n_beta, pl.cf,
                 pl.cd, pl.E, pl.wm, gamma_n(ly.terms_bwd), s);
    }
    BC_CHECK(contract_bwd(net, i, Rc, pl.Lam, pl.Abuf[i - 1], s, tc));
  }
  {
    ProfScope ps(net, BCROWN_PROF_CONCRETIZE, s);
    launch_concretize(cert, c, net->d[0], pl.Abuf[0], pl.cf, pl.cd, pl.E, lb, s);
  }
  if (xstar) launch_xstar(c, net->d[0], pl.Abuf[0], xstar + (size_t)r0 * net->d[0], s);
  if (!grad) return BCROWN_OK;
  launch_xstar(c, net->d[0], pl.Abuf[0], pl.Z0, s);
  float* h = pl.Z0;
  float* z = pl.Z1;
  for (int i = 1; i <= L - 1; ++i) {
    BC_CHECK(contract_fwd(net, i, Rc, h, z, s, tc));
    ProfScope ps(net, BCROWN_PROF_ADJOINT, s);
    launch_fwd_epi(c, i, net->d[i], net->hoff[i - 1], z, pl.Abuf[i], alpha, bt->n_alpha, dalpha, dbeta, bt->n_beta, s);
    std::swap(h, z);
  }
  return BCROWN_OK;
}

// tc_plan: group the batch's rows into property tiles first (false when an earlier call on the
// same batch and plan already did).
static int run_bound(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* bt, Plan& pl, int precision,
                     bool grad, const float* alpha, const float* beta, float* lb, float* dalpha, float* dbeta,
                     cudaStream_t s, bool tc_plan = true) {
  const int R = bt->B * net->K;
  net->launch_now = precision == BCROWN_BF16 ? resolve_launch(net, R) : bcrown_net::Launch{};
  const int path = net->launch_now.path;
  if (path == BCROWN_PATH_FUSED) {
    return tc_bound(net, dom, bt, pl.tb, pl.tc_ws, pl.tc_ws_bytes, grad, tc_plan, alpha, beta, lb, dalpha, dbeta, s);
  }
  if (path == BCROWN_PATH_LAYER_EPI && pl.lt_ws)
    return lt_bound(net, dom, bt, pl.tb, pl.lt_ws, pl.lt_ws_bytes, grad, alpha, beta, lb, dalpha, dbeta, s);
  bool cert = precision == BCROWN_CERTIFY;
  // BF16 beyond the fused kernel (conv layers, wide fc layers): the contractions on the tensor
  // cores, the rest of the layer-by-layer path in FP32; planned when the plan has an im2col buffer
  const bool tc_layers = precision == BCROWN_BF16 && pl.col != nullptr;
  for (int r0 = 0; r0 < R; r0 += pl.Rc) {
    int Rc = std::min(pl.Rc, R - r0);
    BC_CHECK(chunk_simt(net, dom, bt, pl, r0, Rc, cert, grad, alpha, beta, lb, dalpha, dbeta, s, tc_layers));
  }
  return BCROWN_OK;
}

// The BF16 layer-by-layer path with fused epilogues: workspace bytes (0: not taken).
static size_t layer_lt_bytes(bcrown_net* net, int precision, int R, int P, int64_t n_alpha, bool grad) {
  return bf16_path(net, precision, R) == BCROWN_PATH_LAYER_EPI ? lt_workspace_bytes(net, R, P, n_alpha, grad) : 0;
}

// im2col bytes per row for the older BF16 layer path (GEMMs only, FP32 epilogue kernels), taken
// for networks the fused-epilogue path does not take (0: not taken).
static size_t layer_tc_col(bcrown_net* net, int precision, int R) {
  // at least 16 bytes, so that the plan's col pointer also marks the path taken
  const int path = bf16_path(net, precision, R);
  return path == BCROWN_PATH_LAYER_GATHER || path == BCROWN_PATH_LAYER_IM2COL
             ? std::max<size_t>(tcg_col_bytes_per_row(net, path == BCROWN_PATH_LAYER_GATHER), 16)
             : 0;
}

// Workspace of the fused kernel (0 unless the call takes it).
static size_t fused_bytes(bcrown_net* net, int precision, const bcrown_batch* bt, int P, bool grad) {
  return bf16_path(net, precision, (long long)bt->B * net->K) == BCROWN_PATH_FUSED
             ? tc_workspace_bytes(net, bt->B, P, grad)
             : 0;
}

static int check_precision(bcrown_net* net, int precision, bool grad) {
  if (precision != BCROWN_FP32 && precision != BCROWN_BF16 && precision != BCROWN_CERTIFY)
    return fail(BCROWN_ERR_ARG, "unknown precision");
  if (grad && precision == BCROWN_CERTIFY) return fail(BCROWN_ERR_ARG, "gradient in CERTIFY precision is not offered");
  if (precision == BCROWN_BF16 && resolve_launch(net, 1).path == 0)
    return fail(BCROWN_ERR_UNIMPLEMENTED,
                "BF16 tensor-core path needs conv layers of at most 256 channels (and K = channels x taps <= 2048) "
                "and fc layers of at most 65536 neurons");
  return BCROWN_OK;
}

}  // namespace bcrown

extern "C" int bcrown_bound(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                            const float* alpha, const float* beta, int precision, float* lb, void* stream) {
  if (!net) return fail(BCROWN_ERR_ARG, "bound: null net");
  BC_CHECK(check_domain(net, dom));
  BC_CHECK(check_batch(batch));
  BC_CHECK(check_precision(net, precision, false));
  if (batch->B == 0) return BCROWN_OK;
  if (!lb) return fail(BCROWN_ERR_ARG, "bound: null lb");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  Plan pl;
  int R = batch->B * net->K;
  size_t tcb = fused_bytes(net, precision, batch, dom->n_props, false);
  BC_CHECK(make_plan(net, dom->n_props, R, precision == BCROWN_CERTIFY, false, 0, 0, tcb, pl,
                     layer_tc_col(net, precision, R), layer_lt_bytes(net, precision, R, dom->n_props, batch->n_alpha, false)));
  build_tables(net, dom, pl, s);
  if (precision == BCROWN_CERTIFY) build_wm(net, dom, pl, s);
  BC_CHECK(run_bound(net, dom, batch, pl, precision, false, alpha, beta, lb, nullptr, nullptr, s));
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

extern "C" int bcrown_bound_grad(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                                 const float* alpha, const float* beta, int precision, float* lb, float* dalpha,
                                 float* dbeta, void* stream) {
  if (!net) return fail(BCROWN_ERR_ARG, "bound_grad: null net");
  BC_CHECK(check_domain(net, dom));
  BC_CHECK(check_batch(batch));
  BC_CHECK(check_precision(net, precision, true));
  if (batch->B == 0) return BCROWN_OK;
  if (!lb || (batch->n_alpha && !dalpha) || (batch->n_beta && !dbeta))
    return fail(BCROWN_ERR_ARG, "bound_grad: null output");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  Plan pl;
  int R = batch->B * net->K;
  size_t tcb = fused_bytes(net, precision, batch, dom->n_props, true);
  BC_CHECK(make_plan(net, dom->n_props, R, false, false, 0, 0, tcb, pl,
                     layer_tc_col(net, precision, R), layer_lt_bytes(net, precision, R, dom->n_props, batch->n_alpha, true)));
  build_tables(net, dom, pl, s);
  BC_CHECK(run_bound(net, dom, batch, pl, precision, true, alpha, beta, lb, dalpha, dbeta, s));
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

extern "C" int bcrown_optimize(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                               const bcrown_opt_cfg* cfg, float* alpha, float* beta, float* lb_out,
                               bcrown_opt_state* state, void* stream) {
  if (!net || !cfg) return fail(BCROWN_ERR_ARG, "optimize: null net or cfg");
  BC_CHECK(check_domain(net, dom));
  BC_CHECK(check_batch(batch));
  BC_CHECK(check_precision(net, cfg->precision, true));
  if (cfg->iters < 0) return fail(BCROWN_ERR_ARG, "optimize: negative iterations");
  if (batch->B == 0) return BCROWN_OK;
  if (!lb_out || (batch->n_alpha && !alpha) || (batch->n_beta && !beta))
    return fail(BCROWN_ERR_ARG, "optimize: null buffer");
  if (state && state->t < 0) return fail(BCROWN_ERR_ARG, "optimize: negative state iteration count");
  if (state && ((batch->n_alpha && (!state->alpha_cur || !state->m_alpha || !state->v_alpha)) ||
                (batch->n_beta && (!state->beta_cur || !state->m_beta || !state->v_beta)) || !state->best_lb))
    return fail(BCROWN_ERR_ARG, "optimize: state with a null array");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  const int R = batch->B * net->K;
  const int64_t na = batch->n_alpha, nb = batch->n_beta;
  Plan pl;
  size_t tcb = fused_bytes(net, cfg->precision, batch, dom->n_props, true);
  bool cert = cfg->certify != 0;
  BC_CHECK(make_plan(net, dom->n_props, R, cert, true, na, nb, tcb, pl,
                     layer_tc_col(net, cfg->precision, R), layer_lt_bytes(net, cfg->precision, R, dom->n_props, na, true)));
  build_tables(net, dom, pl, s);
  if (cert) build_wm(net, dom, pl, s);
  const bool fused16 = bf16_path(net, cfg->precision, R) == BCROWN_PATH_FUSED;
  // the BF16 path keeps alpha's gradient and moments in BF16 (the first half of each buffer)
  __nv_bfloat16* ma16 = reinterpret_cast<__nv_bfloat16*>(pl.ma);
  __nv_bfloat16* va16 = reinterpret_cast<__nv_bfloat16*>(pl.va);
  const bool resume = state && state->t > 0;
  const int t0 = state ? state->t : 0;
  if (na) {
    const size_t st = fused16 ? 2 : 4;
    BC_CUDA(cudaMemcpyAsync(pl.a_cur, resume ? state->alpha_cur : alpha, na * 4, cudaMemcpyDeviceToDevice, s));
    if (resume && fused16) {
      launch_f32_to_bf16(state->m_alpha, ma16, na, s);
      launch_f32_to_bf16(state->v_alpha, va16, na, s);
    } else if (resume) {
      BC_CUDA(cudaMemcpyAsync(pl.ma, state->m_alpha, na * 4, cudaMemcpyDeviceToDevice, s));
      BC_CUDA(cudaMemcpyAsync(pl.va, state->v_alpha, na * 4, cudaMemcpyDeviceToDevice, s));
    } else {
      BC_CUDA(cudaMemsetAsync(pl.ma, 0, na * st, s));
      BC_CUDA(cudaMemsetAsync(pl.va, 0, na * st, s));
    }
    BC_CUDA(cudaMemsetAsync(pl.ga, 0, na * st, s));
  }
  if (nb) {
    BC_CUDA(cudaMemcpyAsync(pl.b_cur, resume ? state->beta_cur : beta, nb * 4, cudaMemcpyDeviceToDevice, s));
    if (resume) {
      BC_CUDA(cudaMemcpyAsync(pl.mb, state->m_beta, nb * 4, cudaMemcpyDeviceToDevice, s));
      BC_CUDA(cudaMemcpyAsync(pl.vb, state->v_beta, nb * 4, cudaMemcpyDeviceToDevice, s));
    } else {
      BC_CUDA(cudaMemsetAsync(pl.mb, 0, nb * 4, s));
      BC_CUDA(cudaMemsetAsync(pl.vb, 0, nb * 4, s));
    }
    BC_CUDA(cudaMemsetAsync(pl.gb, 0, nb * 4, s));
  }
  if (resume)
    BC_CUDA(cudaMemcpyAsync(pl.best_lb, state->best_lb, (size_t)R * 4, cudaMemcpyDeviceToDevice, s));
  else
    launch_fill(pl.best_lb, R, -INFINITY, s);
  BatchView bv = view_of(batch);
  // a frozen group takes zero steps (the Adam kernels then leave an iterate inside its box as it was)
  const float lr_a0 = (cfg->freeze & BCROWN_FREEZE_ALPHA) ? 0.f : cfg->lr_alpha;
  const float lr_b0 = (cfg->freeze & BCROWN_FREEZE_BETA) ? 0.f : cfg->lr_beta;
  for (int it = 0; it < cfg->iters; ++it) {
    const int t = t0 + it;   // iteration index of the whole ascent (learning-rate decay, bias correction)
    float fac = std::pow(cfg->decay, (float)t);
    float bc1 = 1.f - std::pow(cfg->adam_beta1, (float)(t + 1));
    float bc2 = 1.f - std::pow(cfg->adam_beta2, (float)(t + 1));
    if (fused16) {
      // BF16 path: gradient and Adam moments of alpha in BF16 (the FP32 buffers hold them)
      __nv_bfloat16* ga16 = reinterpret_cast<__nv_bfloat16*>(pl.ga);
      BC_CHECK(tc_bound(net, dom, batch, pl.tb, pl.tc_ws, pl.tc_ws_bytes, true, it == 0, pl.a_cur, pl.b_cur, pl.lb_t,
                        nullptr, pl.gb, s, ga16));
      ProfScope ps(net, BCROWN_PROF_ADAM, s);
      launch_adam16(R, net->K, bv, pl.U, dom->n_props, pl.lb_t, pl.best_lb, pl.a_cur, alpha, ga16,
                    ma16, va16, pl.b_cur, beta,
                    pl.gb, pl.mb, pl.vb, lr_a0 * fac, lr_b0 * fac, cfg->adam_beta1, cfg->adam_beta2,
                    cfg->adam_eps, bc1, bc2, na, nb, s);
      continue;
    }
    BC_CHECK(run_bound(net, dom, batch, pl, cfg->precision, true, pl.a_cur, pl.b_cur, pl.lb_t, pl.ga, pl.gb, s,
                       it == 0));
    ProfScope ps(net, BCROWN_PROF_ADAM, s);
    launch_adam(R, net->K, bv, pl.U, dom->n_props, pl.lb_t, pl.best_lb, pl.a_cur, alpha, pl.ga, pl.ma, pl.va,
                pl.b_cur, beta, pl.gb, pl.mb, pl.vb, lr_a0 * fac, lr_b0 * fac, cfg->adam_beta1,
                cfg->adam_beta2, cfg->adam_eps, bc1, bc2, na, nb, s);
  }
  if (state) {
    // the state after this call's iterations, for the next call to continue from
    if (na) {
      BC_CUDA(cudaMemcpyAsync(state->alpha_cur, pl.a_cur, na * 4, cudaMemcpyDeviceToDevice, s));
      if (fused16) {
        launch_bf16_to_f32(ma16, state->m_alpha, na, s);
        launch_bf16_to_f32(va16, state->v_alpha, na, s);
      } else {
        BC_CUDA(cudaMemcpyAsync(state->m_alpha, pl.ma, na * 4, cudaMemcpyDeviceToDevice, s));
        BC_CUDA(cudaMemcpyAsync(state->v_alpha, pl.va, na * 4, cudaMemcpyDeviceToDevice, s));
      }
    }
    if (nb) {
      BC_CUDA(cudaMemcpyAsync(state->beta_cur, pl.b_cur, nb * 4, cudaMemcpyDeviceToDevice, s));
      BC_CUDA(cudaMemcpyAsync(state->m_beta, pl.mb, nb * 4, cudaMemcpyDeviceToDevice, s));
      BC_CUDA(cudaMemcpyAsync(state->v_beta, pl.vb, nb * 4, cudaMemcpyDeviceToDevice, s));
    }
    BC_CUDA(cudaMemcpyAsync(state->best_lb, pl.best_lb, (size_t)R * 4, cudaMemcpyDeviceToDevice, s));
    state->t = t0 + cfg->iters;
  }
  BC_CHECK(run_bound(net, dom, batch, pl, cert ? BCROWN_CERTIFY : BCROWN_FP32, false, alpha, beta, lb_out, nullptr,
                     nullptr, s));
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

extern "C" int bcrown_root_bounds(bcrown_net* net, int n_props, const float* x_lo, const float* x_hi,
                                  int alpha_rule, float alpha_value, int precision, float* l, float* u,
                                  int32_t* unstable_count, void* stream) {
  if (!net || n_props < 1 || !x_lo || !x_hi || (net->H > 0 && (!l || !u)))
    return fail(BCROWN_ERR_ARG, "root_bounds: bad argument");
  if (alpha_rule != BCROWN_ALPHA_ADAPTIVE && alpha_rule != BCROWN_ALPHA_FIXED)
    return fail(BCROWN_ERR_ARG, "root_bounds: unknown alpha rule");
  if (precision != BCROWN_FP32 && precision != BCROWN_CERTIFY)
    return fail(BCROWN_ERR_ARG, "root_bounds: precision must be FP32 or CERTIFY");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  const bool cert = precision == BCROWN_CERTIFY;
  const int L = net->L;
  int maxrows = 2 * std::max(net->max_hidden, 1);
  Plan pl;
  BC_CHECK(make_plan(net, n_props, maxrows, cert, false, 0, 0, 0, pl));
  bcrown_domain dom{n_props, x_lo, x_hi, l, u};
  for (int top = 1; top <= L - 1; ++top) {
    // tables and |W| M terms of layers < top are complete once l, u of those layers are.
    build_tables(net, &dom, pl, s);
    if (cert) {
      long long hprev = top >= 2 ? net->hoff[top - 2] : -1;
      // wm of layers 1..top-1 (recomputed: cheap)
      for (int m = 1; m < top; ++m) {
        long long hp = m >= 2 ? net->hoff[m - 2] : -1;
        launch_absw_m(geom_of(net->ly[m - 1]), net->ly[m - 1].W, n_props, net->H, net->hoff[m - 1], hp, u, x_lo,
                      x_hi, net->d[0], pl.wm, s);
      }
      (void)hprev;
    }
    const int d_top = net->d[top];
    const int rows = 2 * d_top;
    for (int p = 0; p < n_props; ++p) {
      for (int q0 = 0; q0 < rows; q0 += pl.Rc) {
        int Rc = std::min(pl.Rc, rows - q0);
        launch_root_top(q0, Rc, d_top, net->ly[top - 1].b, pl.Lam, pl.cf, pl.cd, pl.E, s);
        contract_bwd(net, top, Rc, pl.Lam, pl.Abuf[top - 1], s);
        for (int m = top - 1; m >= 1; --m) {
          const LayerDev& ly = net->ly[m - 1];
          launch_relax_root(cert, Rc, p, net->H, net->d[m], net->hoff[m - 1], l, u, pl.tb, alpha_rule, alpha_value,
                            pl.Abuf[m], pl.Lam, ly.b, pl.cf, pl.cd, pl.E, pl.wm, gamma_n(ly.terms_bwd), s);
          contract_bwd(net, m, Rc, pl.Lam, pl.Abuf[m - 1], s);
        }
        launch_concretize_root(cert, q0, Rc, p, net->d[0], d_top, net->H, net->hoff[top - 1], x_lo, x_hi, pl.Abuf[0],
                               pl.cf, pl.cd, pl.E, l, u, s);
      }
    }
  }
  build_tables(net, &dom, pl, s);
  launch_copy_count(n_props, net->H, pl.U, unstable_count, s);
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

extern "C" int bcrown_neuron_codes(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                                   int8_t* codes, void* stream) {
  if (!net) return fail(BCROWN_ERR_ARG, "neuron_codes: null net");
  BC_CHECK(check_domain(net, dom));
  BC_CHECK(check_batch(batch));
  if (batch->B == 0 || net->H == 0) return BCROWN_OK;
  if (!codes) return fail(BCROWN_ERR_ARG, "neuron_codes: null output");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  Plan pl;
  int R = batch->B * net->K;
  BC_CHECK(make_plan(net, dom->n_props, R, false, false, 0, 0, 0, pl));
  build_tables(net, dom, pl, s);
  RowsCtx c = ctx_of(net, dom, batch, pl, 0, R);
  for (int i = 1; i < net->L; ++i) launch_codes(c, i, net->d[i], net->hoff[i - 1], net->H, codes, s);
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

extern "C" int bcrown_batch_split(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* parent,
                                  const uint8_t* pick_layer, const uint32_t* pick_idx, const float* alpha,
                                  const float* beta, int32_t* c_prop, int32_t* c_off, int32_t* c_cnt,
                                  uint8_t* c_layer, uint32_t* c_idx, int8_t* c_sign, int64_t* c_aoff,
                                  float* c_alpha, float* c_beta, void* stream) {
  if (!net) return fail(BCROWN_ERR_ARG, "batch_split: null net");
  BC_CHECK(check_domain(net, dom));
  BC_CHECK(check_batch(parent));
  if (parent->B == 0) return BCROWN_OK;
  if (!pick_layer || !pick_idx || !c_prop || !c_off || !c_cnt || !c_layer || !c_idx || !c_sign || !c_aoff)
    return fail(BCROWN_ERR_ARG, "batch_split: null output");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  Plan pl;
  BC_CHECK(make_plan(net, dom->n_props, 1, false, false, 0, 0, 0, pl));
  build_tables(net, dom, pl, s);
  launch_split(view_of(parent), net->K, pl.U, dom->n_props, pick_layer, pick_idx, alpha, beta, c_prop, c_off, c_cnt,
               c_aoff, c_layer, c_idx, c_sign, c_alpha, c_beta, net->status, s);
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

extern "C" int bcrown_bound_xstar(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                                  const float* alpha, const float* beta, float* lb, float* xstar, void* stream) {
  if (!net) return fail(BCROWN_ERR_ARG, "bound_xstar: null net");
  BC_CHECK(check_domain(net, dom));
  BC_CHECK(check_batch(batch));
  if (batch->B == 0) return BCROWN_OK;
  if (!lb || !xstar) return fail(BCROWN_ERR_ARG, "bound_xstar: null output");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  Plan pl;
  const int R = batch->B * net->K;
  BC_CHECK(make_plan(net, dom->n_props, R, false, false, 0, 0, 0, pl));
  build_tables(net, dom, pl, s);
  for (int r0 = 0; r0 < R; r0 += pl.Rc) {
    const int Rc = std::min(pl.Rc, R - r0);
    BC_CHECK(chunk_simt(net, dom, batch, pl, r0, Rc, false, false, alpha, beta, lb, nullptr, nullptr, s, false, xstar));
  }
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

extern "C" int bcrown_forward(bcrown_net* net, int n, const float* x, float* out, void* stream) {
  if (!net || n < 0) return fail(BCROWN_ERR_ARG, "forward: bad argument");
  if (n == 0) return BCROWN_OK;
  if (!x || !out) return fail(BCROWN_ERR_ARG, "forward: null pointer");
  std::lock_guard<std::mutex> g(net->mu);
  cudaStream_t s = (cudaStream_t)stream;
  Plan pl;
  BC_CHECK(make_plan(net, 1, n, false, false, 0, 0, 0, pl));
  const int L = net->L;
  for (int r0 = 0; r0 < n; r0 += pl.Rc) {
    const int Rc = std::min(pl.Rc, n - r0);
    const float* h = x + (size_t)r0 * net->d[0];
    float* z = pl.Z0;
    float* other = pl.Z1;
    for (int i = 1; i <= L - 1; ++i) {
      BC_CHECK(contract_fwd(net, i, Rc, h, z, s));
      launch_relu(z, (long long)Rc * net->d[i], s);
      h = z;
      std::swap(z, other);
    }
    launch_spec_out(Rc, net->K, net->d[L - 1], h, net->Wbar, net->bbar, out + (size_t)r0 * net->K, s);
  }
  BC_CUDA(cudaGetLastError());
  return BCROWN_OK;
}

// ---- launch configuration and the autotuner ----

static bool known_path(int path) { return path >= BCROWN_PATH_DEFAULT && path <= BCROWN_PATH_LAYER_IM2COL; }

extern "C" int bcrown_path_supported(bcrown_net* net, int path) {
  if (!net || !known_path(path) || path == BCROWN_PATH_DEFAULT) return 0;
  return path_ok(net, path) ? 1 : 0;
}

extern "C" int bcrown_set_launch(bcrown_net* net, const bcrown_launch_cfg* cfg) {
  if (!net || !cfg) return fail(BCROWN_ERR_ARG, "set_launch: null argument");
  if (!known_path(cfg->path) || cfg->grid_per_sm < 0 || cfg->grid_per_sm > 32)
    return fail(BCROWN_ERR_ARG, "set_launch: unknown path or grid_per_sm outside 0..32");
  if (cfg->path != BCROWN_PATH_DEFAULT && !path_ok(net, cfg->path))
    return fail(BCROWN_ERR_UNIMPLEMENTED, "set_launch: the net cannot take this path");
  std::lock_guard<std::mutex> g(net->mu);
  net->launch_set.path = cfg->path;
  net->launch_set.grid_per_sm = cfg->grid_per_sm;
  return BCROWN_OK;
}

extern "C" int bcrown_get_launch(bcrown_net* net, int rows, bcrown_launch_cfg* cfg) {
  if (!net || !cfg || rows < 0) return fail(BCROWN_ERR_ARG, "get_launch: bad argument");
  std::lock_guard<std::mutex> g(net->mu);
  const bcrown_net::Launch l = resolve_launch(net, std::max(rows, 1));
  cfg->path = l.path;
  cfg->grid_per_sm = l.grid_per_sm;
  return BCROWN_OK;
}

extern "C" int bcrown_autotune(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                               const float* alpha, const float* beta, int reps, bcrown_launch_cfg* cands,
                               double* ms, int max_cands, int* n_cands, bcrown_launch_cfg* best, void* stream) {
  if (!net || !batch || !best || reps < 1 || max_cands < 0) return fail(BCROWN_ERR_ARG, "autotune: bad argument");
  BC_CHECK(check_domain(net, dom));
  BC_CHECK(check_batch(batch));
  if (batch->B == 0) return fail(BCROWN_ERR_ARG, "autotune: empty batch");
  const long long R = (long long)batch->B * net->K;
  // candidates: every supported path; the layer GEMM paths with 1 and 2 CTAs per SM
  std::vector<bcrown_net::Launch> cand;
  for (int p : {BCROWN_PATH_FUSED, BCROWN_PATH_LAYER_EPI, BCROWN_PATH_LAYER_GATHER, BCROWN_PATH_LAYER_IM2COL}) {
    if (!path_ok(net, p)) continue;
    const bool grid = p == BCROWN_PATH_LAYER_GATHER || p == BCROWN_PATH_LAYER_IM2COL;
    for (int g : grid ? std::vector<int>{1, 2} : std::vector<int>{0}) {
      bcrown_net::Launch l;
      l.path = p;
      l.grid_per_sm = g;
      cand.push_back(l);
    }
  }
  if (cand.empty()) return fail(BCROWN_ERR_UNIMPLEMENTED, "autotune: the net takes no BF16 path");
  cudaStream_t s = (cudaStream_t)stream;
  float *lb = nullptr, *da = nullptr, *dbt = nullptr;
  BC_CUDA(cudaMalloc(&lb, (size_t)R * 4));
  if (cudaMalloc(&da, std::max<size_t>(batch->n_alpha, 1) * 4) != cudaSuccess ||
      cudaMalloc(&dbt, std::max<size_t>(batch->n_beta, 1) * 4) != cudaSuccess) {
    cudaFree(lb);
    cudaFree(da);
    return fail(BCROWN_ERR_OOM, "autotune: outputs");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const bcrown_net::Launch saved = net->launch_set;
  std::vector<double> t(cand.size(), 0.0);
  int rc = BCROWN_OK;
  for (size_t c = 0; c < cand.size() && rc == BCROWN_OK; ++c) {
    {
      std::lock_guard<std::mutex> g(net->mu);
      net->launch_set = cand[c];
      // the tuner's earlier choice for this bucket would take precedence: drop it while timing
      const int bk = bucket_of(R);
      net->tuned.erase(std::remove_if(net->tuned.begin(), net->tuned.end(),
                                      [bk](const std::pair<int, bcrown_net::Launch>& x) { return x.first == bk; }),
                       net->tuned.end());
    }
    rc = bcrown_bound_grad(net, dom, batch, alpha, beta, BCROWN_BF16, lb, da, dbt, stream);   // untimed
    if (rc != BCROWN_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && rc == BCROWN_OK; ++r)
      rc = bcrown_bound_grad(net, dom, batch, alpha, beta, BCROWN_BF16, lb, da, dbt, stream);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(BCROWN_ERR_CUDA, "autotune: timing");
    float el = 0.f;
    cudaEventElapsedTime(&el, e0, e1);
    t[c] = (double)el / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(lb);
  cudaFree(da);
  cudaFree(dbt);
  std::lock_guard<std::mutex> g(net->mu);
  net->launch_set = saved;
  if (rc != BCROWN_OK) return rc;
  size_t bi = 0;
  for (size_t c = 1; c < cand.size(); ++c)
    if (t[c] < t[bi]) bi = c;
  net->tuned.emplace_back(bucket_of(R), cand[bi]);
  best->path = cand[bi].path;
  best->grid_per_sm = cand[bi].grid_per_sm;
  for (size_t c = 0; c < cand.size() && (int)c < max_cands; ++c) {
    if (cands) {
      cands[c].path = cand[c].path;
      cands[c].grid_per_sm = cand[c].grid_per_sm;
    }
    if (ms) ms[c] = t[c];
  }
  if (n_cands) *n_cands = (int)cand.size();
  return BCROWN_OK;
}
