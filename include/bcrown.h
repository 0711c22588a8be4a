/*
 * bcrown.h -- C ABI of the GB300 batched beta-CROWN bound library.
 *
 * The library computes, for a ReLU network f, an input box [x_lo, x_hi] and
 * linear specifications c_k, a sound lower bound of c_k^T f(x) on many
 * branch-and-bound subdomains at once (Wang et al., arXiv 2103.06624,
 * Theorem 3.1 and Eq. beta_crown_lp), its gradient with respect to the
 * relaxation slopes alpha and the split multipliers beta, and the projected
 * Adam ascent on (alpha, beta) of Eq. opt_alpha_beta (Appendix C.1).
 *
 * Conventions shared by every call:
 *  - Status codes are returned (BCROWN_OK = 0, negative on error); no C++
 *    exception crosses this boundary.  bcrown_last_error() gives a message for
 *    the calling thread's last failure.
 *  - bcrown_load_net copies host data.  Every other array argument is a
 *    caller-owned DEVICE pointer; the call enqueues its kernels on `stream`
 *    (a cudaStream_t passed as void*) and returns without synchronising.
 *    Outputs are complete once the stream reaches that point.
 *  - Problems that only the device can see (a split index out of range, a
 *    non-finite bound, a wait that ran out of time) are recorded in a device
 *    status word of the net; bcrown_status() synchronises the stream, returns
 *    that code and clears it.  A row whose bound is not finite gets -inf,
 *    which is sound, and sets BCROWN_ERR_NONFINITE; the other rows are written.
 *  - Calls on one net share the net's device workspace, so calls on the same
 *    net issued to different streams must not overlap.
 *
 * Index conventions (paper notation): layers i = 1..L are the linear layers;
 * hidden layers are i = 1..L-1 with d_i neurons (for a convolution, flattened
 * channel-major: c*H*W + y*W + x).  A property's hidden neurons are numbered
 * layer-major, H = d_1 + ... + d_{L-1}.  Row r = b*K + k is subdomain b under
 * spec k.
 */
#ifndef BCROWN_H
#define BCROWN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bcrown_net bcrown_net; /* opaque, library-owned */

enum {
  BCROWN_OK = 0,
  BCROWN_ERR_ARG = -1,
  BCROWN_ERR_OOM = -2,
  BCROWN_ERR_CUDA = -3,
  BCROWN_ERR_TIMEOUT = -4,
  BCROWN_ERR_NONFINITE = -5,
  BCROWN_ERR_UNIMPLEMENTED = -6
};

enum { BCROWN_LAYER_FC = 0, BCROWN_LAYER_CONV = 1 };

/* Arithmetic of a bound pass.
 *  FP32    : FP32 coefficients and products, FP32 accumulation.
 *  BF16    : A.W contractions with BF16 operands and FP32 accumulation on the
 *            tensor cores; everything else FP32.  Fully connected networks (hidden
 *            widths <= 256, at most 1536 hidden neurons, input <= 1024) run one fused
 *            kernel per call; other networks (conv layers of <= 256 channels with
 *            channels x taps <= 2048, fc layers of <= 65536 neurons) run every
 *            contraction as a tensor-core GEMM (conv layers over an im2col operand,
 *            transposed convolutions split into stride phases; the operand gathered
 *            in shared memory, or written to an HBM buffer first when the environment
 *            holds BCROWN_CONV_IM2COL=1 at library load, for comparison) and the
 *            relaxation in FP32.  Any alpha, beta gives a valid bound (Section 3.1), so this is used
 *            for the optimisation iterations.  Other networks get
 *            BCROWN_ERR_UNIMPLEMENTED.
 *  CERTIFY : FP32 contractions plus a priori rounding-error terms, upper-chord
 *            constants rounded outward and sums rounded down (error terms rounded
 *            up); the result is a lower bound of the exact-arithmetic bound at the
 *            same alpha, beta. */
enum { BCROWN_FP32 = 0, BCROWN_BF16 = 1, BCROWN_CERTIFY = 2 };

/* Lower slope rule for root (intermediate) bounds: ADAPTIVE takes alpha' = 1
 * where u >= -l else 0; FIXED takes alpha' = alpha_value. */
enum { BCROWN_ALPHA_ADAPTIVE = 0, BCROWN_ALPHA_FIXED = 1 };

/* Largest split list one subdomain may carry. */
#define BCROWN_MAX_SPLITS 64

/* One linear layer of Eq. 1, z^(i) = W^(i) h^(i-1) + b^(i); ReLU follows every
 * layer but the last.  Host pointers, copied by bcrown_load_net.
 *  fc  : in_c = d_{i-1}, out_c = d_i, the h/w fields 1; W [out_c][in_c] row-major.
 *  conv: W [out_c][in_c][k][k]; out_h = (in_h + 2 pad - k)/stride + 1 (same for w);
 *        b has out_c entries (one per channel). */
typedef struct {
  int kind;
  int in_c, in_h, in_w;
  int out_c, out_h, out_w;
  int k, stride, pad;
  const float* W;
  const float* b;
} bcrown_layer;

/* Build a network from n_layers layers and a spec matrix C [K][d_L] (host,
 * row-major).  The spec is merged into the last layer (Section 2.1):
 * Wbar = C W^(L), bbar = C b^(L).  The last layer must be fully connected.
 * Returns BCROWN_ERR_ARG on inconsistent shapes, BCROWN_ERR_OOM/CUDA on
 * device failures; *out is set only on success. */
int bcrown_load_net(const bcrown_layer* layers, int n_layers, const float* C, int K,
                    bcrown_net** out);

void bcrown_free_net(bcrown_net* net);

/* Widths d_0..d_L (widths must hold n_layers+1 ints; either pointer may be NULL). */
int bcrown_net_info(const bcrown_net* net, int* n_layers, int* widths, int* K);

/* The properties a batch refers to: input boxes and root intermediate bounds.
 * Device pointers, caller-owned, read during the calls that take them. */
typedef struct {
  int n_props;
  const float* x_lo; /* [P][d_0] */
  const float* x_hi; /* [P][d_0] */
  const float* l;    /* [P][H] pre-activation lower bounds (Section 2.1) */
  const float* u;    /* [P][H] pre-activation upper bounds */
} bcrown_domain;

/* Root intermediate bounds (Section 3.3; CROWN, Lemma 2.2, with alpha' fixed by
 * the rule and beta' = 0): for every hidden neuron, l and u of z^(i)_j over the
 * box.  Layer 1 is the exact interval; layer i >= 2 bounds +-z^(i)_j by back-
 * substitution through layers i-1..1.  With precision BCROWN_CERTIFY the bounds
 * are computed with outward rounding (sound in floating point), else in FP32.
 * Outputs: l, u [P][H]; unstable_count [P] (number of l < 0 < u), device. */
int bcrown_root_bounds(bcrown_net* net, int n_props, const float* x_lo, const float* x_hi,
                       int alpha_rule, float alpha_value, int precision,
                       float* l, float* u, int32_t* unstable_count, void* stream);

/* A batch of subdomains (Section 2.3 split sets; Eq. 3 encoding).  Device
 * pointers, caller-owned.
 *  prop_of[b]      property of subdomain b
 *  split_off[b], split_cnt[b]  its splits are entries split_off..+cnt-1 of:
 *  split_layer[s]  hidden layer i in 1..L-1
 *  split_idx[s]    neuron index j in layer i
 *  split_sign[s]   S^(i)_jj: -1 for the split z >= 0, +1 for z < 0
 *  alpha_off[b]    alpha of row (b,k) for the property's t-th unstable neuron
 *                  (layer-major order of l < 0 < u) is alpha[alpha_off[b] + k*U_p + t]
 * beta of split t of subdomain b under spec k is beta[split_off[b]*K + k*split_cnt[b] + t].
 * n_alpha, n_beta: total lengths of the alpha and beta arrays. */
typedef struct {
  int B;
  const int32_t* prop_of;
  const int32_t* split_off;
  const int32_t* split_cnt;
  const uint8_t* split_layer;
  const uint32_t* split_idx;
  const int8_t* split_sign;
  const int64_t* alpha_off;
  int64_t n_alpha;
  int64_t n_beta;
} bcrown_batch;

/* Lower bound of every row at fixed alpha, beta (Theorem 3.1):
 *   A^(L-1) = Wbar_k, c = bbar_k; for i = L-1..1:
 *   Lambda = A D + beta^T S; c += Lambda b + A lambda; A^(i-1) = Lambda W^(i);
 *   lb = c + sum_m min(A^(0)_m x_lo_m, A^(0)_m x_hi_m).
 * D, lambda follow Eq. definition_D / definition_lowerb with split overriding
 * stability.  alpha [n_alpha], beta [n_beta] device; lb [B*K] device output. */
int bcrown_bound(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                 const float* alpha, const float* beta, int precision, float* lb, void* stream);

/* lb and its gradient: dalpha[t] = A^(i)_j zhat^(i)_j where alpha_j is the slope
 * in use (unstable, unsplit, A_j >= 0), else 0; dbeta = S_jj zhat^(i)_j, with
 * zhat the pre-activations along x* (x_lo where A^(0)_m >= 0, else x_hi) pushed
 * through the relaxed network.  Shapes as alpha/beta.  precision FP32 or BF16. */
int bcrown_bound_grad(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                      const float* alpha, const float* beta, int precision,
                      float* lb, float* dalpha, float* dbeta, void* stream);

/* Projected Adam ascent (Eq. opt_alpha_beta; Appendix C.1: 20 iterations, lr
 * 0.1 for alpha and 0.05 for beta, decayed by 0.98 per iteration).  Iteration t
 * evaluates lb and its gradient at theta_t with `precision`, keeps per row the
 * best lb and its theta, then steps uphill with lr0*decay^t, Adam moments
 * (beta1, beta2, eps) with bias correction, and clamps alpha to [0,1], beta to
 * >= 0.  At the end one BCROWN_CERTIFY pass (if certify != 0, else FP32) at the
 * best theta writes lb_out [B*K].  alpha, beta: in = initial values (or, when
 * resuming, the best theta so far), out = best. */
typedef struct {
  int iters;
  float lr_alpha, lr_beta, decay;
  float adam_beta1, adam_beta2, adam_eps;
  int precision; /* of the iterations: BCROWN_FP32 or BCROWN_BF16 */
  int certify;   /* final pass: nonzero = BCROWN_CERTIFY, 0 = FP32 */
  int freeze;    /* BCROWN_FREEZE_* bits: groups held at their inputs (Table A4's ablations):
                    bcrown_optimize steps them with a zero learning rate (entries inside their
                    boxes stay bit for bit), bcrown_optimize_joint does not step them */
} bcrown_opt_cfg;

#define BCROWN_FREEZE_ALPHA 1 /* alpha (and alpha' of bcrown_optimize_joint): the beta-only ablation */
#define BCROWN_FREEZE_BETA 2  /* beta (and beta'): the alpha-only ablation */

/* Optimiser state, for continuing an ascent across calls (checkpoint / resume, or a caller
 * that keeps stepping the same batch).  Caller-owned FP32 device arrays in the batch's alpha
 * and beta layouts, plus a host iteration counter:
 *   alpha_cur [n_alpha], beta_cur [n_beta]   the current iterate theta_t (the next point evaluated)
 *   m_alpha, v_alpha [n_alpha]; m_beta, v_beta [n_beta]   Adam's first and second moments
 *   best_lb [B*K]                            best lb seen per row (-inf before any iteration)
 *   t                                        iterations taken so far
 * With t == 0 on entry the arrays are not read: the ascent starts at alpha, beta with zero
 * moments.  With t > 0 they are read, alpha and beta must hold the best theta so far, and the
 * learning rate and bias corrections continue from iteration t.  On return every array holds
 * the state after the call and t has grown by cfg->iters.  The BF16 precision keeps alpha's
 * moments in BF16 inside a call (they are rounded to BF16 on entry and widened on return), so
 * a run split into several calls reproduces an uninterrupted run bit for bit in both precisions. */
typedef struct {
  float* alpha_cur;
  float* beta_cur;
  float* m_alpha;
  float* v_alpha;
  float* m_beta;
  float* v_beta;
  float* best_lb;
  int t;
} bcrown_opt_state;

/* state may be NULL (a fresh ascent whose state is discarded). */
int bcrown_optimize(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                    const bcrown_opt_cfg* cfg, float* alpha, float* beta, float* lb_out,
                    bcrown_opt_state* state, void* stream);

/* batch_split of Algorithm 1: parent b splits neuron (pick_layer[b], pick_idx[b]).
 * Child 2b is C^l (z >= 0, S = -1), child 2b+1 is C^u (z < 0, S = +1).  Each
 * child carries the parent's splits followed by the new one, a copy of the
 * parent's alpha block and the parent's beta with 0 for the new split.
 * Outputs (device, caller-allocated for 2B children): prop_of, split_off,
 * split_cnt [2B]; split_layer, split_idx, split_sign [2*(S_parent + B)];
 * alpha_off [2B] (packed in child order); alpha [2*n_alpha];
 * beta [2*(n_beta + B*K)].  child_* pointers describe the result. */
int bcrown_batch_split(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* parent,
                       const uint8_t* pick_layer, const uint32_t* pick_idx,
                       const float* alpha, const float* beta,
                       int32_t* child_prop_of, int32_t* child_split_off, int32_t* child_split_cnt,
                       uint8_t* child_split_layer, uint32_t* child_split_idx, int8_t* child_split_sign,
                       int64_t* child_alpha_off, float* child_alpha, float* child_beta,
                       void* stream);

/* The bound of bcrown_bound (FP32) and, per row, the point x* of the box that minimises the
 * row's linear bound over it (Theorem 3.1: x_lo where A^(0)_m >= 0, else x_hi).  Evaluating
 * the network there gives an upper bound of the row's minimum over the box (Appendix B.1,
 * Algorithm 1's upper bound f(x*)).  lb [B*K], xstar [B*K][d_0] device outputs. */
int bcrown_bound_xstar(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                       const float* alpha, const float* beta, float* lb, float* xstar, void* stream);

/* The network itself with the specifications merged (Eq. 1, Section 2.1): out[r][k] =
 * c_k^T f(x_r) for n inputs x [n][d_0] (device), FP32; out [n][K] device. */
int bcrown_forward(bcrown_net* net, int n, const float* x, float* out, void* stream);

/* Per (row, hidden neuron) relaxation code as the kernels use it: 0 inactive
 * (u <= 0), 1 active (l >= 0), 2 unstable, 3 split z >= 0, 4 split z < 0
 * (split overrides stability).  codes: device [B*K][H] int8. */
int bcrown_neuron_codes(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                        int8_t* codes, void* stream);

/* Timing hook.  With enable != 0 the library records a CUDA event pair on the
 * launching stream around each of its kernels of the classes below; enable = 0
 * stops recording.  Either call discards earlier records.  bcrown_profile_read
 * waits for the recorded events and returns the summed device milliseconds and
 * the launch count of one class.  Calls enqueued while the stream is being captured
 * into a CUDA graph record their pairs as event nodes of the graph: after replays,
 * the read gives the latest replay's times (the pairs stay valid while the net lives). */
enum {
  BCROWN_PROF_CONTRACT = 0,   /* A.W contractions (dense or convolution), both directions */
  BCROWN_PROF_RELAX = 1,      /* relaxation + beta + bias epilogue */
  BCROWN_PROF_CONCRETIZE = 2, /* concretisation over the box */
  BCROWN_PROF_ADJOINT = 3,    /* adjoint epilogue (gradients) */
  BCROWN_PROF_ADAM = 4,       /* projected Adam */
  BCROWN_PROF_FUSED = 5,      /* fused tensor-core iteration kernel */
  BCROWN_PROF_LAYER_GEMM = 6, /* tensor-core GEMMs of the BF16 layer paths (LAYER_EPI: with the fused epilogues) */
  BCROWN_PROF_NCLASS = 7
};
int bcrown_profile(bcrown_net* net, int enable);
int bcrown_profile_read(bcrown_net* net, int cls, double* total_ms, long long* launches);

/* Number of kernels this library has launched in the process so far (all nets). */
long long bcrown_kernel_launches(void);

/* Peak-rate probe for the rooflines of the SIMT kernels (not part of the method): kind 0 runs
 * independent FP32 FFMA chains, kind 1 FP64 DFMA chains, in 8 blocks of 256 threads per SM for
 * `iters` x 128 FMAs per thread; the launch is timed with CUDA events on `stream` (the call
 * synchronises it) and *tflops receives the measured rate, 2 flops per FMA. */
int bcrown_peak_probe(int kind, int iters, double* tflops, void* stream);

/* ---- Joint optimisation of intermediate-layer bounds (Section 3.3, Eq. opt_non_convex) ----
 *
 * Fully connected networks (BCROWN_ERR_UNIMPLEMENTED otherwise), FP32.  Per subdomain, the
 * bounds l^(T), u^(T) of every hidden layer T = 2..L-1 are recomputed by the bound of Theorem
 * 3.1 with the objective z^(T)_j (for l) and -z^(T)_j (for u = -bound), from the subdomain's
 * bounds of layers 1..T-1 (layer 1: the domain's), its split constraints and free variables
 * alpha' in [0,1], beta' >= 0 shared by all target neurons of layer T (the O(L^2 d) variant);
 * each is intersected with the domain's bound (both are valid on the subdomain).  The rows'
 * bounds then use these l, u.  A neuron the tighter bounds make stable takes D = 1 or 0; its
 * alpha entries stay in the layout.
 *
 * Layout of alpha' (subdomain b of property p, first[p][T] = the domain-unstable neurons of p
 * in layers 1..T-1, rank = a neuron's rank among p's unstable neurons in layer-major order):
 * subdomain b's block starts after the earlier subdomains' blocks (2 sum_{T=2}^{L-1}
 * first[p][T] entries each); inside it, target layers T = 2..L-1 in order, for each the lower
 * direction (dir 0) then the upper (dir 1), first[p][T] entries indexed by rank.  beta' of
 * (b, T, dir) holds split_cnt[b] entries at 2 (L-2) split_off[b] + (2 (T-2) + dir) split_cnt[b]
 * indexed by the split's position in b's list (entries of splits in layers >= T are unused).
 * alpha, beta as in bcrown_bound.  All arrays are device memory; n_alpha_p, n_beta_p are the
 * caller's array lengths (indices beyond them set BCROWN_ERR_ARG in the status word). */

/* The lengths of alpha' and beta' for the batch (synchronises the stream). */
int bcrown_joint_sizes(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                       int64_t* n_alpha_p, int64_t* n_beta_p, void* stream);

/* alpha' at the rule the root bounds use (1 where u >= -l, else 0, per source neuron), so that
 * with beta' = 0 and no split the recomputed bounds are the domain's. */
int bcrown_joint_init_alpha(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                            float* alpha_p, int64_t n_alpha_p, void* stream);

/* The bound of every row (lb [B*K]) with the recomputed intermediate bounds, which are written
 * to l_out, u_out [B][H] (either may be NULL). */
int bcrown_bound_joint(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                       const float* alpha, const float* beta, const float* alpha_p, int64_t n_alpha_p,
                       const float* beta_p, int64_t n_beta_p, float* lb, float* l_out, float* u_out,
                       void* stream);

/* lb and the gradient of the sum of all rows' bounds with respect to alpha, beta, alpha' and
 * beta' (the adjoint of each pass, chained through the recomputed bounds). */
int bcrown_bound_joint_grad(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                            const float* alpha, const float* beta, const float* alpha_p, int64_t n_alpha_p,
                            const float* beta_p, int64_t n_beta_p, float* lb, float* dalpha, float* dbeta,
                            float* dalpha_p, float* dbeta_p, void* stream);

/* Projected Adam on (alpha, beta, alpha', beta') with cfg's iterations, learning rates (alpha'
 * at lr_alpha, beta' at lr_beta), decay and freeze bits; cfg->precision must be BCROWN_FP32 and
 * cfg->certify 0.  Per subdomain, the iterate with the largest sum of its spec bounds is kept
 * (the intermediate bounds belong to the subdomain); on return alpha .. beta_p hold it, lb_out
 * its bounds and l_out, u_out (may be NULL) its intermediate bounds.  Allocates its optimiser
 * state with cudaMalloc and synchronises the stream. */
int bcrown_optimize_joint(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                          const bcrown_opt_cfg* cfg, float* alpha, float* beta, float* alpha_p, int64_t n_alpha_p,
                          float* beta_p, int64_t n_beta_p, float* lb_out, float* l_out, float* u_out,
                          void* stream);

/* ---- BF16 launch configuration and its tuner (the paper has no counterpart: these choose
 * among this library's own kernels for the same computation) ----
 *
 * The BF16 precision of bcrown_bound, bcrown_bound_grad and bcrown_optimize can run the bound
 * pass (Theorem 3.1) and its adjoint on one of these paths; they compute the same quantities
 * and differ only in rounding order and speed:
 *   BCROWN_PATH_FUSED         fully connected nets up to the fused kernel's limits: the whole
 *                             backward recursion and adjoint of a 64-row tile in one persistent
 *                             tcgen05 kernel
 *   BCROWN_PATH_LAYER_EPI     layer by layer: one tcgen05 GEMM per contraction (conv operands
 *                             gathered in shared memory), the relaxation, beta shift, bias sums,
 *                             concretisation and adjoint applied in the GEMM's epilogue
 *   BCROWN_PATH_LAYER_GATHER  layer by layer: tcgen05 GEMMs (conv operands gathered in shared
 *                             memory), FP32 CUDA-core kernels for the steps between them
 *   BCROWN_PATH_LAYER_IM2COL  as LAYER_GATHER with the conv operands written to an im2col
 *                             buffer in HBM and read by TMA
 * grid_per_sm: persistent CTAs per SM for the LAYER_GATHER / LAYER_IM2COL GEMMs (0 = 2); the
 * other paths run one CTA per SM and ignore it. */
#define BCROWN_PATH_DEFAULT 0
#define BCROWN_PATH_FUSED 1
#define BCROWN_PATH_LAYER_EPI 2
#define BCROWN_PATH_LAYER_GATHER 3
#define BCROWN_PATH_LAYER_IM2COL 4

typedef struct {
  int path;        /* BCROWN_PATH_*; DEFAULT = the first supported of FUSED, LAYER_EPI, LAYER_GATHER */
  int grid_per_sm; /* 0 = the path's default */
} bcrown_launch_cfg;

/* 1 if the net can take `path` on this device, else 0 (unknown paths: 0). */
int bcrown_path_supported(bcrown_net* net, int path);

/* The configuration used from now on for every row count the tuner has no choice for.
 * BCROWN_ERR_ARG for an unknown path, BCROWN_ERR_UNIMPLEMENTED for one the net cannot take. */
int bcrown_set_launch(bcrown_net* net, const bcrown_launch_cfg* cfg);

/* The configuration a BF16 call with `rows` rows (subdomains x specs) takes: the tuner's choice
 * for rows' bucket, else the one set, else the built-in order (path resolved, never DEFAULT). */
int bcrown_get_launch(bcrown_net* net, int rows, bcrown_launch_cfg* cfg);

/* Autotuner: times every supported configuration on the caller's batch and keeps the fastest
 * for the batch's row-count bucket (rows rounded up to a power of two), which every later BF16
 * call with rows in that bucket takes.  Each candidate runs bcrown_bound_grad (BCROWN_BF16) at
 * `alpha`, `beta` (device, the batch's layouts) once untimed, then `reps` >= 1 times timed with
 * CUDA events on `stream`; the call synchronises the stream and allocates (then frees) its own
 * device outputs.  cands / ms (host, max_cands entries each, either may be NULL) receive the
 * candidates and their mean milliseconds per call; *n_cands their count; *best the choice.
 * Errors of a candidate end the call with that error. */
int bcrown_autotune(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                    const float* alpha, const float* beta, int reps, bcrown_launch_cfg* cands, double* ms,
                    int max_cands, int* n_cands, bcrown_launch_cfg* best, void* stream);

/* Size in bytes of the fixed device scratch of bcrown_bound_static (set when the library is built). */
#define BCROWN_STATIC_SCRATCH_BYTES (16u << 20)

/* bcrown_bound_static -- the FP32 bound pass of bcrown_bound (BCROWN_FP32), for callers that
 * cannot allocate device memory.  The paper has no counterpart: this entry point exists for
 * hosts that must not call cudaMalloc while the pass runs -- a real-time loop that cannot take
 * cudaMalloc's implicit synchronisation, a process confined to a device-memory budget handed
 * out by its own allocator.
 *
 * It allocates nothing.  Its scratch (per-neuron tables and row-chunk buffers) is one
 * file-scope device array of BCROWN_STATIC_SCRATCH_BYTES bytes that every GPU loading the
 * library holds until the process exits.  The caller passes inputs and outputs exactly as for
 * bcrown_bound.  The first call on a device looks the array's device address up (once per
 * device, with that device current); make that first call before any stream capture begins.
 * Problems whose per-property tables and a single row do not fit in the array are rejected
 * with BCROWN_ERR_ARG and a message naming the limit; larger batches are processed in row
 * chunks that fit.  Every call shares the one array and it keeps the last call's contents
 * (each call writes every part of it that it reads, so nothing needs clearing): calls that
 * overlap on the GPU -- on different streams, or from different host threads, on any net --
 * race.  Like the other entry points it takes the net's lock while it enqueues.  Its kernels
 * are left out of bcrown_profile's totals (recording them could create CUDA events). */
int bcrown_bound_static(bcrown_net* net, const bcrown_domain* dom, const bcrown_batch* batch,
                        const float* alpha, const float* beta, float* lb, void* stream);

/* The net's device workspace, which every call reuses (it grows when a call needs more; the
 * growth synchronises the device and reallocates it): grows it to at least reserve_bytes (0:
 * leaves it), then reports its address and size in *ptr, *bytes (either may be NULL).  A CUDA
 * graph captured from calls on this net refers to the workspace: it stays valid while the
 * address reported here is unchanged. */
int bcrown_workspace(bcrown_net* net, int64_t reserve_bytes, void** ptr, int64_t* bytes);

/* Synchronise `stream`, return the device status word of the net (BCROWN_OK or
 * the first device-detected error since the last call) and clear it. */
int bcrown_status(bcrown_net* net, void* stream);

/* Message of the calling thread's last error (static storage, never NULL). */
const char* bcrown_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BCROWN_H */
