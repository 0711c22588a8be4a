"""Python binding of the C ABI (include/bcrown.h), same names, torch tensors for memory and streams.

Every computation runs in the native library's CUDA kernels; this module only
marshals arguments (device pointers of contiguous CUDA tensors and the current
stream).  Calls are asynchronous on the current stream, like the C ABI.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import native as N

FP32, BF16, CERTIFY = N.FP32, N.BF16, N.CERTIFY
ALPHA_ADAPTIVE, ALPHA_FIXED = N.ALPHA_ADAPTIVE, N.ALPHA_FIXED
BcrownError = N.BcrownError


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return C.c_void_p(t.data_ptr()) if t.numel() else None


def _dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


class Net:
    """A loaded network (bcrown_load_net); the spec matrix C is merged into the last layer."""

    def __init__(self, layers, C_spec):
        lib = N.load()
        keep = []
        arr = (N.Layer * len(layers))()
        for i, ly in enumerate(layers):
            W = np.ascontiguousarray(ly.W, np.float32)
            b = np.ascontiguousarray(ly.b, np.float32)
            keep += [W, b]
            if ly.kind == "fc":
                arr[i] = N.Layer(N.LAYER_FC, ly.d_in, 1, 1, ly.d_out, 1, 1, 1, 1, 0,
                                 W.ctypes.data, b.ctypes.data)
            else:
                ci, h, w = ly.in_shape
                co, ho, wo = ly.out_shape
                arr[i] = N.Layer(N.LAYER_CONV, ci, h, w, co, ho, wo, ly.k, ly.stride, ly.pad,
                                 W.ctypes.data, b.ctypes.data)
        Cs = np.ascontiguousarray(C_spec, np.float32)
        h = C.c_void_p()
        N.check(lib.bcrown_load_net(arr, len(layers), Cs.ctypes.data, Cs.shape[0], C.byref(h)))
        self._h = h
        self.L = len(layers)
        self.K = int(Cs.shape[0])
        self.widths = [layers[0].d_in] + [ly.d_out for ly in layers]
        self.hidden_widths = self.widths[1:self.L]
        self.H = int(sum(self.hidden_widths))
        self.d0 = int(self.widths[0])

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            N.load().bcrown_free_net(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Domain:
    """Input boxes and root intermediate bounds of the properties (device tensors)."""
    x_lo: torch.Tensor
    x_hi: torch.Tensor
    l: torch.Tensor
    u: torch.Tensor

    @property
    def n_props(self):
        return int(self.x_lo.shape[0])

    def c(self):
        return N.Domain(self.n_props, _ptr(self.x_lo), _ptr(self.x_hi), _ptr(self.l), _ptr(self.u))


@dataclass
class DeviceBatch:
    """A batch of subdomains in the C-ABI layout, on the device."""
    prop_of: torch.Tensor
    split_off: torch.Tensor
    split_cnt: torch.Tensor
    split_layer: torch.Tensor
    split_idx: torch.Tensor
    split_sign: torch.Tensor
    alpha_off: torch.Tensor
    n_alpha: int
    n_beta: int

    @property
    def B(self):
        return int(self.prop_of.shape[0])

    @staticmethod
    def from_host(b):
        return DeviceBatch(_dev(b.prop_of, torch.int32), _dev(b.split_off, torch.int32),
                           _dev(b.split_cnt, torch.int32), _dev(b.split_layer, torch.uint8),
                           _dev(np.asarray(b.split_idx).astype(np.int64), torch.int64).to(torch.int32),
                           _dev(b.split_sign, torch.int8), _dev(b.alpha_off, torch.int64),
                           int(b.n_alpha), int(b.n_beta))

    def c(self):
        return N.Batch(self.B, _ptr(self.prop_of), _ptr(self.split_off), _ptr(self.split_cnt),
                       _ptr(self.split_layer), _ptr(self.split_idx), _ptr(self.split_sign),
                       _ptr(self.alpha_off), self.n_alpha, self.n_beta)


def domain_from_host(x_lo, x_hi, l, u):
    return Domain(_dev(x_lo, torch.float32), _dev(x_hi, torch.float32), _dev(l, torch.float32),
                  _dev(u, torch.float32))


def load_net(layers, C_spec):
    return Net(layers, C_spec)


def root_bounds(net, x_lo, x_hi, alpha_rule=ALPHA_ADAPTIVE, alpha_value=0.5, precision=CERTIFY, stream=None):
    """CROWN root bounds l, u [P, H] and the unstable count per property (device tensors)."""
    lib = N.load()
    P = int(x_lo.shape[0])
    l = torch.empty((P, net.H), device="cuda", dtype=torch.float32)
    u = torch.empty((P, net.H), device="cuda", dtype=torch.float32)
    cnt = torch.empty(P, device="cuda", dtype=torch.int32)
    N.check(lib.bcrown_root_bounds(net.handle, P, _ptr(x_lo), _ptr(x_hi), alpha_rule, float(alpha_value),
                                   precision, _ptr(l), _ptr(u), _ptr(cnt), _stream(stream)))
    return l, u, cnt


def bound(net, dom, batch, alpha, beta, precision=FP32, out=None, stream=None):
    lib = N.load()
    lb = out if out is not None else torch.empty(batch.B * net.K, device="cuda", dtype=torch.float32)
    d, b = dom.c(), batch.c()
    N.check(lib.bcrown_bound(net.handle, C.byref(d), C.byref(b), _ptr(alpha), _ptr(beta), precision,
                             _ptr(lb), _stream(stream)))
    return lb


def bound_static(net, dom, batch, alpha, beta, out=None, stream=None):
    """FP32 bound through bcrown_bound_static: no device allocation by the library (its scratch
    is a fixed array built into the library), for callers that cannot allocate."""
    lib = N.load()
    lb = out if out is not None else torch.empty(batch.B * net.K, device="cuda", dtype=torch.float32)
    d, b = dom.c(), batch.c()
    N.check(lib.bcrown_bound_static(net.handle, C.byref(d), C.byref(b), _ptr(alpha), _ptr(beta), _ptr(lb),
                                    _stream(stream)))
    return lb


def bound_grad(net, dom, batch, alpha, beta, precision=FP32, stream=None):
    lib = N.load()
    lb = torch.empty(batch.B * net.K, device="cuda", dtype=torch.float32)
    da = torch.empty(max(batch.n_alpha, 0), device="cuda", dtype=torch.float32)
    db = torch.empty(max(batch.n_beta, 0), device="cuda", dtype=torch.float32)
    d, b = dom.c(), batch.c()
    N.check(lib.bcrown_bound_grad(net.handle, C.byref(d), C.byref(b), _ptr(alpha), _ptr(beta), precision,
                                  _ptr(lb), _ptr(da), _ptr(db), _stream(stream)))
    return lb, da, db


@dataclass
class OptCfg:
    """Projected Adam settings; defaults from Appendix C.1 (20 iterations, lr 0.1/0.05, decay 0.98)."""
    iters: int = 20
    lr_alpha: float = 0.1
    lr_beta: float = 0.05
    decay: float = 0.98
    adam_beta1: float = 0.9
    adam_beta2: float = 0.999
    adam_eps: float = 1e-8
    precision: int = FP32
    certify: bool = True
    freeze_alpha: bool = False   # the beta-only ablation (Table A4)
    freeze_beta: bool = False    # the alpha-only ablation

    def c(self):
        fr = (N.FREEZE_ALPHA if self.freeze_alpha else 0) | (N.FREEZE_BETA if self.freeze_beta else 0)
        return N.OptCfg(self.iters, self.lr_alpha, self.lr_beta, self.decay, self.adam_beta1, self.adam_beta2,
                        self.adam_eps, self.precision, 1 if self.certify else 0, fr)


class OptState:
    """Adam state of an ascent (bcrown_opt_state): the current iterate, both moments of alpha and
    beta (FP32, in the alpha/beta layouts), the best lb per row and the iteration count t."""

    def __init__(self, batch, K):
        def z(n):
            return torch.zeros(max(int(n), 0), device="cuda", dtype=torch.float32)
        self.alpha_cur, self.m_alpha, self.v_alpha = z(batch.n_alpha), z(batch.n_alpha), z(batch.n_alpha)
        self.beta_cur, self.m_beta, self.v_beta = z(batch.n_beta), z(batch.n_beta), z(batch.n_beta)
        self.best_lb = torch.full((batch.B * K,), -float("inf"), device="cuda")
        self.t = 0

    def c(self):
        return N.OptState(_ptr(self.alpha_cur), _ptr(self.beta_cur), _ptr(self.m_alpha), _ptr(self.v_alpha),
                          _ptr(self.m_beta), _ptr(self.v_beta), _ptr(self.best_lb), self.t)


def optimize(net, dom, batch, alpha, beta, cfg=OptCfg(), out=None, stream=None, state=None):
    """Runs the ascent; alpha, beta are overwritten with the per-row best values. Returns lb [B*K].
    state (OptState, optional) is read when state.t > 0 and holds the state after the call."""
    lib = N.load()
    lb = out if out is not None else torch.empty(batch.B * net.K, device="cuda", dtype=torch.float32)
    d, b, cc = dom.c(), batch.c(), cfg.c()
    st = state.c() if state is not None else None
    N.check(lib.bcrown_optimize(net.handle, C.byref(d), C.byref(b), C.byref(cc), _ptr(alpha), _ptr(beta),
                                _ptr(lb), C.byref(st) if st is not None else None, _stream(stream)))
    if state is not None:
        state.t = st.t
    return lb


def neuron_codes(net, dom, batch, stream=None):
    lib = N.load()
    codes = torch.empty((batch.B * net.K, net.H), device="cuda", dtype=torch.int8)
    d, b = dom.c(), batch.c()
    N.check(lib.bcrown_neuron_codes(net.handle, C.byref(d), C.byref(b), _ptr(codes), _stream(stream)))
    return codes


def batch_split(net, dom, batch, pick_layer, pick_idx, alpha, beta, U, stream=None):
    """Children of batch_split (Algorithm 1); U: per-property unstable counts (host ints)."""
    lib = N.load()
    B = batch.B
    K = net.K
    S = int(batch.split_layer.shape[0])
    cprop = torch.empty(2 * B, device="cuda", dtype=torch.int32)
    coff = torch.empty(2 * B, device="cuda", dtype=torch.int32)
    ccnt = torch.empty(2 * B, device="cuda", dtype=torch.int32)
    clay = torch.empty(2 * (S + B), device="cuda", dtype=torch.uint8)
    cidx = torch.empty(2 * (S + B), device="cuda", dtype=torch.int32)
    csgn = torch.empty(2 * (S + B), device="cuda", dtype=torch.int8)
    caoff = torch.empty(2 * B, device="cuda", dtype=torch.int64)
    ca = torch.empty(2 * batch.n_alpha, device="cuda", dtype=torch.float32)
    cb = torch.empty(2 * (batch.n_beta + B * K), device="cuda", dtype=torch.float32)
    d, b = dom.c(), batch.c()
    N.check(lib.bcrown_batch_split(net.handle, C.byref(d), C.byref(b), _ptr(pick_layer), _ptr(pick_idx),
                                   _ptr(alpha), _ptr(beta), _ptr(cprop), _ptr(coff), _ptr(ccnt), _ptr(clay),
                                   _ptr(cidx), _ptr(csgn), _ptr(caoff), _ptr(ca), _ptr(cb), _stream(stream)))
    child = DeviceBatch(cprop, coff, ccnt, clay, cidx, csgn, caoff, 2 * batch.n_alpha, 2 * (batch.n_beta + B * K))
    return child, ca, cb


def status(net, stream=None):
    """Synchronise and return (and clear) the device status word."""
    return N.load().bcrown_status(net.handle, _stream(stream))


class BoundFunction(torch.autograd.Function):
    """lb = bound(alpha, beta) with the hand-written adjoint kernel as its backward."""

    @staticmethod
    def forward(ctx, alpha, beta, net, dom, batch, row_of_alpha, row_of_beta, precision):
        lb, da, db = bound_grad(net, dom, batch, alpha.detach().contiguous(), beta.detach().contiguous(), precision)
        ctx.save_for_backward(da, db, row_of_alpha, row_of_beta)
        return lb

    @staticmethod
    def backward(ctx, g):
        da, db, ra, rb = ctx.saved_tensors
        return da * g[ra], db * g[rb], None, None, None, None, None, None


def param_rows(batch, K, U):
    """Row index of every alpha and beta entry (device int64), for BoundFunction."""
    B = batch.B
    prop = batch.prop_of.long()
    Up = torch.as_tensor(np.asarray(U), device="cuda").long()[prop]                 # [B]
    rows_b = torch.arange(B, device="cuda") * K
    ra = torch.repeat_interleave(
        (rows_b[:, None] + torch.arange(K, device="cuda")[None, :]).reshape(-1),
        Up.repeat_interleave(K))
    cnt = batch.split_cnt.long()
    rb = torch.repeat_interleave(
        (rows_b[:, None] + torch.arange(K, device="cuda")[None, :]).reshape(-1),
        cnt.repeat_interleave(K))
    return ra, rb


def profile(net, enable=True):
    N.check(N.load().bcrown_profile(net.handle, 1 if enable else 0))


def profile_read(net, cls):
    """(total device ms, launches) of one kernel class recorded since profile(net, True)."""
    t = C.c_double()
    n = C.c_longlong()
    N.check(N.load().bcrown_profile_read(net.handle, cls, C.byref(t), C.byref(n)))
    return t.value, n.value


def bound_xstar(net, dom, batch, alpha, beta, stream=None):
    """FP32 bound of every row and the box point x* minimising its linear bound: (lb [B*K], x* [B*K, d0])."""
    lib = N.load()
    lb = torch.empty(batch.B * net.K, device="cuda", dtype=torch.float32)
    xs = torch.empty((batch.B * net.K, net.d0), device="cuda", dtype=torch.float32)
    d, b = dom.c(), batch.c()
    N.check(lib.bcrown_bound_xstar(net.handle, C.byref(d), C.byref(b), _ptr(alpha), _ptr(beta), _ptr(lb), _ptr(xs),
                                   _stream(stream)))
    return lb, xs


def forward(net, x, stream=None):
    """c_k^T f(x) for rows of x [n, d0] (FP32): the network's specification outputs."""
    lib = N.load()
    x = x.contiguous()
    out = torch.empty((x.shape[0], net.K), device="cuda", dtype=torch.float32)
    N.check(lib.bcrown_forward(net.handle, int(x.shape[0]), _ptr(x), _ptr(out), _stream(stream)))
    return out


def peak_probe(kind, iters=2000, stream=None):
    """Measured FP32 (kind 0) or FP64 (kind 1) FMA throughput of this GPU in TFLOP/s."""
    t = C.c_double()
    N.check(N.load().bcrown_peak_probe(kind, iters, C.byref(t), _stream(stream)))
    return t.value


def kernel_launches():
    return int(N.load().bcrown_kernel_launches())


# ---- BF16 launch configuration and the autotuner ----

def path_supported(net, path):
    return bool(N.load().bcrown_path_supported(net.handle, int(path)))


def set_launch(net, path, grid_per_sm=0):
    cfg = N.LaunchCfg(int(path), int(grid_per_sm))
    N.check(N.load().bcrown_set_launch(net.handle, C.byref(cfg)))


def get_launch(net, rows):
    """(path, grid_per_sm) a BF16 call with `rows` rows takes."""
    cfg = N.LaunchCfg()
    N.check(N.load().bcrown_get_launch(net.handle, int(rows), C.byref(cfg)))
    return cfg.path, cfg.grid_per_sm


def autotune(net, dom, batch, alpha, beta, reps=3, stream=None):
    """Times every supported BF16 configuration on this batch and keeps the fastest for its
    row-count bucket.  Returns ((path, grid_per_sm) chosen, [((path, grid_per_sm), ms), ...])."""
    lib = N.load()
    cands = (N.LaunchCfg * 16)()
    ms = (C.c_double * 16)()
    n = C.c_int()
    best = N.LaunchCfg()
    d, b = dom.c(), batch.c()
    N.check(lib.bcrown_autotune(net.handle, C.byref(d), C.byref(b), _ptr(alpha), _ptr(beta), int(reps), cands, ms,
                                16, C.byref(n), C.byref(best), _stream(stream)))
    return (best.path, best.grid_per_sm), [((cands[i].path, cands[i].grid_per_sm), ms[i]) for i in range(n.value)]


# ---- joint optimisation of intermediate-layer bounds (Section 3.3) ----

def joint_sizes(net, dom, batch, stream=None):
    """(n_alpha', n_beta') of the batch (synchronises)."""
    na, nb = C.c_int64(), C.c_int64()
    d, b = dom.c(), batch.c()
    N.check(N.load().bcrown_joint_sizes(net.handle, C.byref(d), C.byref(b), C.byref(na), C.byref(nb),
                                        _stream(stream)))
    return na.value, nb.value


def joint_init_alpha(net, dom, batch, stream=None):
    """alpha' at the root bounds' rule and beta' = 0 (device tensors)."""
    na, nb = joint_sizes(net, dom, batch, stream)
    ap = torch.zeros(max(na, 1), device="cuda", dtype=torch.float32)[:na]
    bp = torch.zeros(max(nb, 1), device="cuda", dtype=torch.float32)[:nb]
    d, b = dom.c(), batch.c()
    N.check(N.load().bcrown_joint_init_alpha(net.handle, C.byref(d), C.byref(b), _ptr(ap), na, _stream(stream)))
    return ap, bp


def bound_joint(net, dom, batch, alpha, beta, alpha_p, beta_p, stream=None):
    """(lb [B*K], l [B, H], u [B, H]) with the intermediate bounds recomputed per subdomain."""
    lb = torch.empty(batch.B * net.K, device="cuda", dtype=torch.float32)
    l = torch.empty((batch.B, net.H), device="cuda", dtype=torch.float32)
    u = torch.empty_like(l)
    d, b = dom.c(), batch.c()
    N.check(N.load().bcrown_bound_joint(net.handle, C.byref(d), C.byref(b), _ptr(alpha), _ptr(beta), _ptr(alpha_p),
                                        int(alpha_p.numel()), _ptr(beta_p), int(beta_p.numel()), _ptr(lb), _ptr(l),
                                        _ptr(u), _stream(stream)))
    return lb, l, u


def bound_joint_grad(net, dom, batch, alpha, beta, alpha_p, beta_p, stream=None):
    """(lb, d/dalpha, d/dbeta, d/dalpha', d/dbeta') of the sum of all rows' bounds."""
    lb = torch.empty(batch.B * net.K, device="cuda", dtype=torch.float32)
    g = [torch.empty_like(t) for t in (alpha, beta, alpha_p, beta_p)]
    d, b = dom.c(), batch.c()
    N.check(N.load().bcrown_bound_joint_grad(net.handle, C.byref(d), C.byref(b), _ptr(alpha), _ptr(beta),
                                             _ptr(alpha_p), int(alpha_p.numel()), _ptr(beta_p), int(beta_p.numel()),
                                             _ptr(lb), *[_ptr(t) for t in g], _stream(stream)))
    return (lb, *g)


def optimize_joint(net, dom, batch, alpha, beta, alpha_p, beta_p, cfg=None, stream=None):
    """Projected Adam on (alpha, beta, alpha', beta') (FP32); the four are overwritten with the kept
    iterate.  Returns (lb, l, u) there."""
    cfg = cfg or OptCfg(certify=False)
    lb = torch.empty(batch.B * net.K, device="cuda", dtype=torch.float32)
    l = torch.empty((batch.B, net.H), device="cuda", dtype=torch.float32)
    u = torch.empty_like(l)
    d, b, cc = dom.c(), batch.c(), cfg.c()
    N.check(N.load().bcrown_optimize_joint(net.handle, C.byref(d), C.byref(b), C.byref(cc), _ptr(alpha), _ptr(beta),
                                           _ptr(alpha_p), int(alpha_p.numel()), _ptr(beta_p), int(beta_p.numel()),
                                           _ptr(lb), _ptr(l), _ptr(u), _stream(stream)))
    return lb, l, u


# ---- optimisation steps replayed from CUDA graphs, per bucket of the batch size ----

def workspace(net, reserve=0):
    """(address, bytes) of the net's device workspace after growing it to `reserve` bytes."""
    p, n = C.c_void_p(), C.c_int64()
    N.check(N.load().bcrown_workspace(net.handle, int(reserve), C.byref(p), C.byref(n)))
    return p.value, n.value


def bucket(n):
    """n rounded up to a multiple of 2^(floor(log2 n) - 3): 8 buckets per power of two, at most
    12.5 % padding (n <= 8 stays as it is)."""
    n = int(n)
    if n <= 8:
        return max(n, 1)
    g = 1 << (n.bit_length() - 4)
    return (n + g - 1) // g * g


class GraphOptimizer:
    """bcrown_optimize replayed from a CUDA graph captured once per bucket of the batch sizes.

    A batch of B subdomains is padded to bucket(B) subdomains with copies of its last one (their
    rows are computed and dropped: rows are independent), and its alpha, beta and split arrays to
    capacities that only the bucket fixes (K U_max alphas, K MAX_SPLITS betas and MAX_SPLITS split
    entries per subdomain; entries past the real ones are referenced by no subdomain).  The first
    batch of a bucket runs once eagerly (which sizes the net's workspace, converts weights and
    builds tables), then one call is captured; later batches of the bucket copy their arrays into
    the captured buffers and replay.  A graph refers to the net's workspace, so one whose
    workspace has since been reallocated (a larger call on the same net) is captured again."""

    def __init__(self, net, dom, cfg, unstable_counts):
        self.net, self.dom, self.cfg = net, dom, cfg
        self.U = np.asarray(unstable_counts, np.int64)
        self.K = net.K
        self.entries = {}
        self.captures = 0

    def _pad_batch(self, hb):
        """The batch arrays padded to the bucket, and the capacities that key its graph."""
        B, K = hb.B, self.K
        Bb = bucket(B)
        last = B - 1
        o, c = int(hb.split_off[last]), int(hb.split_cnt[last])
        na_last = int(self.U[hb.prop_of[last]]) * K
        extra = Bb - B
        prop = np.concatenate([hb.prop_of, np.full(extra, hb.prop_of[last], np.int32)]).astype(np.int32)
        cnt = np.concatenate([hb.split_cnt, np.full(extra, c, np.int32)]).astype(np.int32)
        off = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.int32)
        aoff = np.concatenate([hb.alpha_off, int(hb.alpha_off[last]) + na_last * np.arange(1, extra + 1)]).astype(np.int64)
        lay = np.concatenate([hb.split_layer] + [hb.split_layer[o:o + c]] * extra)
        idx = np.concatenate([hb.split_idx] + [hb.split_idx[o:o + c]] * extra)
        sgn = np.concatenate([hb.split_sign] + [hb.split_sign[o:o + c]] * extra)
        # capacities fixed by the bucket alone (one graph per bucket, whatever the batch holds):
        # K U_max alphas and K MAX_SPLITS betas per subdomain, MAX_SPLITS split entries
        caps = (Bb, Bb * K * int(self.U.max(initial=0)), Bb * K * N.MAX_SPLITS, Bb * N.MAX_SPLITS)
        return caps, dict(prop_of=prop, split_off=off, split_cnt=cnt, alpha_off=aoff, split_layer=lay,
                          split_idx=idx, split_sign=sgn)

    def _pad(self, hb, alpha, beta):
        B, K = hb.B, self.K
        last = B - 1
        o, c = int(hb.split_off[last]), int(hb.split_cnt[last])
        na_last = int(self.U[hb.prop_of[last]]) * K
        extra = bucket(B) - B
        caps, arrays = self._pad_batch(hb)
        a_last = np.asarray(alpha[int(hb.alpha_off[last]):int(hb.alpha_off[last]) + na_last], np.float32)
        b_last = np.asarray(beta[o * K:(o + c) * K], np.float32)
        a = np.concatenate([np.asarray(alpha, np.float32)] + [a_last] * extra)
        b = np.concatenate([np.asarray(beta, np.float32)] + [b_last] * extra)
        return caps, arrays, a, b

    def _capture(self, caps, load):
        Bb, na, nb, ns = caps
        dev = {"prop_of": torch.zeros(Bb, dtype=torch.int32, device="cuda"),
               "split_off": torch.zeros(Bb, dtype=torch.int32, device="cuda"),
               "split_cnt": torch.zeros(Bb, dtype=torch.int32, device="cuda"),
               "alpha_off": torch.zeros(Bb, dtype=torch.int64, device="cuda"),
               "split_layer": torch.zeros(max(ns, 1), dtype=torch.uint8, device="cuda"),
               "split_idx": torch.zeros(max(ns, 1), dtype=torch.int32, device="cuda"),
               "split_sign": torch.zeros(max(ns, 1), dtype=torch.int8, device="cuda")}
        e = {"dev": dev, "alpha": torch.zeros(max(na, 1), device="cuda"), "beta": torch.zeros(max(nb, 1), device="cuda"),
             "lb": torch.empty(Bb * self.K, device="cuda")}
        e["db"] = DeviceBatch(dev["prop_of"], dev["split_off"], dev["split_cnt"], dev["split_layer"], dev["split_idx"],
                              dev["split_sign"], dev["alpha_off"], na, nb)
        load(e)
        optimize(self.net, self.dom, e["db"], e["alpha"], e["beta"], self.cfg, out=e["lb"])   # sizes everything
        torch.cuda.synchronize()
        ws = workspace(self.net)[0]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            optimize(self.net, self.dom, e["db"], e["alpha"], e["beta"], self.cfg, out=e["lb"])
        torch.cuda.synchronize()
        if workspace(self.net)[0] != ws:
            raise RuntimeError("workspace reallocated during capture")
        e["graph"], e["ws"] = g, ws
        self.entries[caps] = e
        self.captures += 1
        return e

    @staticmethod
    def _load(e, arrays, a, b):
        for k, v in arrays.items():
            t = torch.from_numpy(np.ascontiguousarray(v.astype(np.int32) if k == "split_idx" else v))
            e["dev"][k][:len(v)].copy_(t)
        e["alpha"][:len(a)].copy_(torch.from_numpy(a))
        e["beta"][:len(b)].copy_(torch.from_numpy(b))

    def _replay(self, caps, load):
        e = self.entries.get(caps)
        if e is not None and e["ws"] != workspace(self.net)[0]:
            e = None
        if e is None:
            e = self._capture(caps, load)
        load(e)
        e["graph"].replay()
        return e

    def rows(self, hb, alpha, beta):
        """As a call, for a host batch whose alpha (device tensor) and compact beta (device tensor)
        stay on the device: they are copied into the captured buffers, and the per-row best values
        back into them.  Returns lb [B K] on the device."""
        B, K = hb.B, self.K
        last = B - 1
        o, c = int(hb.split_off[last]), int(hb.split_cnt[last])
        a0, na_last = int(hb.alpha_off[last]), int(self.U[hb.prop_of[last]]) * K
        extra = bucket(B) - B
        caps, arrays = self._pad_batch(hb)
        av, bv = alpha.reshape(-1), beta.reshape(-1)

        def load(e):
            e["alpha"][:hb.n_alpha].copy_(av[:hb.n_alpha])
            if extra:   # the padding subdomains' copies of the last one's alpha and beta
                e["alpha"][a0 + na_last:a0 + na_last * (extra + 1)].copy_(av[a0:a0 + na_last].repeat(extra))
                e["beta"][hb.n_beta:hb.n_beta + extra * c * K].copy_(bv[o * K:(o + c) * K].repeat(extra))
            e["beta"][:hb.n_beta].copy_(bv[:hb.n_beta])
            for k, v in arrays.items():
                t = torch.from_numpy(np.ascontiguousarray(v.astype(np.int32) if k == "split_idx" else v))
                e["dev"][k][:len(v)].copy_(t)

        e = self._replay(caps, load)
        av.copy_(e["alpha"][:hb.n_alpha])
        bv.copy_(e["beta"][:hb.n_beta])
        return e["lb"][:B * K].clone()

    def __call__(self, hb, alpha, beta):
        """The optimised bounds (B K rows), alpha and beta of host batch hb (numpy outputs)."""
        caps, arrays, a, b = self._pad(hb, alpha, beta)
        e = self._replay(caps, lambda e: self._load(e, arrays, a, b))
        n = hb.B * self.K
        return (e["lb"][:n].cpu().numpy(), e["alpha"][:hb.n_alpha].cpu().numpy(),
                e["beta"][:hb.n_beta].cpu().numpy())
