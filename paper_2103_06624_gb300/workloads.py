"""Seeded synthetic inputs: networks, input boxes, specifications and split sets.

This module only draws random numbers and lays them out. It holds none of the
bound-propagation arithmetic, so both the CPU oracle (test infrastructure) and
the CUDA path take their inputs from here.

Shapes follow the problem statement of the paper (Section 2.1, Eq. 1): an
L-layer ReLU network with weights W^(i) in R^{d_i x d_{i-1}} and biases b^(i),
an L-infinity box around x0, and margin specifications c = e_y - e_j merged
into the last layer.  Split sets follow Eq. 3 (S = -1 for a "z >= 0" split,
+1 for a "z < 0" split) and the batch_split step of Algorithm 1.

Weight law: W ~ N(0, 2/fan_in) (He variance), b ~ N(0, 0.01) (variance 0.01,
standard deviation 0.1); for convolutions fan_in = Cin * k * k.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Layer:
    """One linear layer: 'fc' (W [d_out, d_in]) or 'conv' (W [Cout, Cin, k, k])."""
    kind: str
    W: np.ndarray
    b: np.ndarray
    in_shape: tuple
    out_shape: tuple
    stride: int = 1
    pad: int = 0

    @property
    def d_in(self) -> int:
        return int(np.prod(self.in_shape))

    @property
    def d_out(self) -> int:
        return int(np.prod(self.out_shape))

    @property
    def k(self) -> int:
        return int(self.W.shape[-1]) if self.kind == "conv" else 1


@dataclass
class Problem:
    """A network, its specification matrix C and a set of input boxes."""
    name: str
    layers: list
    C: np.ndarray            # [K, d_L] float32
    x0: np.ndarray           # [P, d0] float32
    x_lo: np.ndarray         # [P, d0] float32
    x_hi: np.ndarray         # [P, d0] float32
    eps: float
    labels: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    specs_per_prop: np.ndarray | None = None   # [P, K, d_L] when specs differ per property

    @property
    def widths(self) -> list:
        return [self.layers[0].d_in] + [ly.d_out for ly in self.layers]

    @property
    def hidden_widths(self) -> list:
        return [ly.d_out for ly in self.layers[:-1]]

    @property
    def K(self) -> int:
        return int(self.C.shape[0])

    @property
    def P(self) -> int:
        return int(self.x0.shape[0])


@dataclass
class Batch:
    """Subdomains with their split lists, in the layout the C-ABI takes.

    Row (b, k) is subdomain b under spec k.  alpha for that row lives at
    alpha[alpha_off[b] + k*U[prop_of[b]] + t] (t = rank of the neuron among its
    property's unstable neurons in layer-major order); beta of split t of
    subdomain b lives at beta[split_off[b]*K + k*split_cnt[b] + t].
    """
    prop_of: np.ndarray      # [B] int32
    split_off: np.ndarray    # [B] int32
    split_cnt: np.ndarray    # [B] int32
    split_layer: np.ndarray  # [S] uint8, paper layer index 1..L-1
    split_idx: np.ndarray    # [S] uint32, neuron index within its layer
    split_sign: np.ndarray   # [S] int8, S^(i)_jj of Eq. 3
    alpha_off: np.ndarray    # [B] int64
    n_alpha: int
    n_beta: int

    @property
    def B(self) -> int:
        return int(self.prop_of.shape[0])


def _rng(seed):
    return np.random.default_rng(seed)


def fc_layer(rng, d_in, d_out, bias_var=0.01):
    W = rng.normal(0.0, math.sqrt(2.0 / d_in), size=(d_out, d_in)).astype(np.float32)
    b = rng.normal(0.0, math.sqrt(bias_var), size=(d_out,)).astype(np.float32)
    return Layer("fc", W, b, (d_in,), (d_out,))


def conv_layer(rng, in_shape, cout, k, stride, pad, bias_var=0.01):
    cin, h, w = in_shape
    ho = (h + 2 * pad - k) // stride + 1
    wo = (w + 2 * pad - k) // stride + 1
    fan_in = cin * k * k
    W = rng.normal(0.0, math.sqrt(2.0 / fan_in), size=(cout, cin, k, k)).astype(np.float32)
    b = rng.normal(0.0, math.sqrt(bias_var), size=(cout,)).astype(np.float32)
    return Layer("conv", W, b, (cin, h, w), (cout, ho, wo), stride, pad)


def mlp_layers(widths, seed):
    rng = _rng(seed)
    return [fc_layer(rng, widths[i], widths[i + 1]) for i in range(len(widths) - 1)]


def conv_layers(in_shape, convs, fcs, seed):
    """convs: list of (cout, k, stride, pad); fcs: widths after flattening."""
    rng = _rng(seed)
    layers = []
    shape = tuple(in_shape)
    for cout, k, s, p in convs:
        ly = conv_layer(rng, shape, cout, k, s, p)
        layers.append(ly)
        shape = ly.out_shape
    d = int(np.prod(shape))
    for w in fcs:
        ly = fc_layer(rng, d, w)
        layers.append(ly)
        d = w
    return layers


def reference_forward(layers, x):
    """Network function of Eq. 1 in float64 (labels only; no bound arithmetic)."""
    import torch
    import torch.nn.functional as F
    h = torch.as_tensor(np.asarray(x, np.float64))
    single = h.dim() == 1
    if single:
        h = h[None]
    n = h.shape[0]
    for i, ly in enumerate(layers):
        W = torch.as_tensor(ly.W.astype(np.float64))
        b = torch.as_tensor(ly.b.astype(np.float64))
        if ly.kind == "fc":
            z = h.reshape(n, -1) @ W.T + b
        else:
            z = F.conv2d(h.reshape((n,) + tuple(ly.in_shape)), W, b, stride=ly.stride,
                         padding=ly.pad).reshape(n, -1)
        h = torch.relu(z) if i < len(layers) - 1 else z
    out = h.numpy()
    return out[0] if single else out


def margin_C(y, n_classes, js):
    C = np.zeros((len(js), n_classes), np.float32)
    for r, j in enumerate(js):
        C[r, y] = 1.0
        C[r, j] = -1.0
    return C


def make_boxes(rng, n_props, d0, eps):
    x0 = rng.uniform(0.0, 1.0, size=(n_props, d0)).astype(np.float32)
    x_lo = (x0.astype(np.float64) - eps).astype(np.float32)
    x_hi = (x0.astype(np.float64) + eps).astype(np.float32)
    return x0, x_lo, x_hi


def make_problem(name, layers, n_props, eps, n_specs, seed):
    """Boxes around x0 ~ U[0,1]^d0, spec rows e_y - e_j, y = argmax f(x0) of property 0.

    All properties share one spec matrix C (so the merged last layer is
    shared); the label is taken from property 0's centre.  With n_specs <
    n_classes - 1, the j's are the first n_specs classes other than y.
    """
    rng = _rng(seed + 7919)
    d0 = layers[0].d_in
    x0, x_lo, x_hi = make_boxes(rng, n_props, d0, eps)
    logits = reference_forward(layers, x0[0])
    y = int(np.argmax(logits))
    n_classes = layers[-1].d_out
    js = [j for j in range(n_classes) if j != y][:n_specs]
    C = margin_C(y, n_classes, js)
    return Problem(name, layers, C, x0, x_lo, x_hi, float(eps), np.array([y]))


# --------------------------------------------------------------------------------------
# Split sets (Eq. 3) and batches
# --------------------------------------------------------------------------------------

def neuron_layer_index(hidden_widths, gidx):
    """Global hidden-neuron index -> (paper layer i in 1..L-1, index j in layer)."""
    offs = np.cumsum([0] + list(hidden_widths))
    layer = np.searchsorted(offs, gidx, side="right")
    return layer.astype(np.int64), (np.asarray(gidx) - offs[layer - 1]).astype(np.int64)


def random_split_sets(rng, unstable, depth_lo, depth_hi):
    """One subdomain: depth ~ U{lo..hi} distinct root-unstable neurons, signs +-1 (p=1/2)."""
    depth = int(rng.integers(depth_lo, depth_hi + 1))
    depth = min(depth, len(unstable))
    if depth == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int8)
    pick = rng.choice(len(unstable), size=depth, replace=False)
    signs = np.where(rng.random(depth) < 0.5, -1, 1).astype(np.int8)
    return np.asarray(unstable)[pick].astype(np.int64), signs


def bab_tree_leaves(rng, unstable, n_leaves, max_depth, min_depth=1):
    """Leaves of a random branch-and-bound tree, like repeated batch_split (Algorithm 1).

    Starting from the unsplit root, repeatedly pick a random leaf with depth <
    max_depth, split one of its unsplit root-unstable neurons, and keep both
    children (C^l: z >= 0, sign -1; C^u: z < 0, sign +1), until n_leaves leaves
    exist.  Leaves share prefixes exactly as children of batch_split do.
    """
    unstable = np.asarray(unstable, np.int64)
    leaves = [([], [])]
    if len(unstable) == 0:
        return [(np.zeros(0, np.int64), np.zeros(0, np.int8))] * n_leaves
    while len(leaves) < n_leaves:
        cand = [i for i, (ns, _) in enumerate(leaves) if len(ns) < min(max_depth, len(unstable))]
        if not cand:
            break
        i = cand[int(rng.integers(len(cand)))]
        ns, ss = leaves.pop(i)
        used = set(ns)
        free = [n for n in unstable.tolist() if n not in used]
        n = free[int(rng.integers(len(free)))]
        leaves.append((ns + [n], ss + [-1]))
        leaves.append((ns + [n], ss + [1]))
    # every leaf has depth >= min_depth by construction when n_leaves >= 2
    return [(np.array(ns, np.int64), np.array(ss, np.int8)) for ns, ss in leaves]


def pack_batch(hidden_widths, K, U, subdomains):
    """subdomains: list of (prop, neuron_gidx[], signs[]) -> Batch (C-ABI layout)."""
    B = len(subdomains)
    prop_of = np.array([s[0] for s in subdomains], np.int32)
    cnt = np.array([len(s[1]) for s in subdomains], np.int32)
    off = np.zeros(B, np.int32)
    if B > 1:
        off[1:] = np.cumsum(cnt)[:-1]
    gidx = np.concatenate([s[1] for s in subdomains]) if cnt.sum() else np.zeros(0, np.int64)
    signs = np.concatenate([s[2] for s in subdomains]) if cnt.sum() else np.zeros(0, np.int8)
    layer, idx = neuron_layer_index(hidden_widths, gidx) if len(gidx) else (np.zeros(0, np.int64),) * 2
    U = np.asarray(U, np.int64)
    per = U[prop_of] * K
    alpha_off = np.zeros(B, np.int64)
    if B > 1:
        alpha_off[1:] = np.cumsum(per)[:-1]
    return Batch(prop_of, off, cnt, layer.astype(np.uint8), idx.astype(np.uint32),
                 signs.astype(np.int8), alpha_off, int(per.sum()), int(cnt.sum()) * K)


def random_batch(problem, unstable_lists, B, depth_lo, depth_hi, seed, props=None):
    """B subdomains, each with independent random splits on its property's unstable neurons."""
    rng = _rng(seed + 104729)
    P = problem.P
    subs = []
    for b in range(B):
        p = int(props[b]) if props is not None else b % P
        ns, ss = random_split_sets(rng, unstable_lists[p], depth_lo, depth_hi)
        subs.append((p, ns, ss))
    return pack_batch(problem.hidden_widths, problem.K, [len(u) for u in unstable_lists], subs)


def tree_batch(problem, unstable_lists, counts, max_depth, seed):
    """For property p, counts[p] leaves of a random BaB tree of depth <= max_depth."""
    rng = _rng(seed + 1299709)
    subs = []
    for p, n in enumerate(counts):
        for ns, ss in bab_tree_leaves(rng, unstable_lists[p], int(n), max_depth):
            subs.append((p, ns, ss))
    return pack_batch(problem.hidden_widths, problem.K, [len(u) for u in unstable_lists], subs)


def initial_alpha_beta(batch, value=0.5, beta_value=0.0):
    return (np.full(batch.n_alpha, value, np.float32), np.full(batch.n_beta, beta_value, np.float32))


def random_alpha_beta(batch, seed, beta_max=1.0):
    rng = _rng(seed + 15485863)
    a = rng.uniform(0.0, 1.0, size=batch.n_alpha).astype(np.float32)
    b = rng.uniform(0.0, beta_max, size=batch.n_beta).astype(np.float32)
    return a, b


# --------------------------------------------------------------------------------------
# The workloads, each a seeded synthetic stand-in for the paper's models (Table A4 shapes,
# batch sizes of Appendix C.1).  The trained CIFAR/MNIST models are not available.
# --------------------------------------------------------------------------------------

def problem_mlp_small(seed=0):
    """ReLU MLP 16-32-32-4, eps=0.05, 3 margin specs (the small case)."""
    layers = mlp_layers([16, 32, 32, 4], seed)
    return make_problem("mlp_16_32_32_4", layers, 1, 0.05, 3, seed)


def problem_mlp_784(seed=0, n_props=1):
    """ReLU MLP 784-256x6-10, eps=0.015, 9 margin specs."""
    layers = mlp_layers([784] + [256] * 6 + [10], seed)
    return make_problem("mlp_784_256x6_10", layers, n_props, 0.015, 9, seed)


def problem_conv_small(seed=0):
    """3x32x32 -> conv32 4x4 s2 p1 -> conv64 4x4 s2 p1 -> fc 4096-512-512-10, eps=2/255."""
    layers = conv_layers((3, 32, 32), [(32, 4, 2, 1), (64, 4, 2, 1)], [512, 512, 10], seed)
    return make_problem("conv_3x32x32_c32_c64_fc512_512_10", layers, 1, 2.0 / 255.0, 9, seed)


def problem_conv_big(seed=0):
    """3x32x32 -> conv64,64,128,128 3x3 (strides 1,2,1,2, pad 1) -> fc 8192-512-10, eps=2/255."""
    layers = conv_layers((3, 32, 32), [(64, 3, 1, 1), (64, 3, 2, 1), (128, 3, 1, 1), (128, 3, 2, 1)],
                         [512, 10], seed)
    return make_problem("conv_3x32x32_c64_c64_c128_c128_fc512_10", layers, 1, 2.0 / 255.0, 9, seed)


def loguniform_counts(n_props, lo, hi, seed):
    rng = _rng(seed + 32452843)
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_props))).astype(np.int64)
