"""Shared set-up for the GPU parity tests: problems, oracle values, device copies."""
from __future__ import annotations

import numpy as np

from oracle import bcrown_oracle as O
from paper_2103_06624_gb300 import workloads as wl

# FP32 parity bar against the FP64 oracle at fixed alpha, beta: |gpu - oracle| <= RTOL * max(|oracle|, 1)
RTOL = 1e-5


def rel_err(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(gpu - ref) / np.maximum(np.abs(ref), 1.0)


def oracle_setup(pb):
    """Oracle net, root bounds rounded to float32 (both sides then see identical l, u)."""
    net = O.OracleNet(pb.layers, pb.C)
    l, u = O.root_bounds(net, pb.x_lo, pb.x_hi)
    l32, u32 = l.astype(np.float32), u.astype(np.float32)
    unst = [np.nonzero(O.unstable_mask(l32[p], u32[p]))[0] for p in range(pb.P)]
    props = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=l32, u=u32)
    return net, props, unst


def repack(pb, batch, U, idx, alpha, beta):
    """Host Batch of subdomains idx with their alpha/beta slices."""
    K = pb.K
    offs = np.concatenate([[0], np.cumsum(pb.hidden_widths)])
    subs, a_parts, b_parts = [], [], []
    for b in idx:
        o, c = int(batch.split_off[b]), int(batch.split_cnt[b])
        g = offs[batch.split_layer[o:o + c].astype(np.int64) - 1] + batch.split_idx[o:o + c].astype(np.int64)
        subs.append((int(batch.prop_of[b]), g.astype(np.int64), batch.split_sign[o:o + c]))
        n = int(U[batch.prop_of[b]]) * K
        a_parts.append(alpha[batch.alpha_off[b]:batch.alpha_off[b] + n])
        b_parts.append(beta[o * K:(o + c) * K])
    nb = wl.pack_batch(pb.hidden_widths, K, U, subs)
    return nb, np.concatenate(a_parts) if a_parts else np.zeros(0), np.concatenate(b_parts) if b_parts else np.zeros(0)


def grad_groups(net, batch, props):
    """Hidden layer of every alpha and every beta entry (for per-layer gradient comparisons)."""
    rows = O.expand_rows(net, batch, props["l"], props["u"])
    la = np.zeros(batch.n_alpha, np.int64)
    lb = np.zeros(batch.n_beta, np.int64)
    for i in range(1, net.L):
        ai = rows.alpha_idx[i]
        la[ai[ai >= 0]] = i
        bi = rows.beta_idx[i]
        lb[bi[bi >= 0]] = i
    return la, lb


def grad_agreement(g, g_ref, layer, tol, floor=1e-2):
    """Per hidden layer: the fraction of entries with |g - g_ref| <= tol (|g_ref| + floor * max |g_ref|)
    (the max taken over the layer's entries), and the cosine of the layer's gradient vectors."""
    out = {}
    for i in np.unique(layer):
        m = layer == i
        gi, ri = np.asarray(g, np.float64)[m], np.asarray(g_ref, np.float64)[m]
        sc = np.abs(ri).max(initial=0.0)
        ok = np.abs(gi - ri) <= tol * (np.abs(ri) + floor * sc)
        den = np.linalg.norm(gi) * np.linalg.norm(ri)
        out[int(i)] = (float(ok.mean()) if ok.size else 1.0, float(gi @ ri / den) if den > 0 else 1.0, int(m.sum()))
    return out
