"""Host-side logic of bench.py (no GPU): the byte models behind the roofline numbers, the
workload table, and when a committed DRAM-traffic record is used."""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2103_06624_gb300 import workloads as wl  # noqa: E402


def test_layer_path_byte_model_matches_the_per_row_figures():
    """Lambda (backward) and h (forward) of every hidden neuron written and read once in BF16: 8 bytes
    per hidden neuron per row and iteration, 4 per input (x*), 16 per unstable neuron and 8 per
    split: 98 KB of activations for the small conv net ((8192 + 4096 + 512 + 512) hidden neurons)
    and 987 KB for the large one ((65536 + 16384 + 32768 + 8192 + 512))."""
    zero = np.zeros(1)
    for pb, hidden in ((wl.problem_conv_small(), 8192 + 4096 + 512 + 512),
                       (wl.problem_conv_big(), 65536 + 16384 + 32768 + 8192 + 512)):
        assert bench.layer_gemm_bytes_per_row_iter(pb, zero, zero)[0] == 8 * hidden + 4 * 3072
    pb = wl.problem_conv_small()
    b = bench.layer_gemm_bytes_per_row_iter(pb, np.array([10.0]), np.array([3.0]))[0]
    assert b == 8 * (8192 + 4096 + 1024) + 4 * 3072 + 16 * 10 + 8 * 3


def test_flop_models():
    # 784-256x6-10: one backward pass of one row contracts layers 1..L-1
    assert bench.algorithmic_flops_per_row_pass(wl.problem_mlp_784().layers) == 2 * (784 * 256 + 5 * 256 * 256)
    # the precision workload's conv net: 87.4 MFLOP per row and pass (conv 3->64, 64->64 s2,
    # 64->128, 128->128 s2, all 3x3, then fc 8192->512)
    f = bench.algorithmic_flops_per_row_pass(wl.problem_conv_big().layers)
    assert f == 2 * (64 * 1024 * 3 * 9 + 64 * 256 * 64 * 9 + 128 * 256 * 64 * 9 + 128 * 64 * 128 * 9 + 512 * 8192)
    assert abs(f - 87.4e6) < 0.1e6


def test_workload_table_builds_each_problem():
    for name, w in bench.WORKLOADS.items():
        pb = bench.make_problem(name, 0, wl)
        assert pb.K == 9
        assert "{n}" in w["desc"]
        if name == "batching":
            assert pb.P == 64
            counts = wl.loguniform_counts(pb.P, 16, 4096, 0)
            assert counts.min() >= 16 and counts.max() <= 4096
        else:
            assert pb.P == 1 and w["subdomains"] > 0


def _record(tmp, sources, data=b"kernel source", sha=None):
    os.makedirs(os.path.join(tmp, "profiles"), exist_ok=True)
    for f in sources:
        p = os.path.join(tmp, f)
        os.makedirs(os.path.dirname(p), exist_ok=True)
        open(p, "wb").write(data)
    h = hashlib.sha256()
    for _ in sources:
        h.update(data)
    rec = {"sources": sources, "sources_sha256": sha or h.hexdigest(), "dram_bytes_per_launch": 1000.0}
    json.dump(rec, open(os.path.join(tmp, "profiles", "k.json"), "w"))


def test_traffic_record_is_used_only_while_its_sources_are_unchanged(tmp_path, monkeypatch):
    tmp = str(tmp_path)
    monkeypatch.setattr(bench, "ROOT", tmp)
    assert bench.measured_traffic("k", 500.0) is None                     # no record
    _record(tmp, ["a.cu", "b.cuh"])
    tr = bench.measured_traffic("k", 500.0)
    assert tr["dram_bytes_per_launch"] == 1000.0 and tr["vs_algorithmic"] == 2.0
    open(os.path.join(tmp, "b.cuh"), "ab").write(b" changed")            # a source changed
    assert bench.measured_traffic("k", 500.0) is None
    json.dump({"source": "a.cu", "source_sha256": "x"}, open(os.path.join(tmp, "profiles", "k.json"), "w"))
    assert bench.measured_traffic("k", 500.0) is None                     # older record format


def test_committed_fused_record_names_existing_sources():
    rec = json.load(open(os.path.join(ROOT, "profiles", "k_fused_grad.json")))
    assert all(os.path.exists(os.path.join(ROOT, f)) for f in rec["sources"])
    assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]


def test_joint_flop_model():
    """784-256x6-10: target layer T (2..6) back-substitutes 512 rows through T-1 layers (the
    first 784x256, the rest 256x256) three times (backward, recomputed backward, adjoint); the 9
    spec rows go through all six hidden layers twice."""
    w = [784] + [256] * 6 + [10]
    first, rest = 2 * 256 * 784, 2 * 256 * 256
    expect = sum(512 * (first + (T - 2) * rest) * 3 for T in range(2, 7)) + 9 * (first + 5 * rest) * 2
    assert bench.joint_flops_per_subdomain_iter(w, 9) == expect


def test_layer_gemm_operand_byte_model():
    """conv_big: hidden layers of 65536, 16384, 32768, 8192 and 512 neurons over a 3072-input
    image; each contraction's FP32 operand read and output written once per direction."""
    w = wl.problem_conv_big().widths
    assert w[:6] == [3072, 65536, 16384, 32768, 8192, 512]
    expect = 8 * ((65536 + 3072) + (16384 + 65536) + (32768 + 16384) + (8192 + 32768) + (512 + 8192))
    assert bench.tcg_bytes_per_row_iter(w) == expect == 1994752


def test_end_to_end_parts_are_the_batch_in_order():
    """The parts the end-to-end measurement pipelines: contiguous ranges of subdomains whose
    rebased split lists, alpha and beta slices put back together give the whole batch."""
    pb = wl.problem_mlp_small()
    unst = [np.arange(40)]
    hb = wl.tree_batch(pb, unst, [37], 6, 3)
    K = pb.K
    parts = bench._split_host_batch(hb, K, 4)
    assert len(parts) == 4 and parts[0][1][0] == 0 and parts[-1][1][1] == hb.B
    for (sub, (b0, b1), (a0, a1), (s0, s1)), nxt in zip(parts, parts[1:] + [None]):
        assert sub.B == b1 - b0 and sub.n_alpha == a1 - a0 and sub.n_beta == s1 - s0
        np.testing.assert_array_equal(sub.split_off + hb.split_off[b0], hb.split_off[b0:b1])
        np.testing.assert_array_equal(sub.alpha_off + hb.alpha_off[b0], hb.alpha_off[b0:b1])
        S0 = int(hb.split_off[b0])
        np.testing.assert_array_equal(sub.split_idx, hb.split_idx[S0:S0 + len(sub.split_idx)])
        np.testing.assert_array_equal(sub.split_sign, hb.split_sign[S0:S0 + len(sub.split_sign)])
        assert s0 == S0 * K
        if nxt is not None:
            assert nxt[1][0] == b1 and nxt[2][0] == a1 and nxt[3][0] == s1
    assert parts[-1][2][1] == hb.n_alpha and parts[-1][3][1] == hb.n_beta
