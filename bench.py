"""Throughput of batched beta-CROWN subdomain bounding on one or more GB300s.

One step = one call of bcrown_optimize on a batch of subdomains: 20 projected-
Adam iterations on alpha, beta (each a bound pass plus its adjoint) and the
final certifying pass.  Workload (default, --workload conv_big, the largest
single-GPU configuration): the CIFAR-shaped conv net 3x32x32 -> conv
64,64,128,128 (3x3, strides 1,2,1,2) -> fc 8192-512-10 (He init, seeded),
eps = 2/255, 9 margin specs, 4096 subdomains that are the leaves of a random
branch-and-bound tree of depth <= 24; BF16 iterations and an FP32 certifying
pass.  Other workloads (--workload): mlp784 (the ReLU MLP 784-256x6-10,
x0 ~ U[0,1]^784, eps = 0.015, 1024 subdomains, depth <= 12), batching (the same
MLP, 64 properties with log-uniform 16-4096 subdomains each, depth <= 20) and
conv_small (3x32x32 -> conv 32,64 (4x4, stride 2) -> fc 4096-512-512-10, 2048
subdomains, depth <= 16).

Prints one JSON line (rank 0).  Under torchrun each rank bounds its own batch
(weak scaling, no collective on the data path); the barrier and the maximum
over ranks are for timing only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "subdomain lower bounds/sec (20 alpha,beta iters)"
UNIT = "subdomains/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--workload", default="conv_big", choices=sorted(WORKLOADS))
    ap.add_argument("--subdomains", type=int, default=None, help="per property (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-form", action="store_true", help="skip timing the plain FP32 form beside BF16")
    ap.add_argument("--fp32-steps", type=int, default=10, help="timed steps of the plain FP32 form")
    ap.add_argument("--no-autotune", action="store_true", help="skip the launch-configuration tuner")
    ap.add_argument("--launch-path", default=None, choices=["fused", "layer_epi", "layer_gather", "layer_im2col"],
                    help="take this BF16 path instead of tuning (for profiling one path)")
    ap.add_argument("--no-joint", action="store_true", help="skip the joint intermediate-bound measurement")
    ap.add_argument("--bab", action="store_true",
                    help="instead of the bound throughput: host and engine time per child of the two branch-and-"
                         "bound drivers (array pool, list pool) on the workload's first property")
    ap.add_argument("--bab-rounds", type=int, default=14)
    ap.add_argument("--bab-batch", type=int, default=512)
    ap.add_argument("--joint-subdomains", type=int, default=64,
                    help="subdomains of the joint intermediate-bound measurement (784-256x6-10 MLP)")
    ap.add_argument("--no-graph", action="store_true", help="launch the timed steps eagerly instead of replaying "
                                                             "one captured CUDA graph")
    ap.add_argument("--profile-timed", action="store_true",
                    help="open a CUDA profiler range around the timed steps only (ncu --profile-from-start off)")
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help="subdomains timed on the oracle (default: the workload's, about 10-25 s)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.subdomains is None:
        args.subdomains = w["subdomains"]
    if args.cpu_sample is None:
        args.cpu_sample = w["cpu_sample"]
    return args


# ------------------------------------------------------------------------------ workload

# subdomains: per property (batching: the upper end of the log-uniform range is fixed instead)
WORKLOADS = {
# cpu_sample: subdomains of the oracle leg of our arm (about 10-25 s); ref_sample: subdomains per
# step of the --impl reference arm (so that 25 steps end within a few minutes)
    "mlp784": {"subdomains": 1024, "depth": 12, "cpu_sample": 640, "ref_sample": 256,
               "desc": "mlp_784_256x6_10 eps=0.015, {n} BaB-tree subdomains (depth<=12), 9 specs"},
    "batching": {"subdomains": None, "depth": 20, "cpu_sample": 640, "ref_sample": 256,
                 "desc": "mlp_784_256x6_10 eps=0.015, 64 properties x log-uniform 16-4096 BaB-tree subdomains "
                         "({n} in all, depth<=20), 9 specs"},
    "conv_small": {"subdomains": 2048, "depth": 16, "cpu_sample": 16, "ref_sample": 8,
                   "desc": "conv_3x32x32_c32_c64_fc512_512_10 eps=2/255, {n} BaB-tree subdomains (depth<=16), 9 specs"},
    "conv_big": {"subdomains": 4096, "depth": 24, "cpu_sample": 2, "ref_sample": 1,
                 "desc": "conv_3x32x32_c64_c64_c128_c128_fc512_10 eps=2/255, {n} BaB-tree subdomains (depth<=24), "
                         "9 specs"},
}


def make_problem(workload, seed, wl):
    if workload == "batching":
        return wl.problem_mlp_784(seed=seed, n_props=64)
    if workload == "conv_small":
        return wl.problem_conv_small(seed=seed)
    if workload == "conv_big":
        return wl.problem_conv_big(seed=seed)
    return wl.problem_mlp_784(seed=seed)


def make_batch(workload, pb, unst, n_sub, seed, wl):
    w = WORKLOADS[workload]
    counts = wl.loguniform_counts(pb.P, 16, 4096, seed) if workload == "batching" else [n_sub]
    return wl.tree_batch(pb, unst, counts, w["depth"], seed + 1)


def build_workload(workload, seed, n_sub, torch, bc, wl):
    pb = make_problem(workload, seed, wl)
    net = bc.load_net(pb.layers, pb.C)
    x_lo = torch.as_tensor(pb.x_lo).cuda()
    x_hi = torch.as_tensor(pb.x_hi).cuda()
    l, u, cnt = bc.root_bounds(net, x_lo, x_hi, bc.ALPHA_ADAPTIVE, 0.5, bc.CERTIFY)
    l_h, u_h = l.cpu().numpy(), u.cpu().numpy()
    unst = [np.nonzero((l_h[p] < 0) & (u_h[p] > 0))[0] for p in range(pb.P)]
    batch = make_batch(workload, pb, unst, n_sub, seed, wl)
    dom = bc.Domain(x_lo, x_hi, l, u)
    return pb, net, dom, batch, unst, (l_h, u_h)


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_flops_per_row_pass(layers):
    """FLOPs of one backward pass of one row: the contractions of layers 1..L-1 (the last layer is
    merged with the specification into the top of the recursion): 2 d_i d_{i-1} for a fully
    connected layer, 2 C_out H_out W_out C_in k^2 for a convolution (no work on the zero padding)."""
    f = 0
    for ly in layers[:-1]:
        if ly.kind == "conv":
            cout, ho, wo = ly.out_shape
            f += 2 * cout * ho * wo * ly.in_shape[0] * ly.k * ly.k
        else:
            f += 2 * ly.d_out * ly.d_in
    return f


def layer_gemm_bytes_per_row_iter(pb, U, depth):
    """Algorithmic bytes of the BF16 layer path's GEMM launches for one row and one iteration:
    every hidden layer's Lambda (backward) and h (forward) written once and read once in BF16, x*
    written and read once (BF16), A at the unstable neurons stashed and read back (BF16), alpha
    read in both passes (FP32) and its gradient written (FP32), beta read and its gradient written
    (FP32), per split."""
    hidden = sum(int(np.prod(ly.out_shape)) for ly in pb.layers[:-1])
    d0 = int(np.prod(pb.layers[0].in_shape))
    return 8 * hidden + 4 * d0 + U * (2 + 2 + 4 + 4 + 4) + depth * 8


def tcg_bytes_per_row_iter(widths):
    """Algorithmic bytes of the layer-path GEMMs alone (BCROWN_PATH_LAYER_GATHER / IM2COL) per row
    and iteration: each hidden layer's backward contraction reads Lambda^(i) (FP32) and writes
    A^(i-1) (FP32), its forward contraction reads h^(i-1) and writes zhat^(i): 8 (d_i + d_(i-1))
    bytes per layer i = 1..L-1 (each operand element counted once, however often the gather
    re-reads it from L1)."""
    L = len(widths) - 1
    return 8 * sum(widths[i] + widths[i - 1] for i in range(1, L))


def fp32_simt_peak_tflops(sm_mhz):
    """152 SMs x 128 FP32 lanes x 2 flop per FMA x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# ------------------------------------------------------------------------------ oracle leg

def measured_traffic(name, algorithmic_bytes):
    """DRAM bytes per launch of a kernel from the committed ncu summary profiles/<name>.json, or
    None when the kernel's sources (the files it lists, hashed in order) have changed since
    those counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name + ".json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
        srcs = [os.path.join(ROOT, f) for f in rec["sources"]]
        rec["sources_sha256"], rec["dram_bytes_per_launch"]
    except (OSError, ValueError, KeyError, TypeError):
        return None   # an unreadable or older record: no measured traffic
    if not all(os.path.exists(f) for f in srcs):
        return None
    h = hashlib.sha256()
    for f in srcs:
        h.update(open(f, "rb").read())
    if h.hexdigest() != rec["sources_sha256"]:
        return None
    return {"dram_bytes_per_launch": rec["dram_bytes_per_launch"],
            "vs_algorithmic": rec["dram_bytes_per_launch"] / algorithmic_bytes,
            "from": "profiles/" + name + ".json (ncu capture of the same workload)"}


def cpu_oracle_rate(pb, lu, batch_full, n_sample, seed=0):
    """The FP64 oracle's optimise (20 iters + final bound) on a bounded sample of subdomains."""
    from oracle import bcrown_oracle as O
    from paper_2103_06624_gb300 import workloads as wl
    l_h, u_h = lu
    onet = O.OracleNet(pb.layers, pb.C)
    props = dict(x_lo=pb.x_lo, x_hi=pb.x_hi, l=l_h, u=u_h)
    _, U = O.unstable_ranks(onet, l_h, u_h)
    idx = np.arange(min(n_sample, batch_full.B))
    offs = np.concatenate([[0], np.cumsum(pb.hidden_widths)])
    subs = []
    for b in idx:
        o, c = int(batch_full.split_off[b]), int(batch_full.split_cnt[b])
        g = offs[batch_full.split_layer[o:o + c].astype(np.int64) - 1] + batch_full.split_idx[o:o + c]
        subs.append((int(batch_full.prop_of[b]), g.astype(np.int64), batch_full.split_sign[o:o + c]))
    sb = wl.pack_batch(pb.hidden_widths, pb.K, U, subs)
    a0, b0 = wl.initial_alpha_beta(sb)
    t0 = time.perf_counter()
    O.optimize(onet, props, sb, a0, b0)
    dt = time.perf_counter() - t0
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count()
    return len(idx) / dt, cores, f"{len(idx)} subdomains x {pb.K} specs, 20 iters + final bound, FP64 NumPy ({dt:.1f} s)"


# ------------------------------------------------------------------------------ main

def main():
    args = parse()
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, world)
        return

    torch.cuda.set_device(local)
    from paper_2103_06624_gb300 import bcrown as bc
    from paper_2103_06624_gb300 import workloads as wl

    prec = bc.BF16 if args.precision == "bf16" else bc.FP32
    pb, net, dom, hbatch, unst, lu = build_workload(args.workload, 0, args.subdomains, torch, bc, wl)
    if args.bab:
        measure_bab(args, torch, pb, net, dom, unst, lu)
        return
    if prec == bc.BF16:
        try:
            _probe = bc.DeviceBatch.from_host(wl.tree_batch(pb, unst, [2], 2, 0))
            a_, b_ = wl.initial_alpha_beta(wl.tree_batch(pb, unst, [2], 2, 0))
            bc.bound(net, dom, _probe, torch.as_tensor(a_).cuda(), torch.as_tensor(b_).cuda(), bc.BF16)
        except bc.BcrownError:
            prec = bc.FP32
    db = bc.DeviceBatch.from_host(hbatch)
    a0, b0 = wl.initial_alpha_beta(hbatch)
    a_init = torch.as_tensor(a0).cuda()
    b_init = torch.as_tensor(b0).cuda()
    alpha = torch.empty_like(a_init)
    beta = torch.empty_like(b_init)
    lb = torch.empty(hbatch.B * pb.K, device="cuda")
    cfg = bc.OptCfg(precision=prec, certify=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, device="cuda")
    stream = torch.cuda.current_stream()

    # ---------------------------------------------------------------- launch configuration
    # the tuner times every BF16 path (and grid) the net can take on this batch, outside the
    # timed region, and keeps the fastest for the batch's row-count bucket
    launch = None
    if prec == bc.BF16:
        if args.launch_path:
            code = {v: k for k, v in bc.N.PATH_NAMES.items()}[args.launch_path]
            bc.set_launch(net, code)
            launch = {"path": args.launch_path, "grid_per_sm": 0, "chosen_by": "--launch-path"}
        elif not args.no_autotune:
            best, cands = bc.autotune(net, dom, db, a_init, b_init, reps=2)
            launch = {"path": bc.N.PATH_NAMES[best[0]], "grid_per_sm": best[1], "chosen_by": "autotune",
                      "candidates_ms_per_bound_grad": {"%s/%d" % (bc.N.PATH_NAMES[c[0]], c[1]): ms
                                                       for c, ms in cands}}
        else:
            p_, g_ = bc.get_launch(net, hbatch.B * pb.K)
            launch = {"path": bc.N.PATH_NAMES[p_], "grid_per_sm": g_, "chosen_by": "built-in order"}

    def step():
        alpha.copy_(a_init)
        beta.copy_(b_init)
        bc.optimize(net, dom, db, alpha, beta, cfg, out=lb)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # one step captured into a CUDA graph (with the profiling scopes as event nodes), replayed
    # once per timed step; the first call above made every allocation and table the step needs
    bc.profile(net, True)
    launches0 = bc.kernel_launches()
    graph = None
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        torch.cuda.synchronize()
        launches_per_step = bc.kernel_launches() - launches0
        graph.replay()                             # untimed first replay
        torch.cuda.synchronize()
    run = graph.replay if graph is not None else step
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = bc.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    if args.profile_timed:
        torch.cuda.profiler.start()
    for i in range(args.steps):
        flush.fill_(float(i))                      # write 256 MB > L2 between timed steps
        ev[i][0].record(stream)
        run()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if args.profile_timed:
        torch.cuda.profiler.stop()
    launches = launches_per_step * args.steps if graph is not None else bc.kernel_launches() - launches0
    clk = clocks.stop()
    prof = {c: bc.profile_read(net, c) for c in range(7)}
    bc.profile(net, False)
    # with the graph, the profile holds the latest replay: one step (eager: every timed step)
    prof_steps = 1 if graph is not None else args.steps
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        tt = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    ms_per_step = t_ms / args.steps
    step_ms = sorted(a.elapsed_time(b) for a, b in ev)
    ms_median = step_ms[len(step_ms) // 2] if len(step_ms) % 2 else 0.5 * (
        step_ms[len(step_ms) // 2 - 1] + step_ms[len(step_ms) // 2])
    units = hbatch.B * world
    value = units / (ms_per_step / 1e3)
    assert bc.status(net) == 0, "device status reported an error"

    # ---------------------------------------------------------------- root bounds, once per property
    # (outside the timed step: bcrown_root_bounds in the certified precision the step uses)
    rb_ms = time_root_bounds(bc, torch, net, dom, pb.P)

    # ---------------------------------------------------------------- measured FP32 / FP64 peaks
    probes = {"fp32_tflops": bc.peak_probe(0), "fp64_tflops": bc.peak_probe(1, iters=200),
              "how": "bcrown_peak_probe: independent FMA chains, 8 x 256 threads per SM, CUDA events"}

    # ---------------------------------------------------------------- end to end (host buffers)
    # (in parts that overlap copies with compute where a step is long enough that a quarter of the
    # batch still fills the GPU; a short step runs whole, as parts would each pay its latency)
    e2e = measure_e2e(args, bc, torch, net, dom, hbatch, a0, b0, cfg, pb, world, parts=4 if ms_per_step > 50 else 1)

    # ---------------------------------------------------------------- the plain FP32 form, same GPU
    # Same workload and step (20 iterations + certifying pass) with FP32 SIMT contractions; the
    # certified bounds of both forms are compared to state the tightness at which they are equal.
    lb_main = lb.clone()
    forms = None
    if prec == bc.BF16 and not args.no_fp32_form:
        cfg32 = bc.OptCfg(precision=bc.FP32, certify=True)
        lb32 = torch.empty_like(lb)

        def step32():
            alpha.copy_(a_init)
            beta.copy_(b_init)
            bc.optimize(net, dom, db, alpha, beta, cfg32, out=lb32)

        for _ in range(3):
            step32()
        torch.cuda.synchronize()
        n32 = max(1, args.fp32_steps)
        ev32 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n32)]
        for i in range(n32):
            flush.fill_(float(i))                  # L2 flushed before every timed FP32 step
            ev32[i][0].record(stream)
            step32()
            ev32[i][1].record(stream)
        torch.cuda.synchronize()
        ms32 = sum(a.elapsed_time(b) for a, b in ev32) / n32
        d = (lb_main - lb32).double().cpu().numpy()
        forms = {"fp32": {"value": hbatch.B * world / (ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32,
                          "steps": n32, "warmup": 3, "l2": "flushed before every step"},
                 "bf16_over_fp32": (ms32 / ms_per_step),
                 "certified_lb_bf16_minus_fp32": {"mean": float(d.mean()), "min": float(d.min()),
                                                  "max": float(d.max())},
                 "mean_certified_lb": {"bf16": float(lb_main.double().mean()), "fp32": float(lb32.double().mean())}}

    # ---------------------------------------------------------------- roofline of the dominant kernel
    widths = pb.widths
    rows = hbatch.B * pb.K
    f_row = algorithmic_flops_per_row_pass(pb.layers)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    sm_mhz = clk.get("sm_mhz") or 1432.0
    if prof[5][1] > 0:
        # fused bound + adjoint kernel (one launch per Adam iteration): the data it must move are
        # the alpha/beta it reads, the gradients it writes and the bound of each row
        ms, nl = prof[5]
        U = np.array([len(u) for u in unst])[hbatch.prop_of]
        bytes_per_launch = float(np.sum(pb.K * (6 * U + 8 * hbatch.split_cnt.astype(np.int64) + 4)))
        achieved = bytes_per_launch * nl / (ms / 1e3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        tflops = rows * 2 * f_row * nl / (ms / 1e3) / 1e12
        tpeak = peaks.get("bf16_tflops_sustained", 1700.0)
        roof = {"bound": "hbm", "kernel": "k_fused<2> (tcgen05 bound + adjoint pass, one launch per iteration)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "traffic_note": None,
                "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "bytes_model": "per row: 6 B x unstable neurons (alpha read FP32, dalpha written BF16) + 8 B x "
                               "splits (beta read, dbeta write) + 4 B (lb)",
                "tensor_tflops": tflops, "tensor_frac": tflops / tpeak,
                "tensor_peak_source": "of measured (MEASURED_PEAKS.json bf16_tflops_sustained)",
                "kernel_ms_per_step": ms / prof_steps, "launches_per_step": nl / prof_steps,
                "step_ms_by_class": {n: prof[c][0] / prof_steps for c, n in enumerate(
                    ["contract", "relax", "concretize", "adjoint", "adam", "fused", "layer_gemm"])}}
        # the record was taken on the default workload at its default size
        tr = measured_traffic("k_fused_grad", bytes_per_launch) if (args.workload, args.subdomains) == (
            "mlp784", WORKLOADS["mlp784"]["subdomains"]) else None
        if tr is not None:
            roof["traffic"] = tr["dram_bytes_per_launch"]
            roof["traffic_note"] = tr
    elif prec == bc.BF16 and prof[6][1] > 0:
        # BF16 layer path (conv nets): its tcgen05 GEMM launches with fused epilogues (both passes
        # of every iteration), against the HBM roofline (bytes of the model below) and the tensor
        # roofline (the contractions' algorithmic flops); the bound is the larger fraction
        ms, nl = prof[6]
        U = np.array([len(u) for u in unst])[hbatch.prop_of].astype(np.float64)
        epi = bool(launch and launch["path"] == "layer_epi")
        if epi:
            per_row = layer_gemm_bytes_per_row_iter(pb, U, hbatch.split_cnt.astype(np.float64))
            bytes_all = float(np.sum(per_row)) * pb.K * cfg.iters * prof_steps
        else:
            bytes_all = float(tcg_bytes_per_row_iter(pb.widths)) * rows * cfg.iters * prof_steps
        flops_all = float(rows) * 2 * f_row * cfg.iters * prof_steps
        gbs = bytes_all / (ms / 1e3) / 1e9
        tfl = flops_all / (ms / 1e3) / 1e12
        peak = peaks.get("hbm_gbs", 6800.0)
        tpeak = peaks.get("bf16_tflops_sustained", 1700.0)
        hbm_frac, ten_frac = gbs / peak, tfl / tpeak
        if launch and launch["path"] == "layer_epi":
            kern = ("k_lt (tcgen05 GEMMs of the BF16 layer path, relaxation / concretisation / adjoint fused in "
                    "the epilogue)")
        else:
            kern = ("k_tcg (tcgen05 GEMMs of the BF16 layer path, conv operand gathered in shared memory or read "
                    "from an im2col buffer; relaxation and adjoint in FP32 kernels between them)")
        if hbm_frac >= ten_frac:
            roof = {"bound": "hbm", "kernel": kern, "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": hbm_frac,
                    "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)"}
        else:
            roof = {"bound": "tensor", "kernel": kern, "achieved": tfl, "peak": tpeak, "unit": "TFLOP/s",
                    "frac": ten_frac, "peak_source": "of measured (MEASURED_PEAKS.json bf16_tflops_sustained)"}
        roof.update({"traffic": None, "hbm_gbs": gbs, "hbm_frac": hbm_frac, "tensor_tflops": tfl,
                     "tensor_frac": ten_frac, "algorithmic_bytes_per_launch": bytes_all / nl,
                     "algorithmic_flops_per_launch": flops_all / nl,
                     "bytes_model": ("per row and iteration: 8 B x hidden neurons (Lambda and h, BF16, written and "
                                     "read) + 4 B x inputs (x*) + 16 B x unstable (stash 2+2, alpha 4+4, dalpha 4) + "
                                     "8 B x splits") if epi else
                                    ("per row and iteration, the GEMMs' own operands: per hidden layer i, backward "
                                     "Lambda^(i) read + A^(i-1) written, forward h^(i-1) read + zhat^(i) written, "
                                     "FP32: 8 (d_i + d_(i-1)) B"),
                     "flops_model": "2 x (backward + adjoint) contractions per row and iteration: fc 2 d_i d_(i-1), "
                                    "conv 2 C_out H_out W_out C_in k^2",
                     "kernel_ms_per_step": ms / prof_steps, "launches_per_step": nl / prof_steps,
                     "step_ms_by_class": {n: prof[c][0] / prof_steps for c, n in enumerate(
                         ["contract", "relax", "concretize", "adjoint", "adam", "fused", "layer_gemm"])}})
    else:
        ms, nl = prof[0]
        flops = rows * f_row * (2 * cfg.iters + 1) * prof_steps
        peak = probes["fp32_tflops"]
        achieved = flops / (ms / 1e3) / 1e12 if ms > 0 else None
        roof = {"bound": "alu", "kernel": "k_sgemm (FP32 SIMT contractions)", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None, "traffic": None,
                "peak_source": "of measured (bcrown_peak_probe FFMA throughput on this GPU)",
                "kernel_ms_per_step": ms / prof_steps, "launches_per_step": nl / prof_steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = cpu_oracle_rate(pb, lu, hbatch, args.cpu_sample)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        U = [len(u) for u in unst]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "ms_per_step_median": ms_median, "rows_per_s": value * pb.K,
            "vs_baseline": None, "dtype": "bf16" if prec == bc.BF16 else "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"].format(n=hbatch.B) +
                                   ", 20 Adam iters + certify pass",
                       "subdomains_per_gpu": hbatch.B, "specs": pb.K, "rows_per_gpu": rows,
                       "unstable_neurons": U, "iters": cfg.iters, "precision": args.precision if prec == bc.BF16 else "fp32",
                       "l2": "flushed (256 MB write between timed steps)",
                       "graph": "one captured CUDA graph replayed per step" if graph is not None else "eager launches",
                       "launch": launch},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "forms": forms,
            "root_bounds": {"ms_per_property": rb_ms, "precision": "certify",
                            "note": "once per property, outside the timed step"},
            "measured_peaks": probes,
        }
        if forms is not None:
            forms["fp32"]["frac_of_fp32_peak"] = (
                rows * f_row * (2 * cfg.iters + 1) / (forms["fp32"]["ms_per_step"] / 1e3) / 1e12
                / probes["fp32_tflops"]) if probes["fp32_tflops"] else None
        line["config"]["name"] = args.workload
        line["joint"] = None if args.no_joint else measure_joint(args, bc, torch, wl, probes)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def joint_flops_per_subdomain_iter(widths, K):
    """Algorithmic FLOPs of one joint iteration of one subdomain (fully connected net): for every
    target layer T = 2..L-1, 2 d_T rows back-substituted through layers T-1..1 and their adjoint
    forward pass (2 d_m d_(m-1) each per row and direction), and the K spec rows through all
    hidden layers; the backward recomputation of the target passes for the gradient included."""
    L = len(widths) - 1
    chain = [0] + [2 * widths[m] * widths[m - 1] for m in range(1, L)]   # chain[m]: one layer, one row
    f = 0
    for T in range(2, L):
        f += 2 * widths[T] * sum(chain[1:T]) * 3        # backward, recomputed backward, adjoint
    f += K * sum(chain[1:L]) * 2                        # spec rows: backward and adjoint
    return f


def measure_joint(args, bc, torch, wl, probes, iters=20):
    """Joint optimisation of intermediate bounds (Section 3.3) on the 784-256x6-10 MLP with
    args.joint_subdomains BaB-tree subdomains (FP32, 20 iterations): subdomains/s against the
    plain FP32 optimiser on the same batch, and the ablations of Table A4 -- alpha and/or beta
    optimised, joint on or off -- as the mean bound each reaches."""
    pb, net, dom, hbatch, unst, _ = build_workload("mlp784", 0, args.joint_subdomains, torch, bc, wl)
    db = bc.DeviceBatch.from_host(hbatch)
    a0, b0 = wl.initial_alpha_beta(hbatch)
    a_init, b_init = torch.as_tensor(a0).cuda(), torch.as_tensor(b0).cuda()
    ap_init, bp_init = bc.joint_init_alpha(net, dom, db)
    K, B = pb.K, hbatch.B

    def run(joint, fa=False, fb=False):
        cfg = bc.OptCfg(iters=iters, precision=bc.FP32, certify=False, freeze_alpha=fa, freeze_beta=fb)
        a, b = a_init.clone(), b_init.clone()
        if joint:
            ap, bp = ap_init.clone(), bp_init.clone()
            lb, _, _ = bc.optimize_joint(net, dom, db, a, b, ap, bp, cfg=cfg)
        else:
            lb = bc.optimize(net, dom, db, a, b, cfg)
        return lb

    def timed(joint, reps=3):
        run(joint)                                  # warm: workspace and tables
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            lb = run(joint)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), lb

    ms_joint, lb_joint = timed(True)
    ms_plain, lb_plain = timed(False)
    assert bc.status(net) == 0, "device status reported an error (joint)"
    flops = joint_flops_per_subdomain_iter(pb.widths, K) * B * iters
    tfl = flops / (ms_joint / 1e3) / 1e12
    ablation = {}
    for joint in (False, True):
        for name, fa, fb in (("alpha", False, True), ("beta", True, False), ("alpha+beta", False, False)):
            lb = run(joint, fa, fb).double().cpu().numpy()
            ablation[("joint " if joint else "") + name] = {"mean_lb": float(lb.mean()),
                                                             "verified_rows": int((lb > 0).sum())}
    assert bc.status(net) == 0, "device status reported an error (ablation)"
    return {"workload": "mlp_784_256x6_10 eps=0.015, %d BaB-tree subdomains (depth<=12), 9 specs, 20 Adam iters, "
                        "FP32, intermediate bounds of layers 2-6 recomputed per subdomain" % B,
            "value": B / (ms_joint / 1e3), "unit": UNIT, "ms_per_step": ms_joint,
            "plain_fp32": {"value": B / (ms_plain / 1e3), "ms_per_step": ms_plain},
            "mean_lb": {"joint": float(lb_joint.double().mean()), "plain": float(lb_plain.double().mean())},
            "roofline": {"bound": "alu", "achieved": tfl, "peak": probes["fp32_tflops"], "unit": "TFLOP/s",
                         "frac": tfl / probes["fp32_tflops"] if probes["fp32_tflops"] else None,
                         "scope": "the whole joint optimisation (SIMT GEMMs and epilogues), algorithmic FLOPs "
                                  "(joint_flops_per_subdomain_iter) over its CUDA-event time",
                         "peak_source": "of measured (bcrown_peak_probe FFMA throughput)"},
            "ablation_table_A4": ablation}


def measure_bab(args, torch, pb, net, dom, unst, lu):
    """Branch and bound on property 0 for a fixed number of rounds (no sampling, no descent, no line
    search, so the pool grows to the batch size): wall time of each driver, the time spent inside its
    engine calls (each ends with a device synchronisation), and the rest -- the driver's host time --
    per bounded child.  Prints one JSON line."""
    from paper_2103_06624_gb300 import bab, bab_pool

    class Timed(bab.GpuEngine):
        t = 0.0

        def _timed(self, f, *a, **k):
            t0 = time.perf_counter()
            r = f(*a, **k)
            torch.cuda.synchronize()
            self.t += time.perf_counter() - t0
            return r

        def optimize(self, *a, **k):
            return self._timed(super().optimize, *a, **k)

        def xstar(self, *a, **k):
            return self._timed(super().xstar, *a, **k)

        def optimize_rows(self, *a, **k):
            return self._timed(super().optimize_rows, *a, **k)

        def xstar_rows(self, *a, **k):
            return self._timed(super().xstar_rows, *a, **k)

    case = (0, lu[0][0], lu[1][0], pb.x_lo[0], pb.x_hi[0])
    out = {}
    for name, fn, graphs in (("array_pool", bab_pool.bab_pool, False), ("list_pool", bab.bab_many, False),
                             ("array_pool_graphs", bab_pool.bab_pool, True), ("list_pool_graphs", bab.bab_many, True)):
        eng = Timed(pb, net, dom, [len(unst[0])], graphs=graphs)
        for rep in range(2):   # the first run warms up (library workspaces, launch tuning, graph captures)
            eng.t = 0.0
            t0 = time.perf_counter()
            r = fn(eng, [case], batch_size=args.bab_batch, max_rounds=args.bab_rounds, n_samples=0, pgd_steps=0,
                   line_search=False)[0]
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        out[name] = {"rounds": r.rounds, "bounded": r.bounded, "status": r.status, "wall_s": wall,
                     "engine_s": eng.t, "host_us_per_child": 1e6 * (wall - eng.t) / max(1, r.bounded),
                     "engine_us_per_child": 1e6 * eng.t / max(1, r.bounded)}
    print(json.dumps({"bab": out, "workload": pb.name, "batch_size": args.bab_batch, "K": pb.K,
                      "unstable": int(len(unst[0])), "engine": "BF16 iterations (20) + FP32 certifying pass, "
                      "x* and f(x*) per child"}))


def time_root_bounds(bc, torch, net, dom, P, reps=3):
    """Device milliseconds per property of bcrown_root_bounds (CROWN intermediate bounds with the
    outward-rounded arithmetic), median of reps calls after one warm-up."""
    x_lo, x_hi = dom.x_lo, dom.x_hi
    bc.root_bounds(net, x_lo, x_hi, bc.ALPHA_ADAPTIVE, 0.5, bc.CERTIFY)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bc.root_bounds(net, x_lo, x_hi, bc.ALPHA_ADAPTIVE, 0.5, bc.CERTIFY)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts) / P


def _split_host_batch(hbatch, K, parts):
    """Contiguous ranges of subdomains as batches of their own (offsets rebased), with the slices
    of the alpha and beta arrays they own: [(batch, (a0, a1), (s0, s1)), ...]."""
    from paper_2103_06624_gb300 import workloads as wl
    B = hbatch.B
    cuts = [round(B * j / parts) for j in range(parts + 1)]
    out = []
    for b0, b1 in zip(cuts[:-1], cuts[1:]):
        if b1 <= b0:
            continue
        s0 = int(hbatch.split_off[b0])
        s1 = int(hbatch.split_off[b1 - 1]) + int(hbatch.split_cnt[b1 - 1])
        a0 = int(hbatch.alpha_off[b0])
        a1 = int(hbatch.alpha_off[b1]) if b1 < B else int(hbatch.n_alpha)
        sub = wl.Batch(hbatch.prop_of[b0:b1].copy(), (hbatch.split_off[b0:b1] - s0).astype(np.int32),
                       hbatch.split_cnt[b0:b1].copy(), hbatch.split_layer[s0:s1].copy(),
                       hbatch.split_idx[s0:s1].copy(), hbatch.split_sign[s0:s1].copy(),
                       (hbatch.alpha_off[b0:b1] - a0).astype(np.int64), a1 - a0, (s1 - s0) * K)
        out.append((sub, (b0, b1), (a0, a1), (s0 * K, s1 * K)))
    return out


def measure_e2e(args, bc, torch, net, dom, hbatch, a0, b0, cfg, pb, world, parts=4):
    """Same metric through the public API with HOST buffers: each step copies the batch, alpha and
    beta in from pinned memory and reads lb, alpha, beta back.  The batch goes as `parts`
    contiguous ranges of subdomains, one bcrown_optimize call each, so that copies overlap
    compute: every part's inputs are copied in on one stream, each part is optimised on a second
    stream once its inputs are in, and its results are copied out on a third while the next part
    is optimised.  The timed region spans the first copy in to the last copy out."""
    K = pb.K
    subs = _split_host_batch(hbatch, K, parts)
    ha = torch.from_numpy(a0).pin_memory()
    hb = torch.from_numpy(b0).pin_memory()
    out_lb = torch.empty(hbatch.B * K).pin_memory()
    out_a = torch.empty_like(ha).pin_memory()
    out_b = torch.empty_like(hb).pin_memory()
    P = []
    for sub, (c0, c1), (x0, x1), (y0, y1) in subs:
        host = {}
        for name in ["prop_of", "split_off", "split_cnt", "split_layer", "split_idx", "split_sign", "alpha_off"]:
            arr = np.ascontiguousarray(getattr(sub, name))
            if name == "split_idx":
                arr = arr.astype(np.int32)
            host[name] = torch.from_numpy(arr).pin_memory()
        dev = {k: torch.empty(v.shape, dtype=v.dtype, device="cuda") for k, v in host.items()}
        P.append(dict(sub=sub, host=host, dev=dev, ha=ha[x0:x1], hb=hb[y0:y1], oa=out_a[x0:x1], ob=out_b[y0:y1],
                      olb=out_lb[c0 * K:c1 * K], da=torch.empty(x1 - x0, device="cuda"),
                      db=torch.empty(y1 - y0, device="cuda"), lb=torch.empty((c1 - c0) * K, device="cuda"),
                      ev_in=torch.cuda.Event(), ev_c=torch.cuda.Event(), ev_out=torch.cuda.Event()))
    h2d = sum(v.numel() * v.element_size() for p in P for v in p["host"].values()) + ha.numel() * 4 + hb.numel() * 4
    d2h = out_lb.numel() * 4 + out_a.numel() * 4 + out_b.numel() * 4
    s_in, s_c, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    # the parts' row-count bucket takes the tuner's choice on the first part (the whole batch's
    # bucket was tuned before)
    for p in P[:1]:
        for k in p["dev"]:
            p["dev"][k].copy_(p["host"][k])
        p["da"].copy_(p["ha"])
        p["db"].copy_(p["hb"])
        b = bc.DeviceBatch(p["dev"]["prop_of"], p["dev"]["split_off"], p["dev"]["split_cnt"], p["dev"]["split_layer"],
                           p["dev"]["split_idx"], p["dev"]["split_sign"], p["dev"]["alpha_off"], p["sub"].n_alpha,
                           p["sub"].n_beta)
        if not args.launch_path and not args.no_autotune:
            bc.autotune(net, dom, b, p["da"], p["db"], reps=2)

    def step():
        for p in P:
            with torch.cuda.stream(s_in):
                s_in.wait_event(p["ev_out"])   # the previous step's copies out of this part's buffers
                for k in p["dev"]:
                    p["dev"][k].copy_(p["host"][k], non_blocking=True)
                p["da"].copy_(p["ha"], non_blocking=True)
                p["db"].copy_(p["hb"], non_blocking=True)
                p["ev_in"].record(s_in)
        for p in P:
            s_c.wait_event(p["ev_in"])
            d = p["dev"]
            b = bc.DeviceBatch(d["prop_of"], d["split_off"], d["split_cnt"], d["split_layer"], d["split_idx"],
                               d["split_sign"], d["alpha_off"], p["sub"].n_alpha, p["sub"].n_beta)
            bc.optimize(net, dom, b, p["da"], p["db"], cfg, out=p["lb"], stream=s_c)
            p["ev_c"].record(s_c)
            with torch.cuda.stream(s_out):
                s_out.wait_event(p["ev_c"])
                p["olb"].copy_(p["lb"], non_blocking=True)
                p["oa"].copy_(p["da"], non_blocking=True)
                p["ob"].copy_(p["db"], non_blocking=True)
                p["ev_out"].record(s_out)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(3, args.steps // 2)
    cur = torch.cuda.current_stream()
    s.record(cur)
    s_in.wait_stream(cur)
    for _ in range(n):
        step()
    for p in P:
        cur.wait_event(p["ev_out"])
    e.record(cur)
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / n
    assert bc.status(net) == 0, "device status reported an error"
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    return {"value": hbatch.B * world / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms, "parts": len(P),
            "overlap": ("inputs copied in on one stream, parts optimised on a second, results copied out on a third"
                        if len(P) > 1 else "none: one part, copies in, optimisation and copies out in sequence")}


def run_reference(args, world):
    """The oracle (FP64 NumPy) timed on the host cores, on a bounded sample of the same workload."""
    import torch
    from oracle import bcrown_oracle as O
    from paper_2103_06624_gb300 import workloads as wl
    pb = make_problem(args.workload, 0, wl)
    onet = O.OracleNet(pb.layers, pb.C)
    # CROWN root bounds; for the 123k-neuron conv net the oracle's interval bounds (valid, looser)
    l, u = (O.interval_bounds if args.workload == "conv_big" else O.root_bounds)(onet, pb.x_lo, pb.x_hi)
    l, u = l.astype(np.float32), u.astype(np.float32)
    unst = [np.nonzero((l[p] < 0) & (u[p] > 0))[0] for p in range(pb.P)]
    batch = make_batch(args.workload, pb, unst, args.subdomains, 0, wl)
    times = []
    rate = None
    n_ref = WORKLOADS[args.workload]["ref_sample"]
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rate, cores, sample = cpu_oracle_rate(pb, (l, u), batch, n_ref)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = n_ref / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"].format(n=batch.B) +
                                   ", 20 Adam iters + final bound", "sample_subdomains": n_ref,
                       "name": args.workload},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    _ = torch
    print(json.dumps(line))


if __name__ == "__main__":
    main()
