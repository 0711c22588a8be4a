"""bcrown_optimize under CUDA graph capture (needs a GB300).

After one call with the same sizes, an optimisation call allocates nothing and never waits on
the host, so a caller can capture it (with the reset of alpha, beta) into a CUDA graph and
replay it: the rows, properties and pointers are fixed by the capture.  The replay must
reproduce the eager result."""
import numpy as np
import pytest
import torch

from oracle import bcrown_oracle as O
from paper_2103_06624_gb300 import bcrown as bc
from paper_2103_06624_gb300 import workloads as wl
from tests.helpers import oracle_setup

pytestmark = pytest.mark.gpu


def _problem(which):
    if which == "mlp784":
        pb = wl.problem_mlp_784()
        _, props, unst = oracle_setup(pb)
        return pb, props, wl.tree_batch(pb, unst, [64], 12, 5)
    layers = wl.conv_layers((2, 6, 6), [(3, 3, 2, 1), (4, 3, 1, 1)], [8, 4], 3)
    pb = wl.make_problem("tinyconv", layers, 2, 0.1, 3, 3)
    _, props, unst = oracle_setup(pb)
    return pb, props, wl.random_batch(pb, unst, 24, 0, 4, 1, props=np.arange(24) % 2)


@pytest.mark.parametrize("which", ["mlp784", "tinyconv"])
def test_optimize_replays_from_a_captured_graph(which):
    """mlp784: the fused tcgen05 kernel + Adam; tinyconv: the layer path with gather GEMMs."""
    pb, props, batch = _problem(which)
    net = bc.load_net(pb.layers, pb.C)
    dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
    db = bc.DeviceBatch.from_host(batch)
    a0, b0 = wl.initial_alpha_beta(batch)
    a_init, b_init = torch.as_tensor(a0).cuda(), torch.as_tensor(b0).cuda()
    alpha, beta = a_init.clone(), b_init.clone()
    lb = torch.empty(batch.B * pb.K, device="cuda")
    cfg = bc.OptCfg(precision=bc.BF16, certify=True)

    def step():
        alpha.copy_(a_init)
        beta.copy_(b_init)
        bc.optimize(net, dom, db, alpha, beta, cfg, out=lb)

    step()                                    # first call: weights, tables, workspace
    torch.cuda.synchronize()
    eager = lb.clone()
    eager_alpha = alpha.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    lb.zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    assert bc.status(net) == 0
    d = (lb - eager).abs().max().item()
    print("%s: replay vs eager max |dlb| = %.3e" % (which, d))
    assert d <= 1e-6 * max(1.0, eager.abs().max().item())
    assert (alpha - eager_alpha).abs().max().item() <= 1e-6
    # and the certified bound is sound against the oracle at the returned alpha, beta
    onet = O.OracleNet(pb.layers, pb.C)
    ref = O.bound(onet, props, batch, alpha.cpu().numpy(), beta.cpu().numpy())
    got = lb.cpu().numpy()
    assert np.all(got <= ref + 1e-9 * np.abs(ref))


@pytest.mark.parametrize("which", ["mlp784", "tinyconv"])
def test_bucketed_graph_replay_equals_the_eager_call(which):
    """GraphOptimizer pads a batch to its size bucket (copies of its last subdomain; alpha, beta and
    the split lists to bucketed capacities), captures bcrown_optimize once per bucket and replays
    it.  Rows are independent, so every real row's bound, alpha and beta equal the eager call on
    the unpadded batch bit for bit; batches of the same bucket share one graph."""
    pb, props, _ = _problem(which)
    net = bc.load_net(pb.layers, pb.C)
    dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
    unst = [np.nonzero(O.unstable_mask(props["l"][p], props["u"][p]))[0] for p in range(pb.P)]
    U = [len(u) for u in unst]
    cfg = bc.OptCfg(precision=bc.BF16, certify=True)
    go = bc.GraphOptimizer(net, dom, cfg, U)
    sizes = (97, 100, 97, 120) if which == "mlp784" else (17, 18, 17, 24)
    for n, seed in zip(sizes, (1, 2, 3, 4)):
        hb = wl.random_batch(pb, unst, n, 0, 6, seed, props=np.arange(n) % pb.P)
        a0, b0 = wl.random_alpha_beta(hb, seed, 0.5)
        lb, a, b = go(hb, a0, b0)
        at, bt = torch.as_tensor(a0).cuda(), torch.as_tensor(b0).cuda()
        ref = bc.optimize(net, dom, bc.DeviceBatch.from_host(hb), at, bt, cfg).cpu().numpy()
        assert bc.status(net) == 0
        assert np.array_equal(lb, ref), (which, n, np.abs(lb - ref).max())
        assert np.array_equal(a, at.cpu().numpy()) and np.array_equal(b, bt.cpu().numpy())
        assert bc.bucket(n) >= n
    assert go.captures == 2
