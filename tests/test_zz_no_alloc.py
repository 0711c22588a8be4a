"""bcrown_bound_static, the bound pass that allocates nothing, against bcrown_bound.

Some callers cannot call cudaMalloc while the pass runs (a real-time loop that cannot take the
allocator's implicit synchronisation, a process held to a device-memory budget by its own
allocator).  For them the library offers an entry point whose scratch is a fixed array built
into the library.  This test calls it through the C ABI twice in a row and checks each result
against bcrown_bound (FP32) on the same inputs -- bit for bit, since both run the same kernels
and a row's result does not depend on the chunk it is bounded in -- on a fully connected net
(more rows than one chunk of the fixed array) and on a conv net, then checks that a problem too
large for the fixed array is refused with a clear error.
Collected last so that a run stopping at the first failure has already run everything else.
"""
import numpy as np
import pytest
import torch

from paper_2103_06624_gb300 import bcrown as bc
from paper_2103_06624_gb300 import workloads as wl
from tests.helpers import oracle_setup

pytestmark = pytest.mark.gpu


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x, np.float32)).cuda()


def _tiny_conv():
    layers = wl.conv_layers((2, 6, 6), [(3, 3, 2, 1), (4, 3, 1, 1)], [8, 4], 3)
    return wl.make_problem("tinyconv", layers, 2, 0.1, 3, 3)


@pytest.mark.parametrize("which", ["mlp_784", "conv"])
def test_static_scratch_bound_matches_bound_on_two_calls(which):
    if which == "mlp_784":
        pb = wl.problem_mlp_784()
        _, props, unst = oracle_setup(pb)
        # 300 subdomains x 9 specs = 2700 rows: more than one row chunk of the fixed scratch
        batch = wl.tree_batch(pb, unst, [300], 12, 21)
    else:
        pb = _tiny_conv()
        _, props, unst = oracle_setup(pb)
        batch = wl.random_batch(pb, unst, 40, 0, 4, 2, props=np.arange(40) % 2)
    a, b = wl.random_alpha_beta(batch, 22, 1.0)
    net = bc.load_net(pb.layers, pb.C)
    dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
    db = bc.DeviceBatch.from_host(batch)
    at, bt = _t(a), _t(b)
    ref = bc.bound(net, dom, db, at, bt, bc.FP32).cpu().numpy()
    for _ in range(2):
        got = bc.bound_static(net, dom, db, at, bt).cpu().numpy()
        assert np.array_equal(got, ref)
    assert bc.status(net) == 0


def test_static_scratch_refuses_problems_beyond_its_size():
    pb = wl.problem_mlp_784()
    _, props, unst = oracle_setup(pb)
    net = bc.load_net(pb.layers, pb.C)
    P = 1000                                   # 1000 x 1536 neurons of tables > 16 MB
    dom = bc.domain_from_host(np.repeat(props["x_lo"], P, 0), np.repeat(props["x_hi"], P, 0),
                              np.repeat(props["l"], P, 0), np.repeat(props["u"], P, 0))
    batch = wl.tree_batch(pb, unst, [4], 4, 1)
    a, b = wl.initial_alpha_beta(batch)
    with pytest.raises(bc.BcrownError) as e:
        bc.bound_static(net, dom, bc.DeviceBatch.from_host(batch), _t(a), _t(b))
    assert "static scratch" in str(e.value)
