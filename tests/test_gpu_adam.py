"""Projected Adam (Eq. opt_alpha_beta; Appendix C.1) on the GPU against the oracle's step, element by
element, and resuming an ascent across calls (needs a GB300).

One optimiser iteration is run through bcrown_optimize from a chosen state (iterate, moments,
best bounds, iteration count t).  The expected state is the oracle's loop body (oracle.optimize:
keep the best lb and theta per row, then oracle.adam_ascent_step with lr0 * decay^t) applied to the
gradient the GPU computes at that iterate (bcrown_bound_grad; the same kernels and arithmetic as
inside the iteration), so every alpha, beta, moment and best-tracking decision is compared one by
one without the sign sensitivity of Adam's first step to gradient rounding."""
import numpy as np
import pytest
import torch

from oracle import bcrown_oracle as O
from paper_2103_06624_gb300 import bcrown as bc
from paper_2103_06624_gb300 import workloads as wl
from tests.helpers import oracle_setup

pytestmark = pytest.mark.gpu


def _t(x):
    return torch.as_tensor(np.ascontiguousarray(x, np.float32)).cuda()


def _bf16(x):
    """Round to BF16 (nearest even) and widen to float64: the rounding the BF16 optimiser applies."""
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _case(which):
    if which == "conv":
        layers = wl.conv_layers((2, 6, 6), [(3, 3, 2, 1), (4, 3, 1, 1)], [8, 4], 3)
        pb = wl.make_problem("tinyconv", layers, 2, 0.1, 3, 3)
        onet, props, unst = oracle_setup(pb)
        batch = wl.random_batch(pb, unst, 24, 0, 4, 1, props=np.arange(24) % 2)
    else:
        pb = wl.problem_mlp_784()
        onet, props, unst = oracle_setup(pb)
        batch = wl.tree_batch(pb, unst, [64], 12, 5)
    net = bc.load_net(pb.layers, pb.C)
    dom = bc.domain_from_host(props["x_lo"], props["x_hi"], props["l"], props["u"])
    return pb, onet, props, unst, batch, net, dom, bc.DeviceBatch.from_host(batch)


@pytest.mark.parametrize("path", ["fp32", "bf16_fused", "bf16_layer"])
@pytest.mark.parametrize("t", [0, 7])
def test_adam_step_elementwise(path, t):
    pb, onet, props, unst, batch, net, dom, db = _case("conv" if path == "bf16_layer" else "784")
    prec = bc.FP32 if path == "fp32" else bc.BF16
    bf16_moments = path == "bf16_fused"      # the fused path keeps alpha's gradient and moments in BF16
    rng = np.random.default_rng(10 + t)
    na, nb, R = batch.n_alpha, batch.n_beta, batch.B * pb.K
    th_a = rng.uniform(0, 1, na).astype(np.float32)
    th_b = rng.uniform(0, 1, nb).astype(np.float32)
    # the GPU's gradient and bound at the iterate (the point the iteration evaluates)
    lb_t, ga, gb = bc.bound_grad(net, dom, db, _t(th_a), _t(th_b), prec)
    lb_t, ga, gb = (x.cpu().numpy().astype(np.float64) for x in (lb_t, ga, gb))
    if bf16_moments:
        ga = _bf16(ga)
    st = bc.OptState(db, pb.K)
    if t == 0:
        m_a = v_a = np.zeros(na)
        m_b = v_b = np.zeros(nb)
        best_in = np.full(R, -np.inf)
        a_best_in, b_best_in = th_a.astype(np.float64), th_b.astype(np.float64)
    else:
        m_a = rng.normal(0, 0.05, na).astype(np.float32).astype(np.float64)
        v_a = rng.uniform(1e-4, 1e-2, na).astype(np.float32).astype(np.float64)
        m_b = rng.normal(0, 0.05, nb).astype(np.float32).astype(np.float64)
        v_b = rng.uniform(1e-4, 1e-2, nb).astype(np.float32).astype(np.float64)
        # about half the rows improve on their best bound at this iterate
        best_in = (lb_t + rng.normal(0, 0.5, R) * np.maximum(np.abs(lb_t), 1) * 1e-3).astype(np.float32).astype(np.float64)
        a_best_in = rng.uniform(0, 1, na).astype(np.float32).astype(np.float64)
        b_best_in = rng.uniform(0, 1, nb).astype(np.float32).astype(np.float64)
        st.alpha_cur.copy_(_t(th_a))
        st.beta_cur.copy_(_t(th_b))
        st.m_alpha.copy_(_t(m_a))
        st.v_alpha.copy_(_t(v_a))
        st.m_beta.copy_(_t(m_b))
        st.v_beta.copy_(_t(v_b))
        st.best_lb.copy_(_t(best_in))
        st.t = t
    alpha, beta = _t(a_best_in), _t(b_best_in)
    bc.optimize(net, dom, db, alpha, beta, bc.OptCfg(iters=1, precision=prec, certify=False), state=st)
    assert bc.status(net) == 0 and st.t == t + 1

    # expected: the oracle's loop body, with the hyper-parameters the C ABI receives (FP32 values)
    f32 = lambda x: float(np.float32(x))
    d = O.AdamCfg()
    cfg = O.AdamCfg(iters=d.iters, lr_alpha=f32(d.lr_alpha), lr_beta=f32(d.lr_beta), decay=f32(d.decay),
                    beta1=f32(d.beta1), beta2=f32(d.beta2), eps=f32(d.eps))
    _, U = O.unstable_ranks(onet, props["l"], props["u"])
    ra, rb = O.row_of_params(onet, batch, U)
    improved = lb_t > best_in
    if bf16_moments:
        m_a, v_a = _bf16(m_a), _bf16(v_a)
    fac = cfg.decay ** t
    a1, ma1, va1 = O.adam_ascent_step(th_a.astype(np.float64), m_a, v_a, ga, t, cfg.lr_alpha * fac, cfg, 0.0, 1.0)
    b1, mb1, vb1 = O.adam_ascent_step(th_b.astype(np.float64), m_b, v_b, gb, t, cfg.lr_beta * fac, cfg, 0.0, np.inf)

    got = {k: getattr(st, k).cpu().numpy().astype(np.float64)
           for k in ("alpha_cur", "beta_cur", "m_alpha", "v_alpha", "m_beta", "v_beta", "best_lb")}
    # best tracking: copies, bit for bit
    assert np.array_equal(got["best_lb"], np.where(improved, lb_t, best_in).astype(np.float32))
    assert np.array_equal(alpha.cpu().numpy(), np.where(improved[ra], th_a, a_best_in).astype(np.float32))
    assert np.array_equal(beta.cpu().numpy(), np.where(improved[rb], th_b, b_best_in).astype(np.float32))
    # Moments and the step: FP32 arithmetic against FP64.  A moment is a sum of two terms that may
    # cancel, so its rounding error is bounded by a few FP32 units of the terms' magnitudes (one
    # BF16 unit of the result more where the moment is stored in BF16).  The step's error follows
    # from the moments' through lr * mhat / (sqrt(vhat) + eps).
    u32 = 2.0 ** -24

    def check_moments(m_got, v_got, m_in, v_in, g, m_exp, v_exp, bf16):
        rt = 2.0 ** -8 if bf16 else 0.0
        mterm = cfg.beta1 * np.abs(m_in) + (1 - cfg.beta1) * np.abs(g)
        vterm = cfg.beta2 * v_in + (1 - cfg.beta2) * g * g
        assert np.all(np.abs(m_got - m_exp) <= 8 * u32 * mterm + rt * np.abs(m_exp) + 1e-30)
        assert np.all(np.abs(v_got - v_exp) <= 8 * u32 * vterm + rt * np.abs(v_exp) + 1e-30)
        return mterm, vterm

    def check_step(th_got, th_in, th_exp, m_exp, v_exp, mterm, vterm, lr, lo, hi):
        b1c, b2c = 1 - cfg.beta1 ** (t + 1), 1 - cfg.beta2 ** (t + 1)
        den = np.sqrt(v_exp / b2c) + cfg.eps
        step = lr * (m_exp / b1c) / den
        # first-order error of the step from the moments' and the division's rounding
        err = lr / b1c * (8 * u32 * mterm) / den + np.abs(step) * (8 * u32 * vterm / np.maximum(v_exp, 1e-300) + 16 * u32)
        tol = err + 4 * u32 * (np.abs(th_in) + np.abs(step)) + 1e-12
        # the projection can only shrink a difference
        assert np.all(np.abs(th_got - th_exp) <= tol), np.max(np.abs(th_got - th_exp) - tol)

    ma_t, va_t = check_moments(got["m_alpha"], got["v_alpha"], m_a, v_a, ga, ma1, va1, bf16_moments)
    mb_t, vb_t = check_moments(got["m_beta"], got["v_beta"], m_b, v_b, gb, mb1, vb1, False)
    check_step(got["alpha_cur"], th_a.astype(np.float64), a1, ma1, va1, ma_t, va_t, cfg.lr_alpha * fac, 0, 1)
    check_step(got["beta_cur"], th_b.astype(np.float64), b1, mb1, vb1, mb_t, vb_t, cfg.lr_beta * fac, 0, np.inf)
    # a planted slip in the step's schedule is far outside these tolerances: the decay one
    # iteration off moves the iterate by about lr * 2 %
    a_off, _, _ = O.adam_ascent_step(th_a.astype(np.float64), m_a, v_a, ga, t, cfg.lr_alpha * cfg.decay ** (t + 1),
                                     cfg, 0.0, 1.0)
    moved = np.abs(a_off - a1) > 1e-5
    assert moved.sum() >= 100 and np.all(np.abs(got["alpha_cur"] - a_off)[moved] > 1e-6)


@pytest.mark.parametrize("path", ["fp32", "bf16_fused", "bf16_layer"])
def test_resumed_ascent_equals_one_uninterrupted_run(path):
    """20 iterations in one call, and 7 + 13 iterations in two calls through the state, give the same
    best alpha, beta and certified bounds bit for bit (checkpoint / resume of the ascent)."""
    pb, onet, props, unst, batch, net, dom, db = _case("conv" if path == "bf16_layer" else "784")
    prec = bc.FP32 if path == "fp32" else bc.BF16
    a0, b0 = wl.initial_alpha_beta(batch)
    a1, b1 = _t(a0), _t(b0)
    lb1 = bc.optimize(net, dom, db, a1, b1, bc.OptCfg(iters=20, precision=prec))
    a2, b2 = _t(a0), _t(b0)
    st = bc.OptState(db, pb.K)
    bc.optimize(net, dom, db, a2, b2, bc.OptCfg(iters=7, precision=prec), state=st)
    assert st.t == 7
    lb2 = bc.optimize(net, dom, db, a2, b2, bc.OptCfg(iters=13, precision=prec), state=st)
    assert st.t == 20 and bc.status(net) == 0
    assert torch.equal(a1, a2) and torch.equal(b1, b2) and torch.equal(lb1, lb2)
