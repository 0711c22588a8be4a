"""The stride-phase decomposition of the transposed convolution (no GPU).

The backward contraction of a conv layer, A^(i-1) = Lambda^(i) W^(i), is the adjoint of the
convolution.  The tensor-core path computes it per stride phase: input positions
p = (a + s i, b + s j) receive only the taps ky = ky0(a) + s dy, kx = kx0(b) + s dx, from the
source positions (i + off(a) - dy, j + off(b) - dx).  This test restates those index formulas
(as the library's gather tables use them) and checks that the phase GEMMs reproduce the adjoint
that torch's autograd computes for conv2d, for strides 1-3, paddings 0-2 and odd map sizes."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F


def phase(a, k, s, pad, n_in):
    """(k0, taps, off, positions) of phase a along one axis."""
    k0 = (a + pad) % s
    nk = (k - k0 + s - 1) // s if k0 < k else 0
    off = (a + pad - k0) // s
    n = (n_in - a + s - 1) // s if a < n_in else 0
    return k0, nk, off, n


def transposed_by_phases(lam, W, s, pad, h, w):
    R, cout, ho, wo = lam.shape
    cin, k = W.shape[1], W.shape[2]
    T = (k + s - 1) // s
    out = np.full((R, cin, h, w), np.nan)
    for a in range(s):
        for b in range(s):
            ky0, nky, offa, nI = phase(a, k, s, pad, h)
            kx0, nkx, offb, nJ = phase(b, k, s, pad, w)
            if nI * nJ == 0:
                continue
            # gather table over K = (co, dy, dx) and the phase's weight matrix
            col = np.zeros((R, nI, nJ, cout * T * T))
            Wb = np.zeros((cin, cout * T * T))
            for co in range(cout):
                for dy in range(nky):
                    for dx in range(nkx):
                        K = co * T * T + dy * T + dx
                        Wb[:, K] = W[co, :, ky0 + s * dy, kx0 + s * dx]
                        for i in range(nI):
                            for j in range(nJ):
                                y, x = i + offa - dy, j + offb - dx
                                if 0 <= y < ho and 0 <= x < wo:
                                    col[:, i, j, K] = lam[:, co, y, x]
            res = col @ Wb.T                                    # [R, nI, nJ, cin]
            for i in range(nI):
                for j in range(nJ):
                    out[:, :, a + s * i, b + s * j] = res[:, i, j, :]
    return out


@pytest.mark.parametrize("cin,h,w,cout,k,s,pad", [
    (3, 12, 12, 4, 4, 2, 1),    # 4x4 stride 2 (the small conv net's layers)
    (3, 12, 12, 4, 3, 1, 1),    # 3x3 stride 1
    (4, 12, 12, 4, 3, 2, 1),    # 3x3 stride 2 (the large conv net's strided layers)
    (4, 11, 13, 4, 3, 2, 1),    # odd map sizes: phases of unequal size
    (2, 9, 8, 3, 5, 3, 2),      # stride 3: nine phases
    (2, 10, 10, 3, 2, 2, 0),    # kernel as wide as the stride
    (2, 7, 7, 3, 3, 1, 0),      # no padding
])
def test_phase_gemms_reproduce_the_conv_adjoint(cin, h, w, cout, k, s, pad):
    ho, wo = (h + 2 * pad - k) // s + 1, (w + 2 * pad - k) // s + 1
    rng = np.random.default_rng(cin * 100 + k * 10 + s)
    W = rng.standard_normal((cout, cin, k, k))
    lam = rng.standard_normal((2, cout, ho, wo))
    x = torch.zeros((2, cin, h, w), dtype=torch.float64, requires_grad=True)
    (F.conv2d(x, torch.tensor(W), stride=s, padding=pad) * torch.tensor(lam)).sum().backward()
    got = transposed_by_phases(lam, W, s, pad, h, w)
    assert not np.isnan(got).any()          # the phases cover every input position once
    np.testing.assert_allclose(got, x.grad.numpy(), rtol=1e-12, atol=1e-12)
