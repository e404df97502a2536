"""Pins of the learned preconditioner's CPU oracle (``oracle/convnet.py``) to definitions outside it.

The network, loss and Adam step are not in the paper (it only uses right preconditioning, Sec. 5.3);
they are pinned to an independent convolution (SciPy), to adjointness identities, to finite
differences of the loss, and to Adam's first-step closed form.
"""
import numpy as np
import pytest
from scipy import signal

import scipy.sparse as sp

import synth
from oracle import convnet as oc


def rng(seed=0):
    return np.random.default_rng(seed)


def test_num_params():
    assert oc.num_params() == 608 + 4 * 9248 + 289 == 37889


def test_conv_matches_scipy_correlate2d():
    g = rng(1)
    x = g.standard_normal((2, 3, 9, 11))
    W = g.standard_normal((4, 3, 3, 3))
    b = g.standard_normal(4)
    out = oc.conv3x3(x, W, b)
    for n in range(2):
        for co in range(4):
            ref = b[co] + sum(signal.correlate2d(x[n, ci], W[co, ci], mode="same", boundary="fill")
                              for ci in range(3))
            assert np.allclose(out[n, co], ref, rtol=0, atol=1e-12)


def test_conv_identity_and_shift_kernels():
    g = rng(2)
    x = g.standard_normal((1, 2, 6, 7))
    W = np.zeros((2, 2, 3, 3))
    W[0, 0, 1, 1] = W[1, 1, 1, 1] = 1.0
    assert np.array_equal(oc.conv3x3(x, W), x)
    # tap (dy, dx) = (0, 2) reads in[y - 1, x + 1]: shift down by one row and left by one column
    W = np.zeros((1, 2, 3, 3))
    W[0, 1, 0, 2] = 1.0
    out = oc.conv3x3(x, W)[0, 0]
    ref = np.zeros((6, 7))
    ref[1:, :-1] = x[0, 1, :-1, 1:]
    assert np.array_equal(out, ref)


def test_input_grad_is_adjoint():
    g = rng(3)
    x = g.standard_normal((2, 3, 8, 10))
    W = g.standard_normal((5, 3, 3, 3))
    d = g.standard_normal((2, 5, 8, 10))
    lhs = np.sum(oc.conv3x3(x, W) * d)
    rhs = np.sum(x * oc.conv3x3_input_grad(d, W))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_weight_grad_is_adjoint():
    g = rng(4)
    x = g.standard_normal((2, 3, 8, 10))
    W = g.standard_normal((5, 3, 3, 3))
    d = g.standard_normal((2, 5, 8, 10))
    lhs = np.sum(oc.conv3x3(x, W) * d)
    rhs = np.sum(W * oc.conv3x3_weight_grad(x, d))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_loss_grad_matches_finite_differences():
    g = rng(5)
    p = oc.init_params(0)
    p[-289:] += 0.01 * g.standard_normal(289)
    x = g.standard_normal((2, 2, 8, 16))
    t = g.standard_normal((2, 8, 16))
    L, grad = oc.loss_grad(p, x, t)
    assert L == pytest.approx(oc.loss(oc.forward(p, x)[0], t), rel=1e-14)
    idx = g.choice(len(p), 40, replace=False)
    offs = np.cumsum([0] + [co * ci * 9 + co for co, ci in oc.layer_shapes()])
    idx = np.concatenate([idx, offs[1:] - 1, offs[:-1]])          # a bias and a first weight of every layer
    for i in idx:
        eps = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (oc.loss(oc.forward(pp, x)[0], t) - oc.loss(oc.forward(pm, x)[0], t)) / (2 * eps)
        assert abs(fd - grad[i]) <= 1e-6 * max(abs(grad[i]), 1e-3 * np.abs(grad).max()), i


def test_adam_first_step_is_sign_step():
    g = rng(6).standard_normal(100)
    p0 = rng(7).standard_normal(100)
    p1, m, v = oc.adam_step(p0, g, np.zeros(100), np.zeros(100), 1, lr=1e-3)
    assert np.allclose(p1, p0 - 1e-3 * np.sign(g), rtol=0, atol=1e-3 * 1e-8 / np.abs(g).min() + 1e-16)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_zero_network_is_its_last_bias():
    p = np.zeros(oc.num_params())
    p[-1] = 0.7
    out, _, _ = oc.forward(p, rng(8).standard_normal((1, 2, 8, 16)))
    assert np.all(out == 0.7)


def test_precondition_is_positively_homogeneous():
    p = oc.init_params(1)
    g = rng(9)
    lk = g.standard_normal((8, 16))
    r = g.standard_normal(128)
    z = oc.precondition(p, r, lk)
    assert np.allclose(oc.precondition(p, 3.5 * r, lk), 3.5 * z, rtol=1e-13, atol=0)
    assert np.all(oc.precondition(p, np.zeros(128), lk) == 0)


def test_bf16_emulation_is_close_to_fp64():
    p = oc.init_params(2)
    x = rng(10).standard_normal((2, 2, 16, 16))
    a, _, _ = oc.forward(p, x)
    b, _, _ = oc.forward(p, x, bf16=True)
    assert 1e-5 < np.linalg.norm(a - b) / np.linalg.norm(a) < 3e-2


def test_stencil_apply_and_adjoint_match_the_sparse_matrix():
    # a nonsymmetric operator (convection) so that the adjoint differs from the operator
    H, W = 6, 9
    csr = synth.convdiff_csr((H, W), np.exp(rng(11).standard_normal((H, W))), np.array([3.0, -5.0]))
    A = sp.csr_matrix((csr[2], csr[1], csr[0]))
    S = oc.stencil_from_csr(csr, H, W)[None]
    v = rng(12).standard_normal((1, H, W))
    assert np.allclose(oc.stencil_apply(S, v).ravel(), A @ v.ravel(), rtol=1e-14, atol=1e-12)
    assert np.allclose(oc.stencil_adjoint(S, v).ravel(), A.T @ v.ravel(), rtol=1e-14, atol=1e-12)


def test_residual_loss_grad_matches_finite_differences():
    g = rng(13)
    H, W = 8, 16
    p = oc.init_params(3)
    p[-289:] += 0.01 * g.standard_normal(289)
    csr = synth.convdiff_csr((H, W), np.exp(g.standard_normal((H, W))), np.array([2.0, 1.0]))
    S = np.stack([oc.stencil_from_csr(csr, H, W)] * 2) * (1.0 / (H + 1) ** 2)
    x = g.standard_normal((2, 2, H, W))
    t = g.standard_normal((2, H, W))
    L, grad = oc.loss_grad(p, x, t, stencil=S)
    assert L == pytest.approx(oc.loss(oc.stencil_apply(S, oc.forward(p, x)[0]), t), rel=1e-14)
    for i in g.choice(len(p), 30, replace=False):
        eps = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        f = lambda q: oc.loss(oc.stencil_apply(S, oc.forward(q, x)[0]), t)
        fd = (f(pp) - f(pm)) / (2 * eps)
        assert abs(fd - grad[i]) <= 1e-6 * max(abs(grad[i]), 1e-3 * np.abs(grad).max()), i
