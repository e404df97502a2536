"""Pins of the oracle's unique-precision (FP32 everywhere) setting of Sec. 5.1, CPU only.

The FP32 sketch is checked against exact integer arithmetic (a Walsh-Hadamard transform of small
integers is exact in FP32) and against the FP64 sketch (close to FP32 rounding, but not closer:
it really rounds); the unique-precision RGS against the FP64 method (FP32-level agreement on a
well-conditioned matrix) and against the paper's qualitative finding on an ill-conditioned one:
with everything in FP32 the basis loses orthogonality that the mixed-precision run keeps.
"""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import rgs
from oracle.sketch import Sketch, fwht


def test_fp32_transform_exact_on_integers():
    x = np.random.default_rng(1).integers(-1000, 1000, size=(256, 3)).astype(np.float64)
    H = scipy.linalg.hadamard(256).astype(np.float64)
    assert np.array_equal(fwht(x, np.float32).astype(np.float64), H @ x)


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_fp32_sketch_rounds_like_fp32(kind):
    n, k = 5000, 64
    X = np.random.default_rng(2).standard_normal((n, 4))
    sk = Sketch(kind, n, k, 3)
    a, b = sk.apply_f32(X), sk.apply(X.astype(np.float32).astype(np.float64))
    d = np.linalg.norm(a - b) / np.linalg.norm(b)
    assert 1e-10 < d < 1e-5
    assert np.array_equal(a.astype(np.float32).astype(np.float64), a)


def test_unique_precision_close_to_fp64_on_a_well_conditioned_matrix():
    n, m, k = 4096, 20, 80
    W = synth.gdw_matrix(n, m, 10.0, 4).numpy().T.copy()
    sk = Sketch("srht", n, k, 5)
    up = rgs.rgs_qr(W, sk, storage="f32", fine="f32")
    ex = rgs.rgs_qr(W, sk)
    d = np.linalg.norm(up.R - ex.R) / np.linalg.norm(ex.R)
    assert 1e-9 < d < 1e-5
    assert np.linalg.norm(W - up.Q @ up.R) / np.linalg.norm(W) < 1e-5


def test_unique_precision_loses_orthogonality_that_mixed_precision_keeps():
    """Sec. 5.1 on the f_mu functions: the unique-precision basis ends far less well conditioned
    than the mixed-precision one, whose cond(Q) stays near 1 + O(epsilon)."""
    n, m, k = 1 << 13, 250, 1500
    W = synth.f_mu_matrix(n, m).numpy().T.copy()
    sk = Sketch("srht", n, k, 6)
    up = rgs.rgs_qr(W, sk, storage="f32", fine="f32")
    mp = rgs.rgs_qr(W, sk, storage="f32")
    c_up, c_mp = np.linalg.cond(up.Q), np.linalg.cond(mp.Q)
    c_up100, c_mp100 = np.linalg.cond(up.Q[:, :100]), np.linalg.cond(mp.Q[:, :100])
    print(f"cond(Q_250): unique FP32 {c_up:.3e}, mixed precision {c_mp:.3e}; at i = 100 {c_up100:.3e} {c_mp100:.3e}")
    assert abs(c_up100 - c_mp100) <= 1e-2 * c_mp100        # W_i still well conditioned: no difference
    assert c_mp < 3.0 and c_up > 5 * c_mp
