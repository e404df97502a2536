"""Pins of the oracle's epsilon-embedding certificate (Sec. 3.2, Props. cert01 and cert2), CPU only.

Each check ties ``oracle.certify`` to something other than itself: closed forms for sketches
whose singular values are known (Phi = Theta; a scaled identity), the invariance of both omega
and omega_bar under a change of basis of range(V), the deterministic bound of Prop. cert2 with
Phi's embedding quality computed exactly, and the probabilistic upper bound of Prop. cert01 on
fixed seeds with Phi as large as the proposition's guarantee asks (k' >= 530 for eps* = 1/4).
"""
import numpy as np
import pytest

import synth
from oracle import certify
from oracle.sketch import Sketch


def _V(n, m, seed, cond=1e3):
    return synth.gdw_matrix(n, m, cond, seed).numpy().T.copy()


@pytest.mark.parametrize("eps_star", [0.05, 0.25])
def test_phi_equal_to_theta_gives_eps_star(eps_star):
    V = _V(3000, 20, 1)
    th = Sketch("gaussian", 3000, 80, 4)
    wb, smin, smax = certify.omega_bar(th.apply(V), th.apply(V), eps_star)
    assert abs(smin - 1.0) <= 1e-12 and abs(smax - 1.0) <= 1e-12
    assert abs(wb - eps_star) <= 1e-12


@pytest.mark.parametrize("c", [0.9, 1.1, 1.3])
def test_scaled_identity_closed_forms(c):
    """Theta = c I (k = n), Phi = I: Theta U has every singular value c."""
    eps_star = 0.05
    V = _V(400, 12, 2)
    assert abs(certify.omega_exact(V, lambda U: c * U) - abs(c * c - 1.0)) <= 1e-13
    wb, smin, smax = certify.omega_bar(c * V, V, eps_star)
    want = max(1.0 - (1.0 - eps_star) * c * c, (1.0 + eps_star) * c * c - 1.0)
    assert abs(smin - c) <= 1e-12 and abs(smax - c) <= 1e-12
    assert abs(wb - want) <= 1e-12


def test_invariant_under_change_of_basis():
    """omega and omega_bar depend on range(V) only: V and V G give the same values."""
    n, m = 4096, 16
    V = _V(n, m, 3, cond=10.0)
    G = np.linalg.qr(np.random.default_rng(5).standard_normal((m, m)))[0] @ np.diag(np.linspace(1, 4, m))
    th, ph = Sketch("srht", n, 64, 7), Sketch("srht", n, 64, 8)
    w1 = certify.omega_exact(V, th.apply)
    w2 = certify.omega_exact(V @ G, th.apply)
    b1 = certify.omega_bar(th.apply(V), ph.apply(V))[0]
    b2 = certify.omega_bar(th.apply(V @ G), ph.apply(V @ G))[0]
    assert abs(w1 - w2) <= 1e-12 and abs(b1 - b2) <= 1e-12


@pytest.mark.parametrize("kind", ["gaussian", "srht"])
def test_cert2_bound_holds(kind):
    """Prop. cert2 with eps' = Phi's exact embedding quality for V: a deterministic inequality."""
    n, m, k = 2048, 20, 60
    for seed in range(10):
        V = _V(n, m, 10 + seed)
        th, ph = Sketch(kind, n, k, 100 + seed), Sketch(kind, n, k, 200 + seed)
        w = certify.omega_exact(V, th.apply)
        ep = certify.omega_exact(V, ph.apply)
        if ep >= 1.0:
            continue
        wb = certify.omega_bar(th.apply(V), ph.apply(V))[0]
        assert wb <= certify.cert2_bound(w, ep) * (1 + 1e-12)


def test_cert01_upper_bound_on_fixed_seeds():
    """eps* = 1/4 and a Gaussian Phi with 600 >= 530 rows (the size the proposition names for
    delta* = 0.1 %): omega_bar bounds omega from above on every one of 30 fixed seeds."""
    n, m, k = 2000, 15, 120
    for seed in range(30):
        V = _V(n, m, 300 + seed)
        th = Sketch("gaussian", n, k, 400 + seed)
        ph = Sketch("gaussian", n, 600, 500 + seed)
        w = certify.omega_exact(V, th.apply)
        wb = certify.omega_bar(th.apply(V), ph.apply(V), 0.25)[0]
        assert w <= wb, (seed, w, wb)


def test_same_size_phi_overestimates_by_about_two():
    """The paper's setting (Phi the size of Theta, eps* = 0.05): omega_bar stays above omega and
    within a small factor of it (Sec. 5.1 reports about 2)."""
    n, m, k = 4096, 30, 240
    ratios = []
    for seed in range(12):
        V = _V(n, m, 600 + seed)
        th, ph = Sketch("srht", n, k, 700 + seed), Sketch("srht", n, k, 800 + seed)
        w = certify.omega_exact(V, th.apply)
        wb = certify.omega_bar(th.apply(V), ph.apply(V), 0.05)[0]
        assert w <= wb
        ratios.append(wb / w)
    assert 1.0 < np.median(ratios) < 4.0
