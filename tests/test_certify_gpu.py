"""GPU parity of the epsilon-embedding certificate (Sec. 3.2, Prop. cert01) against the oracle,
through the C ABI.

The GPU's omega_bar, s_min and s_max for the basis an rgs_qr call returns are compared with
``oracle.certify.omega_bar`` computed from the oracle's own sketches Theta Q and Phi Q of the same
basis (FP64, LAPACK QR and SVD).  Tolerance 1e-10 relative: the GPU forms Gram matrices and a
Cholesky factor where the oracle uses Householder QR, which costs cond(V^Phi)^2 u (about 1e-15
here) plus Lanczos rounding.
"""
import numpy as np
import pytest
import torch

import paper_2011_05090_gb300 as rgs
import synth
from oracle import certify
from oracle.sketch import Sketch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2011_05090_gb300 import build
    build.build()
    return rgs.rgs_create()


def _qr(h, sk, W, qd):
    n, m = W.shape
    Q = rgs.colmajor_empty(n, m, dtype=qd)
    R = rgs.colmajor_empty(m, m)
    S = rgs.colmajor_empty(sk.k, m)
    qs = torch.empty(m, dtype=torch.float64, device="cuda")
    rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, S=S, flags=rgs.RGS_FP64_LS)
    torch.cuda.synchronize()
    return Q, qs, S


def _oracle(kind, n, k, seed, kphi, seed_phi, Qb, eps_star):
    th, ph = Sketch(kind, n, k, seed), Sketch(kind, n, kphi, seed_phi)
    return certify.omega_bar(th.apply(Qb), ph.apply(Qb), eps_star), certify.omega_exact(Qb, th.apply)


def _close(a, b, tol=1e-10):
    return abs(a - b) <= tol * max(abs(b), 1e-300)


@pytest.mark.parametrize("kind,qd,n,m,k", [("srht", torch.float64, 20000, 40, 120),
                                           ("srht", torch.float32, 70001, 60, 240),
                                           ("gaussian", torch.float64, 9000, 33, 100),
                                           ("gaussian", torch.bfloat16, 12000, 50, 200)])
@pytest.mark.parametrize("given_s", [True, False])
def test_certificate_matches_oracle(h, kind, qd, n, m, k, given_s):
    W = synth.gdw_matrix(n, m, 1e6, 21, device="cuda").T
    th = rgs.rgs_sketch_create(h, kind, n, k, 3)
    ph = rgs.rgs_sketch_create(h, kind, n, k, 1003)
    Q, qs, S = _qr(h, th, W, qd)
    got = rgs.rgs_certify_embedding(h, th, ph, Q, 0.05, vscale=qs, VTheta=S if given_s else None)
    Qb = Q.double().cpu().numpy() * qs.cpu().numpy()[None, :]
    (wb, smin, smax), omega = _oracle(kind, n, k, 3, k, 1003, Qb, 0.05)
    print(f"{kind}/{qd}/m={m}: omega_bar gpu {got['omega_bar']:.12f} oracle {wb:.12f}; "
          f"s in [{got['s_min']:.6f}, {got['s_max']:.6f}]; exact omega {omega:.4f}")
    assert got["certified"] == (wb < 1.0)
    assert _close(got["omega_bar"], wb) and _close(got["s_min"], smin) and _close(got["s_max"], smax)
    assert omega <= got["omega_bar"]


def test_certificate_of_a_larger_basis_and_of_w(h):
    """m = 300 columns (many Gram tiles, 300 Lanczos steps), certified for Q and for W itself:
    both span the same space, so omega_bar agrees (Sec. 3.2 allows V = Q or W)."""
    n, m, k = 1 << 16, 300, 1200
    W = synth.gdw_matrix(n, m, 1e3, 22, device="cuda").T
    th = rgs.rgs_sketch_create(h, "srht", n, k, 5)
    ph = rgs.rgs_sketch_create(h, "srht", n, k, 6)
    Q, qs, S = _qr(h, th, W, torch.float64)
    gq = rgs.rgs_certify_embedding(h, th, ph, Q, 0.05, vscale=qs, VTheta=S)
    gw = rgs.rgs_certify_embedding(h, th, ph, W, 0.05)
    Qb = Q.cpu().numpy() * qs.cpu().numpy()[None, :]
    (wb, smin, smax), _ = _oracle("srht", n, k, 5, k, 6, Qb, 0.05)
    print(f"m=300: omega_bar Q {gq['omega_bar']:.12f} W {gw['omega_bar']:.12f} oracle {wb:.12f}")
    assert _close(gq["omega_bar"], wb) and _close(gq["s_min"], smin) and _close(gq["s_max"], smax)
    assert _close(gw["omega_bar"], wb, 1e-8)


def test_certificate_fails_for_a_too_small_sketch(h):
    """k = m + 2 Gaussian rows: Theta is far from an embedding, omega_bar >= 1 and the call says
    so (RGS_ERR_CERT_FAILED with the values still returned); m = 1 is certified."""
    n, m = 5000, 30
    W = synth.gdw_matrix(n, m, 10.0, 23, device="cuda").T
    th = rgs.rgs_sketch_create(h, "gaussian", n, m + 2, 7)
    ph = rgs.rgs_sketch_create(h, "gaussian", n, 4 * m, 8)
    got = rgs.rgs_certify_embedding(h, th, ph, W, 0.05)
    Wn = W.cpu().numpy()
    wb, _, _ = certify.omega_bar(Sketch("gaussian", n, m + 2, 7).apply(Wn), Sketch("gaussian", n, 4 * m, 8).apply(Wn))
    assert wb >= 1.0 and not got["certified"] and _close(got["omega_bar"], wb)
    one = rgs.rgs_certify_embedding(h, ph, th, W[:, :1], 0.05)
    wb1, _, _ = certify.omega_bar(Sketch("gaussian", n, 4 * m, 8).apply(Wn[:, :1]),
                                  Sketch("gaussian", n, m + 2, 7).apply(Wn[:, :1]))
    assert _close(one["omega_bar"], wb1)


def test_certificate_rejects_bad_arguments(h):
    n = 1000
    th = rgs.rgs_sketch_create(h, "gaussian", n, 10, 1)
    ph = rgs.rgs_sketch_create(h, "gaussian", n, 10, 2)
    V = rgs.colmajor_empty(n, 11)
    V.normal_()
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_certify_embedding(h, th, ph, V)                  # m > k
    assert e.value.status == rgs.RGS_ERR_INVALID_ARG
    V2 = rgs.colmajor_empty(n, 3)
    V2.zero_()
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_certify_embedding(h, th, ph, V2)                 # Phi V = 0: G_Phi singular
    assert e.value.status == rgs.RGS_ERR_NONFINITE
