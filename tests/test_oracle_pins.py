"""Pins of the CPU oracle against facts fixed outside it (CPU only).

Each check ties an oracle function to something other than itself: published
known-answer vectors, a textbook routine the method reduces to in a special
case, an exact identity of the paper, a closed form, or brute force on a tiny
input.  The NumPy and C oracles are also checked against each other.
"""
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import synth
from oracle import c_oracle, gmres, philox, rgs
from oracle.sketch import Sketch, fwht

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


# ---------------------------------------------------------------- Philox
@pytest.mark.parametrize("case", range(3))
def test_philox_known_answers_numpy(case):
    ctr, key, want = _kat()[case]
    got = philox.philox4x32_10(np.array(ctr, dtype=np.uint64), key)
    assert [int(v) for v in got] == want


@pytest.mark.parametrize("case", range(3))
def test_philox_known_answers_c(case):
    ctr, key, want = _kat()[case]
    assert [int(v) for v in c_oracle.philox(ctr, key)] == want


def test_philox_implementations_agree_on_random_counters():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64)
    key = (0x12345678, 0x9ABCDEF0)
    a = philox.philox4x32_10(ctr, key)
    for r in range(64):
        assert np.array_equal(a[r], c_oracle.philox(ctr[r].astype(np.uint32), key))


# ---------------------------------------------------------------- Gaussian sketch
def test_gaussian_theta_distribution():
    k, n = 64, 4000
    th = philox.gaussian_theta(k, n, seed=11) * np.sqrt(k)
    z = th.ravel()
    assert abs(z.mean()) < 4.0 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 6.0 * np.sqrt(2.0 / z.size)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3
    # even and odd rows (cosine / sine halves of Box-Muller) are uncorrelated
    c = np.corrcoef(th[0::2].ravel(), th[1::2].ravel())[0, 1]
    assert abs(c) < 5.0 / np.sqrt(z.size / 2)


def test_gaussian_theta_column_blocks_are_consistent():
    full = philox.gaussian_theta(9, 50, seed=3)
    part = philox.gaussian_theta(9, 50, seed=3, col0=17, ncols=11)
    assert np.array_equal(full[:, 17:28], part)
    assert not np.allclose(full, philox.gaussian_theta(9, 50, seed=4))


@pytest.mark.parametrize("kind", ["gaussian", "srht"])
def test_sketch_numpy_vs_c(kind):
    n, k = 777, 40
    a, b = Sketch(kind, n, k, 5), c_oracle.CSketch(kind, n, k, 5)
    X = np.random.default_rng(0).standard_normal((n, 3))
    assert np.allclose(a.apply(X), b.apply(X), rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind", ["gaussian", "srht"])
def test_sketch_preserves_norm_in_expectation(kind):
    # E ||Theta x||^2 = ||x||^2 for both families (Sec. 2.1 scaling 1/sqrt(k))
    n, k = 300, 30
    x = np.random.default_rng(2).standard_normal(n)
    vals = [np.sum(Sketch(kind, n, k, s).apply(x) ** 2) for s in range(300)]
    assert abs(np.mean(vals) / np.dot(x, x) - 1.0) < 0.05


# ---------------------------------------------------------------- FWHT / SRHT
def test_fwht_matches_dense_sylvester_hadamard():
    for s in (1, 2, 8, 64, 512):
        X = np.random.default_rng(s).standard_normal((s, 3))
        assert np.allclose(fwht(X), scipy.linalg.hadamard(s) @ X, atol=1e-12)


def test_hadamard_squares_to_s_identity():
    s = 128
    H = fwht(np.eye(s))
    assert np.array_equal(H @ H, s * np.eye(s))


def test_srht_sample_is_a_valid_subset():
    rows = philox.srht_sample(1024, 300, 9)
    assert len(rows) == 300 and len(set(rows.tolist())) == 300
    assert np.all(np.diff(rows) > 0) and rows[0] >= 0 and rows[-1] < 1024
    assert np.array_equal(rows, philox.srht_sample(1024, 300, 9))
    assert np.array_equal(rows, c_oracle.CSketch("srht", 1000, 300, 9).rows())


def test_srht_sample_uniform_over_seeds():
    counts = np.zeros(16)
    for seed in range(2000):
        counts[philox.srht_sample(16, 4, seed)] += 1
    assert scipy.stats.chisquare(counts).pvalue > 1e-3


def test_srht_signs_balanced_and_match_c():
    d = philox.srht_signs(5000, 4)
    assert set(np.unique(d)) == {-1.0, 1.0}
    assert abs(d.mean()) < 5.0 / np.sqrt(5000)
    assert np.array_equal(d, c_oracle.CSketch("srht", 5000, 8, 4).signs())


def test_srht_matches_explicit_definition():
    # Theta = first n columns of (1/sqrt(k)) P H_s D (Sec. 2.1, P-SRHT), built densely
    n, k = 100, 20
    sk = Sketch("srht", n, k, 6)
    H = scipy.linalg.hadamard(128).astype(float)
    D = np.diag(philox.srht_signs(n, 6))
    dense = H[philox.srht_sample(128, k, 6)][:, :n] @ D / np.sqrt(k)
    assert np.allclose(sk.dense(), dense, atol=1e-14)


def test_full_srht_is_orthogonal():
    # k = s = n: Theta = H D / sqrt(n) is orthogonal, Theta^T Theta = I
    sk = Sketch("srht", 64, 64, 1)
    Th = sk.dense()
    assert np.allclose(Th.T @ Th, np.eye(64), atol=1e-13)


# ---------------------------------------------------------------- RGS (Alg. 2)
def _well_conditioned(n, m, seed=0, cond=1e2):
    return synth.gdw_matrix(n, m, cond, seed).numpy().T.copy()


@pytest.mark.parametrize("ls", ["householder", "richardson"])
def test_rgs_orthogonal_theta_is_householder_qr(ls):
    # Theta orthogonal => the sketched LS is the exact l2 projection: RGS = classical QR
    W = _well_conditioned(64, 12, seed=3)
    out = rgs.rgs_qr(W, Sketch("srht", 64, 64, 2), ls=ls)
    Qh, Rh = np.linalg.qr(W)
    sgn = np.sign(np.diag(Rh))
    assert np.allclose(out.Q, Qh * sgn, atol=1e-13)
    assert np.allclose(out.R, Rh * sgn[:, None], atol=1e-13 * np.abs(Rh).max())


@pytest.mark.parametrize("kind", ["gaussian", "srht"])
@pytest.mark.parametrize("ls", ["householder", "richardson"])
def test_rgs_R_is_R_factor_of_sketched_W(kind, ls):
    # Theta W = S R with S orthonormal => R is the (positive-diagonal) R factor of Theta W
    W = _well_conditioned(600, 15, seed=4)
    sk = Sketch(kind, 600, 45, 8)
    out = rgs.rgs_qr(W, sk, ls=ls)
    Rp = np.linalg.qr(sk.apply(W))[1]
    Rp = Rp * np.sign(np.diag(Rp))[:, None]
    assert np.linalg.norm(out.R - Rp) / np.linalg.norm(Rp) < 1e-13
    assert np.all(np.diag(out.R) > 0) and np.allclose(np.tril(out.R, -1), 0)


@pytest.mark.parametrize("kind", ["gaussian", "srht"])
def test_rgs_invariants(kind):
    W = _well_conditioned(500, 20, seed=5)
    sk = Sketch(kind, 500, 60, 1)
    out = rgs.rgs_qr(W, sk)
    assert np.allclose(sk.apply(out.Q), out.S, atol=1e-14)                 # S = Theta Q
    assert out.delta < 1e-13                                               # Theta Q orthonormal
    assert np.linalg.norm(W - out.Q @ out.R) / np.linalg.norm(W) < 1e-13   # W = Q R
    assert out.delta_tilde < 1e-13
    # Cor. 2.2: the singular values of Q follow those of S within the embedding distortion
    assert np.linalg.cond(out.Q) < 10.0


def test_rgs_first_column_and_dropped_update_detected():
    # q_1 = w_1 / ||Theta w_1|| exactly (i = 1 convention of Alg. 2)
    W = _well_conditioned(300, 5, seed=6)
    sk = Sketch("gaussian", 300, 20, 2)
    out = rgs.rgs_qr(W, sk)
    assert np.allclose(out.Q[:, 0], W[:, 0] / np.linalg.norm(sk.apply(W[:, 0])), rtol=1e-14)
    assert out.R[0, 0] == pytest.approx(np.linalg.norm(sk.apply(W[:, 0])), rel=1e-14)


def test_rgs_mixed_precision_bounds():
    # Thm. 3.2 / 3.3 regime: u_crs cond(W) m^2 << 1 (FP32 storage, cond 10)
    W = _well_conditioned(2000, 10, seed=7, cond=10.0)
    sk = Sketch("srht", 2000, 80, 3)
    u = 2.0 ** -24
    m = 10
    for storage in ("f32",):
        out = rgs.rgs_qr(W, sk, storage=storage)
        assert out.delta_tilde <= 6 * u * m ** 1.5
        assert out.delta <= 20 * u * m ** 2 * 10.0
        assert np.linalg.norm(W - out.Q @ out.R) <= 3.7 * u * m ** 1.5 * np.linalg.norm(W)


def test_bf16_rounding_matches_torch():
    import torch
    x = np.random.default_rng(3).standard_normal(10000) * 10.0 ** np.random.default_rng(4).uniform(-8, 8, 10000)
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(rgs.round_bf16(x), want)


@pytest.mark.parametrize("kind", ["gaussian", "srht"])
@pytest.mark.parametrize("ls", ["householder", "richardson"])
@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_rgs_numpy_vs_c_oracle(kind, ls, storage):
    W = synth.gdw_matrix(700, 12, 1e6, 2).numpy().T.copy()
    a = rgs.rgs_qr(W, Sketch(kind, 700, 40, 4), ls=ls, storage=storage)
    b = c_oracle.rgs_qr(W, c_oracle.CSketch(kind, 700, 40, 4), ls=ls, storage=storage)
    assert np.linalg.norm(a.R - b.R) / np.linalg.norm(a.R) < 1e-12
    # FP64: Delta_m is rounding noise (~u cond(W)); reduced storage: same rounding, same Delta_m
    assert abs(a.delta - b.delta) <= max(1e-6 * a.delta, 1e-9)


def test_rgs_breakdown_on_dependent_column():
    W = _well_conditioned(200, 4, seed=8)
    W[:, 3] = W[:, 0] - 2.0 * W[:, 1]
    with pytest.raises(rgs.BreakdownError) as e:
        rgs.rgs_qr(W, Sketch("gaussian", 200, 12, 1))
    assert e.value.column == 3


# ---------------------------------------------------------------- RGS-Arnoldi / RGMRES
def _small_system(nx=12, ny=10, pe=20.0, seed=0):
    csr = synth.convdiff_2d(nx, ny, pe, 0.4)
    A = synth.csr_dense(csr)
    b = synth.rhs(nx * ny, seed)
    return csr, A, b


def test_arnoldi_hessenberg_identity():
    # H_m = R_m(1:m, 2:m) and A Q_{m-1} = Q_m H_m (Sec. 4.1)
    csr, A, b = _small_system()
    sk = Sketch("gaussian", A.shape[0], 40, 3)
    cyc = gmres.rgs_arnoldi(lambda v: A @ v, b, sk, 15)
    j = cyc.steps
    H = cyc.R[: j + 1, 1 : j + 1]
    assert np.allclose(np.tril(H, -2), 0)
    lhs = A @ cyc.Q[:, :j]
    assert np.linalg.norm(lhs - cyc.Q[:, : j + 1] @ H) <= 1e-12 * np.linalg.norm(lhs)


def test_rgmres_minimises_sketched_residual():
    # Eq. hls2: x_{m-1} = argmin_{v in K_{m-1}} ||Theta (A v - b)||  (brute force)
    csr, A, b = _small_system()
    n = A.shape[0]
    sk = Sketch("srht", n, 40, 5)
    steps = 12
    res = gmres.rgmres(A, b, sk, restart=steps, max_cycles=1, fixed_steps=True)
    K = np.column_stack([np.linalg.matrix_power(A, j) @ b for j in range(steps)])
    Kq = np.linalg.qr(K)[0]
    Th = sk.dense()
    z = np.linalg.lstsq(Th @ A @ Kq, Th @ b, rcond=None)[0]
    x_bf = Kq @ z
    assert np.linalg.norm(res.x - x_bf) <= 1e-9 * np.linalg.norm(x_bf)


def test_rgmres_full_krylov_solves_exactly():
    csr, A, b = _small_system(6, 5, 5.0)
    n = A.shape[0]
    res = gmres.rgmres(A, b, Sketch("gaussian", n, n + 5, 2), restart=n, max_cycles=1, tol=1e-14)
    x = np.linalg.solve(A, b)
    assert np.linalg.norm(res.x - x) <= 1e-10 * np.linalg.norm(x)


def test_rgmres_sketched_residual_monotone_and_converges():
    csr, A, b = _small_system(16, 16, 30.0)
    n = A.shape[0]
    res = gmres.rgmres(A, b, Sketch("srht", n, 60, 1), restart=25, tol=1e-8, max_cycles=40)
    assert res.converged and res.true_residuals[-1] <= 1e-8
    for rho in res.rho:
        assert np.all(np.diff(rho) <= 1e-12 * rho[0])
    assert np.all(np.diff(res.true_residuals) < 0)


def test_rgmres_quasi_optimal_against_l2_gmres():
    # ||r_rgmres|| <= sqrt((1+eps)/(1-eps)) min ||r|| over K (Sec. 4.2); eps <= 1/2 gives sqrt(3)
    csr, A, b = _small_system(14, 12, 15.0)
    n = A.shape[0]
    steps = 10
    r1 = gmres.rgmres(A, b, Sketch("gaussian", n, 80, 7), restart=steps, max_cycles=1, fixed_steps=True)
    r2 = gmres.cgs2_gmres(A, b, restart=steps, max_cycles=1, fixed_steps=True)
    assert r1.true_residuals[-1] <= np.sqrt(3.0) * r2.true_residuals[-1]
    assert r2.true_residuals[-1] <= r1.true_residuals[-1] * (1 + 1e-10)


def test_cgs2_gmres_is_minimal_residual():
    csr, A, b = _small_system()
    steps = 9
    res = gmres.cgs2_gmres(A, b, restart=steps, max_cycles=1, fixed_steps=True)
    K = np.linalg.qr(np.column_stack([np.linalg.matrix_power(A, j) @ b for j in range(steps)]))[0]
    z = np.linalg.lstsq(A @ K, b, rcond=None)[0]
    assert np.linalg.norm(res.x - K @ z) <= 1e-9 * np.linalg.norm(K @ z)


@pytest.mark.parametrize("ls", ["householder", "richardson"])
def test_rgmres_numpy_vs_c_oracle(ls):
    csr, A, b = _small_system(14, 13, 25.0)
    n = A.shape[0]
    a = gmres.rgmres(A, b, Sketch("srht", n, 50, 3), restart=20, tol=1e-9, max_cycles=30, ls=ls)
    c = c_oracle.rgmres(csr, b, c_oracle.CSketch("srht", n, 50, 3), restart=20, tol=1e-9,
                        max_cycles=30, ls=ls)
    assert a.converged and c.converged and a.cycles == c.cycles
    assert np.linalg.norm(a.x - c.x) <= 1e-9 * np.linalg.norm(a.x)


def test_cgs2_numpy_vs_c_oracle():
    csr, A, b = _small_system(14, 13, 25.0)
    a = gmres.cgs2_gmres(A, b, restart=20, tol=1e-9, max_cycles=30)
    c = c_oracle.cgs2_gmres(csr, b, restart=20, tol=1e-9, max_cycles=30)
    assert a.converged and c.converged and a.cycles == c.cycles
    assert np.linalg.norm(a.x - c.x) <= 1e-9 * np.linalg.norm(a.x)


def test_right_preconditioned_rgmres_solves_original_system():
    csr, A, b = _small_system(10, 10, 10.0)
    n = A.shape[0]
    dinv = 1.0 / np.diag(A)
    for flexible in (False, True):
        res = gmres.rgmres(A, b, Sketch("gaussian", n, 50, 2), restart=15, tol=1e-10, max_cycles=40,
                           precond=lambda v: dinv * v, flexible=flexible)
        assert res.converged
        assert np.linalg.norm(b - A @ res.x) <= 1e-10 * np.linalg.norm(b)


def test_gaussian_bf16_sketch_is_the_rounded_gaussian():
    from oracle.rgs import round_bf16
    k, n = 40, 300
    g = Sketch("gaussian", n, k, 7).dense()
    b = Sketch("gaussian_bf16", n, k, 7).dense()
    scaled = b * np.sqrt(k)
    assert np.allclose(round_bf16(scaled), scaled, rtol=1e-15, atol=0)   # bf16 values before the scale
    assert np.all(np.abs(b - g) <= 2.0 ** -8 * np.abs(g) + 1e-300)  # within half a bf16 ulp of N(0,1/k)
    assert np.abs(b - g).max() > 0
    # still an embedding in expectation: mean of ||Theta x||^2 over seeds
    x = np.random.default_rng(3).standard_normal(n)
    vals = [np.linalg.norm(Sketch("gaussian_bf16", n, k, s).apply(x)) ** 2 for s in range(60)]
    assert abs(np.mean(vals) / np.dot(x, x) - 1.0) < 0.08
