"""GPU parity of RGS-Arnoldi (Alg. 3), randomized GMRES (Sec. 4.2) and CGS2-GMRES against the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import paper_2011_05090_gb300 as rgs
import synth
from oracle import c_oracle
from oracle import gmres as og
from oracle.sketch import Sketch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2011_05090_gb300 import build
    build.build()
    return rgs.rgs_create()


def system(nx, ny, pe=20.0, seed=0, angle=0.4):
    csr = synth.convdiff_2d(nx, ny, pe, angle)
    A = sp.csr_matrix((csr[2], csr[1], csr[0]))
    b = synth.rhs(nx * ny, seed)
    return csr, A, b


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dev(v):
    return torch.tensor(np.asarray(v, dtype=np.float64), device="cuda")


# ------------------------------------------------------------------ Arnoldi
@pytest.mark.parametrize("kind", ["srht", "gaussian"])
@pytest.mark.parametrize("given_w", [False, True])
def test_arnoldi_steps_match_oracle(h, kind, given_w):
    csr, A, b = system(30, 27, 25.0, 1)
    n, m, k = A.shape[0], 16, 60
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, kind, n, k, 4)
    a = rgs.rgs_arnoldi_create(h, sk, n, m, torch.float64)
    rgs.rgs_arnoldi_start(h, a, dev(b))
    for i in range(1, m):
        if given_w:
            _, _, qs = rgs.rgs_arnoldi_get(h, a)
            q_prev = rgs.rgs_arnoldi_basis(a, i)[:, i - 1].cpu().numpy() * qs[i - 1]
            rgs.rgs_arnoldi_step(h, a, w=dev(A @ q_prev))
        else:
            rgs.rgs_arnoldi_step(h, a, csr=C)
    nc, R, qs = rgs.rgs_arnoldi_get(h, a)
    assert nc == m
    ref = og.rgs_arnoldi(lambda v: A @ v, b, Sketch(kind, n, k, 4), m - 1)
    assert rel(R, ref.R) <= 1e-12
    Q = rgs.rgs_arnoldi_basis(a, m).cpu().numpy() * qs[None, :]
    assert rel(Q, ref.Q) <= 1e-11
    # Arnoldi identity A Q_{m-1} = Q_m H_m with H = R(1:m, 2:m) (Sec. 4.1)
    H = R[:, 1:]
    assert np.linalg.norm(A @ Q[:, :-1] - Q @ H) <= 1e-12 * np.linalg.norm(A @ Q[:, :-1])


def test_arnoldi_rejects_overflow_and_missing_start(h):
    n = 100
    sk = rgs.rgs_sketch_create(h, "gaussian", n, 10, 1)
    a = rgs.rgs_arnoldi_create(h, sk, n, 3)
    with pytest.raises(rgs.RgsError):
        rgs.rgs_arnoldi_step(h, a, w=dev(np.ones(n)))
    with pytest.raises(rgs.RgsError):
        rgs.rgs_arnoldi_create(h, sk, n, 11)                      # mmax > k


# ------------------------------------------------------------------ RGMRES
@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_rgmres_fp64_one_cycle_matches_oracle(h, kind):
    csr, A, b = system(24, 25, 30.0, 2)
    n, m, k = A.shape[0], 20, 70
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, kind, n, k, 9)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=m, max_cycles=1, qdtype=torch.float64, fixed_steps=True)
    ref = og.rgmres(A, b, Sketch(kind, n, k, 9), restart=m, max_cycles=1, fixed_steps=True)
    refc = c_oracle.rgmres(csr, b, c_oracle.CSketch(kind, n, k, 9), restart=m, max_cycles=1, fixed_steps=True)
    floor = max(1e-12, 10 * rel(refc.x, ref.x))
    assert rel(x.cpu().numpy(), ref.x) <= floor
    assert res["cycles"] == 1 and res["total_steps"] == m
    assert abs(res["history"][1] - ref.true_residuals[1]) <= 1e-10 * ref.true_residuals[0]


@pytest.mark.parametrize("fine", ["ls64", "f64", "df"])
@pytest.mark.parametrize("qdtype,storage", [(torch.float32, "f32"), (torch.bfloat16, "bf16")])
@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_rgmres_reduced_precision_one_cycle_vs_emulated_oracle(h, kind, qdtype, storage, fine):
    """One fixed cycle of RGMRES(20) with an FP32 / BF16 basis against the oracle's emulation of
    the same storage (FP32 step 3 with one rounding per fused multiply-add, FP64 elsewhere).
    With FP64 fine arithmetic (all of it, or the least squares with the Gaussian sketch, whose
    sums are FP64 anyway) the GPU takes the emulation's roundings: x agrees to 1e-10.  Where
    double-float sums or products enter, some FP32 roundings of q' differ, so x lies within 10x of
    the emulation's own distance from the FP64 method, and the true residual after the cycle
    within 10x of the emulation's distance plus ten FP32 storage roundings of it."""
    csr, A, b = system(24, 25, 30.0, 2)
    n, m, k = A.shape[0], 20, 70
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, kind, n, k, 9)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=m, max_cycles=1, qdtype=qdtype, fixed_steps=True,
                           fine64=fine == "f64", ls64=fine == "ls64")
    emu = og.rgmres(A, b, Sketch(kind, n, k, 9), restart=m, max_cycles=1, fixed_steps=True, storage=storage)
    ex = og.rgmres(A, b, Sketch(kind, n, k, 9), restart=m, max_cycles=1, fixed_steps=True)
    xg = x.cpu().numpy()
    d_gpu, d_emu = rel(xg, emu.x), rel(emu.x, ex.x)
    r_gpu, r_emu, r_ex = res["history"][1], emu.true_residuals[1], ex.true_residuals[1]
    print(f"{kind}/{storage}/{fine}: ||x-x_emu||/||x_emu|| {d_gpu:.2e} (emulation vs FP64 {d_emu:.2e}); "
          f"residual gpu {r_gpu:.6e} emulated {r_emu:.6e} fp64 {r_ex:.6e}")
    assert res["cycles"] == 1 and res["total_steps"] == m
    same_roundings = fine == "f64" or (fine == "ls64" and kind == "gaussian")
    if same_roundings:
        assert d_gpu <= 1e-10
        assert abs(r_gpu - r_emu) <= 1e-10 * r_emu
    else:
        u_crs = 2.0 ** -24 if storage == "f32" else 2.0 ** -8
        assert d_gpu <= 10 * d_emu
        assert abs(r_gpu - r_ex) <= 10 * abs(r_emu - r_ex) + 10 * u_crs * r_ex


@pytest.mark.parametrize("qdtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_rgmres_converges_to_1e8(h, qdtype, kind):
    csr, A, b = system(48, 40, 40.0, 3)
    n, m, k = A.shape[0], 30, 90
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, kind, n, k, 1)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=m, rtol=1e-8, max_cycles=200, qdtype=qdtype)
    xs = x.cpu().numpy()
    true_rel = np.linalg.norm(b - A @ xs) / np.linalg.norm(b)
    ref = og.rgmres(A, b, Sketch(kind, n, k, 1), restart=m, tol=1e-8, max_cycles=200)
    print(f"{kind}/{qdtype}: cycles {res['cycles']} steps {res['total_steps']} rel {true_rel:.2e}; "
          f"oracle FP64 cycles {ref.cycles} steps {sum(ref.steps)}")
    assert res["converged"] and true_rel <= 1e-8
    assert abs(true_rel - res["rel_residual"]) <= 1e-3 * 1e-8
    assert res["total_steps"] <= 1.3 * sum(ref.steps) + m
    h_ = res["history"]
    assert all(h_[i + 1] < h_[i] for i in range(len(h_) - 1))


def test_rgmres_happy_breakdown(h):
    # A = 2 I: the Krylov space of any b is one-dimensional; the first cycle is exact
    n = 500
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    va = np.full(n, 2.0)
    (r_, c_, v_), C = rgs.csr_to_device(rp, ci, va)
    sk = rgs.rgs_sketch_create(h, "gaussian", n, 40, 2)
    b = synth.rhs(n, 5)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=10, rtol=1e-12, max_cycles=3, qdtype=torch.float64)
    assert res["converged"] and res["cycles"] == 1 and res["total_steps"] == 1
    assert rel(x.cpu().numpy(), b / 2.0) <= 1e-14


def test_rgmres_nonzero_initial_guess_and_zero_steps(h):
    csr, A, b = system(20, 20, 10.0, 4)
    n = A.shape[0]
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, "srht", n, 60, 3)
    xs = sp.linalg.spsolve(A.tocsc(), b)
    x = dev(xs)
    res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=20, rtol=1e-8, max_cycles=5)
    assert res["converged"] and res["cycles"] == 0
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgmres_solve(h, sk, C, dev(np.zeros(n)), torch.zeros(n, dtype=torch.float64, device="cuda"), restart=20)
    assert e.value.status == rgs.RGS_ERR_INVALID_ARG


# ------------------------------------------------------------------ CGS2-GMRES (FP64 comparator)
def test_cgs2_one_cycle_matches_oracle(h):
    csr, A, b = system(24, 25, 30.0, 2)
    n, m = A.shape[0], 20
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rgs.cgs2_gmres_solve(h, C, dev(b), x, restart=m, max_cycles=1, fixed_steps=True)
    ref = og.cgs2_gmres(A, b, restart=m, max_cycles=1, fixed_steps=True)
    assert rel(x.cpu().numpy(), ref.x) <= 1e-11


def test_cgs2_converges_like_oracle(h):
    csr, A, b = system(48, 40, 40.0, 3)
    n, m = A.shape[0], 30
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = rgs.cgs2_gmres_solve(h, C, dev(b), x, restart=m, rtol=1e-8, max_cycles=200)
    ref = c_oracle.cgs2_gmres(csr, b, restart=m, tol=1e-8, max_cycles=200)
    xs = x.cpu().numpy()
    assert res["converged"] and np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8
    assert abs(res["total_steps"] - ref.steps) <= max(3, 0.05 * ref.steps)


@pytest.mark.parametrize("solver", ["rgmres_f32", "rgmres_f64", "cgs2"])
def test_large_norm_operator_no_overflow(h, solver):
    # ||A|| ~ 1e12: unnormalised Krylov vectors would grow like ||A||^j and overflow
    csr, A, b = system(40, 40, 30.0, 6)
    scale = 1e8
    csr = (csr[0], csr[1], csr[2] * scale)
    A = A * scale
    n = A.shape[0]
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    if solver == "cgs2":
        res = rgs.cgs2_gmres_solve(h, C, dev(b), x, restart=60, rtol=1e-8, max_cycles=100)
    else:
        sk = rgs.rgs_sketch_create(h, "srht", n, 150, 2)
        q = torch.float32 if solver == "rgmres_f32" else torch.float64
        res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=60, rtol=1e-8, max_cycles=100, qdtype=q)
    xs = x.cpu().numpy()
    assert res["converged"] and np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8


@pytest.mark.parametrize("solver", ["rgmres", "cgs2"])
def test_7_point_operator_full_tiles(h, solver):
    # 3D 7-point operator: every 1024-row tile holds ~7,000 nonzeros; one fixed cycle in FP64
    # against the oracle
    csr = synth.convdiff_3d(20, 30.0, 1.0, 3, 4)
    A = sp.csr_matrix((csr[2], csr[1], csr[0]))
    n = A.shape[0]
    b = synth.rhs(n, 9)
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    if solver == "cgs2":
        rgs.cgs2_gmres_solve(h, C, dev(b), x, restart=15, max_cycles=1, fixed_steps=True)
        ref = og.cgs2_gmres(A, b, restart=15, max_cycles=1, fixed_steps=True)
    else:
        sk = rgs.rgs_sketch_create(h, "srht", n, 60, 3)
        rgs.rgmres_solve(h, sk, C, dev(b), x, restart=15, max_cycles=1, qdtype=torch.float64, fixed_steps=True)
        ref = og.rgmres(A, b, Sketch("srht", n, 60, 3), restart=15, max_cycles=1, fixed_steps=True)
    assert rel(x.cpu().numpy(), ref.x) <= 1e-10
    y = rgs.rgs_csr_matvec(h, C, dev(b))
    assert np.allclose(y.cpu().numpy(), A @ b, rtol=1e-13, atol=1e-12 * np.abs(A @ b).max())


def test_c3_full_size_true_residual(h):
    """The benchmark's 128^3 convection-diffusion solve (n = 2,097,152; RGMRES(100), SRHT k = 400,
    FP32 basis, the bench's launch shapes) to 1e-8: convergence and the residual the solver
    reports, checked against b - A x recomputed in FP64 on the CPU from the same CSR matrix."""
    csr = synth.convdiff_3d(128, 50.0, 1.0, 8, 0)
    A = sp.csr_matrix((csr[2], csr[1], csr[0]))
    n = A.shape[0]
    b = synth.rhs(n, 0)
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, "srht", n, 400, 0)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=100, rtol=1e-8, max_cycles=400, qdtype=torch.float32)
    true_rel = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
    print(f"128^3: {res['total_steps']} steps, reported {res['rel_residual']:.3e}, recomputed {true_rel:.3e}")
    assert res["converged"] and true_rel <= 1e-8
    assert abs(true_rel - res["rel_residual"]) <= 1e-3 * true_rel


@pytest.mark.parametrize("qdtype,fine", [(torch.float32, "df"), (torch.float32, "ls64"), (torch.float64, "f64"),
                                         (torch.bfloat16, "df")])
@pytest.mark.parametrize("jacobi", [False, True])
def test_sell_product_bit_identical_to_csr(h, qdtype, fine, jacobi, monkeypatch):
    """The fused product reads A in SELL-32 form (slices of 32 rows, entry-major, padding within
    nnz / 4): the same products and sums in the same order as from CSR, so one fixed RGMRES cycle
    gives bit-identical x whichever layout it read (RGS_SELL=0 keeps CSR), also for A D^{-1}."""
    csr = synth.convdiff_3d(18, 30.0, 1.0, 3, 5)           # 5832 rows: slices with 4-7 nonzeros
    A = sp.csr_matrix((csr[2], csr[1], csr[0]))
    n = A.shape[0]
    b = dev(synth.rhs(n, 11))
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, "srht", n, 80, 6)
    rgs.rgmres_set_preconditioner(h, "jacobi" if jacobi else "none")
    out = {}
    try:
        for layout in ("sell", "csr"):
            if layout == "csr":
                monkeypatch.setenv("RGS_SELL", "0")
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            res = rgs.rgmres_solve(h, sk, C, b, x, restart=25, max_cycles=2, qdtype=qdtype, fixed_steps=True,
                                   fine64=fine == "f64" and qdtype != torch.float64, ls64=fine == "ls64")
            out[layout] = (x.cpu().numpy(), res)
    finally:
        rgs.rgmres_set_preconditioner(h, "none")
    assert out["sell"][1]["sell"] and not out["csr"][1]["sell"]
    assert np.array_equal(out["sell"][0], out["csr"][0])
    assert out["sell"][1]["history"] == out["csr"][1]["history"]


def test_sell_falls_back_to_csr_for_uneven_rows(h):
    """Rows of very different lengths (one dense row per slice) would pad SELL-32 past nnz / 4:
    the solver keeps CSR and still matches the oracle."""
    n = 640
    rows, cols = [], []
    for r in range(n):
        rows.append(r); cols.append(r)
        if r % 32 == 0:
            for c in range(0, n, 7):
                if c != r:
                    rows.append(r); cols.append(c)
        elif r + 1 < n:
            rows.append(r); cols.append(r + 1)
    vals = np.where(np.array(rows) == np.array(cols), 4.0, -0.01)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    A.sort_indices()
    csr = (A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64))
    b = synth.rhs(n, 12)
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, "srht", n, 60, 7)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=15, max_cycles=1, qdtype=torch.float64, fixed_steps=True)
    ref = og.rgmres(A, b, Sketch("srht", n, 60, 7), restart=15, max_cycles=1, fixed_steps=True)
    assert not res["sell"]
    assert rel(x.cpu().numpy(), ref.x) <= 1e-10


@pytest.mark.parametrize("qdtype,tol", [(torch.float64, 1e-8), (torch.float32, 1e-4)])
def test_rgmres_redraws_theta_after_a_stalled_cycle(h, qdtype, tol):
    """From a residual the SRHT cannot see (b - A x0 = D H e_j, j not sampled, plus a small visible
    part; the oracle's restart pins), the first cycle leaves the true residual where it was, so the
    solver draws Theta anew with the oracle's seed rule (seed + 0x9E3779B97F4A7C15): the residual
    after the second cycle matches the oracle's, and the solve converges."""
    from test_oracle_restart_refresh import stalled_start
    A, b, sk_o, x0, _ = stalled_start()
    n = A.shape[0]
    (rp, ci, va), C = rgs.csr_to_device(A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data)
    sk = rgs.rgs_sketch_create(h, "srht", n, 60, 3)
    x = dev(x0)
    res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=20, rtol=1e-8, max_cycles=300, qdtype=qdtype)
    ref = og.rgmres(A, b, sk_o, restart=20, tol=1e-8, max_cycles=300, x0=x0,
                    storage="f64" if qdtype == torch.float64 else "f32")
    hist = res["history"]
    print(f"{qdtype}: gpu cycles {res['cycles']} refreshes {res['sketch_refreshes']} history {hist[:4]}; "
          f"oracle cycles {ref.cycles} refreshes {ref.refreshes} {ref.true_residuals[:4]}")
    assert hist[1] >= (1.0 - 2.0 ** -10) * hist[0] and hist[2] < 0.5 * hist[1]
    assert abs(hist[2] - ref.true_residuals[2]) <= tol * ref.true_residuals[2]
    assert res["converged"] and res["sketch_refreshes"] >= 1
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(b)
