"""GPU parity of the sketch and of RGS QR (Alg. 2) against the CPU oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import paper_2011_05090_gb300 as rgs
import synth
from oracle import c_oracle
from oracle import rgs as orgs
from oracle.sketch import Sketch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2011_05090_gb300 import build
    build.build()
    return rgs.rgs_create()


def to_gpu(a):
    """numpy (n, m) -> column-major CUDA tensor of shape (n, m)."""
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().T


def run_qr(h, sk, W, qdtype=torch.float64, qscale=False, flags=0):
    n, m = W.shape
    Q = rgs.colmajor_empty(n, m, dtype=qdtype)
    R = rgs.colmajor_empty(m, m)
    S = rgs.colmajor_empty(sk.k, m)
    qs = torch.empty(m, dtype=torch.float64, device="cuda") if qscale else None
    info = rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, S=S, flags=flags)
    torch.cuda.synchronize()
    out = {"Q": Q.double().cpu().numpy(), "R": R.cpu().numpy(), "S": S.cpu().numpy(), "info": info}
    if qscale:
        out["qscale"] = qs.cpu().numpy()
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ------------------------------------------------------------------ sketch
@pytest.mark.parametrize("kind", ["srht", "gaussian"])
@pytest.mark.parametrize("n,k", [(1, 1), (5, 3), (1000, 64), (1024, 300), (1025, 64), (4099, 7), (70001, 300)])
def test_sketch_apply_matches_oracle(h, kind, n, k):
    X = np.random.default_rng(n + k).standard_normal((n, 3))
    sk = rgs.rgs_sketch_create(h, kind, n, k, 17)
    Y = rgs.rgs_sketch_apply(h, sk, to_gpu(X)).cpu().numpy()
    ref = Sketch(kind, n, k, 17).apply(X)
    assert np.abs(Y - ref).max() <= 1e-13 * np.linalg.norm(X, axis=0).max()


def test_sketch_tables_match_oracle_definition(h):
    # the SRHT applied to unit vectors reproduces P H D column by column
    n, k = 300, 40
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 5)
    Y = rgs.rgs_sketch_apply(h, sk, to_gpu(np.eye(n))).cpu().numpy()
    assert np.array_equal(Y, Sketch("srht", n, k, 5).dense())


# ------------------------------------------------------------------ QR, FP64
@pytest.mark.parametrize("kind", ["srht", "gaussian"])
@pytest.mark.parametrize("n,m,k", [(1000, 10, 40), (4099, 33, 100), (70001, 40, 160), (2048, 64, 64)])
def test_qr_fp64_matches_oracle(h, kind, n, m, k):
    A = synth.gdw_matrix(n, m, 1e2, n + m).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, kind, n, k, 11)
    g = run_qr(h, sk, to_gpu(A))
    ref = orgs.rgs_qr(A, Sketch(kind, n, k, 11))
    assert rel(g["R"], ref.R) <= 1e-12
    assert rel(g["Q"], ref.Q) <= 1e-12
    assert rel(g["S"], ref.S) <= 1e-12
    assert np.allclose(np.tril(g["R"], -1), 0.0, atol=0) and np.all(np.diag(g["R"]) > 0)
    assert g["info"]["delta"] <= 1e-12 and g["info"]["delta_tilde"] <= 1e-13
    assert rel(A, g["Q"] @ g["R"]) <= 1e-13


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_qr_fp64_ill_conditioned_within_oracle_floor(h, kind):
    # two correct FP64 computations differ by ~cond * u in R: the floor is 10x the A-B oracle gap
    n, m, k = 6000, 40, 120
    A = synth.gdw_matrix(n, m, 1e8, 4).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, kind, n, k, 2)
    g = run_qr(h, sk, to_gpu(A))
    ra = orgs.rgs_qr(A, Sketch(kind, n, k, 2))
    rb = c_oracle.rgs_qr(A, c_oracle.CSketch(kind, n, k, 2))
    floor = max(1e-12, 10 * rel(rb.R, ra.R))
    assert rel(g["R"], ra.R) <= floor
    assert rel(A, g["Q"] @ g["R"]) <= 1e-13


def test_qr_config_c1_full_size(h):
    """n = 10,000, m = 100, D from 1 to 1e-8, Gaussian k = 300, seed 0, FP64."""
    n, m, k = 10000, 100, 300
    A = synth.gdw_matrix(n, m, 1e8, 0).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, "gaussian", n, k, 0)
    g = run_qr(h, sk, to_gpu(A))
    ra = orgs.rgs_qr(A, Sketch("gaussian", n, k, 0))
    rb = c_oracle.rgs_qr(A, c_oracle.CSketch("gaussian", n, k, 0))
    err = rel(g["R"], ra.R)
    print(f"C1: ||R-R_or||/||R_or|| = {err:.3e} (oracle A-B {rel(rb.R, ra.R):.3e}), "
          f"Delta_m = {g['info']['delta']:.3e}, ||A-QR||/||A|| = {rel(A, g['Q'] @ g['R']):.3e}")
    assert err <= max(1e-12, 10 * rel(rb.R, ra.R))
    assert rel(A, g["Q"] @ g["R"]) <= 1e-13
    assert abs(g["info"]["delta"] - ra.delta) <= 10 * max(ra.delta, 1e-15)


def test_qscale_mode_returns_exact_basis(h):
    n, m, k = 3000, 20, 60
    A = synth.gdw_matrix(n, m, 1e3, 9).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 1)
    a = run_qr(h, sk, to_gpu(A), qscale=True)
    b = run_qr(h, sk, to_gpu(A))
    assert np.array_equal(a["R"], b["R"])
    assert np.allclose(a["Q"] * a["qscale"][None, :], b["Q"], rtol=1e-15, atol=0)
    assert np.allclose(a["qscale"], 1.0 / np.diag(a["R"]), rtol=0, atol=0)


# ------------------------------------------------------------------ QR, reduced storage precision
FINE = {"df": 0, "ls64": rgs.RGS_FP64_LS, "f64": rgs.RGS_FP64_FINE}


@pytest.mark.parametrize("fine", ["df", "ls64", "f64"])
@pytest.mark.parametrize("qdtype,storage", [(torch.float32, "f32"), (torch.bfloat16, "bf16")])
@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_qr_reduced_precision_within_emulated_oracle(h, qdtype, storage, kind, fine):
    n, m, k = 20000, 40, 120
    A = synth.gdw_matrix(n, m, 1e6, 3).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, kind, n, k, 8)
    g = run_qr(h, sk, to_gpu(A), qdtype=qdtype, qscale=True, flags=FINE[fine])
    Qg = g["Q"] * g["qscale"][None, :]
    emu = orgs.rgs_qr(A, Sketch(kind, n, k, 8), storage=storage)
    exact = orgs.rgs_qr(A, Sketch(kind, n, k, 8))
    e_gpu, e_emu = rel(A, Qg @ g["R"]), rel(A, emu.Q @ emu.R)
    r_gpu, r_emu = rel(g["R"], exact.R), rel(emu.R, exact.R)
    print(f"{storage}/{kind}: ||A-QR||/||A|| gpu {e_gpu:.3e} emulated {e_emu:.3e}; "
          f"||R-R_fp64||/||R_fp64|| gpu {r_gpu:.3e} emulated {r_emu:.3e}; cond(Q) {np.linalg.cond(Qg):.3f}")
    assert e_gpu <= 10 * e_emu
    assert r_gpu <= 10 * r_emu
    assert np.linalg.cond(Qg) <= 10 * np.linalg.cond(emu.Q)


def test_c2_shaped_precision_errors_vs_fp64_oracle(h):
    """The reduced-precision bases on a smaller copy of the 2^20 x 500 workload (same D range,
    SRHT, k / m = 4): errors of the FP32 and BF16 storage against the FP64 oracle, as numbers,
    and within 10x of the oracle's own emulation of the same storage (C oracle, FP32 step 3 with
    one rounding per fused multiply-add, FP64 everything else): ||R - R_or||/||R_or||,
    ||A - QR||/||A||, cond(Q) and Delta_m, with each of the three fine arithmetics.  The oracle's
    emulation reproduces Delta_m of both storages (FP32 about 2.3, BF16 about 0.07 here): the
    difference is a property of Alg. 2 at that storage precision, not of the kernels."""
    n, m, k = 1 << 16, 200, 800
    A = synth.gdw_matrix(n, m, 1e10, 0).numpy().T.copy()
    csk = c_oracle.CSketch("srht", n, k, 0)
    ref = c_oracle.rgs_qr(A, csk)
    Qref = ref.Qp * ref.sigma[None, :]
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 0)

    def metrics(R, Q, delta):
        return {"R": rel(R, ref.R), "A-QR": rel(A, Q @ R), "condQ": np.linalg.cond(Q), "delta": delta}

    emu = {}
    for st in ("f32", "bf16"):
        e = c_oracle.rgs_qr(A, csk, storage=st)
        emu[st] = metrics(e.R, e.Qp * e.sigma[None, :], e.delta)
    out = {}
    for name, qd, flags in (("f64", torch.float64, 0), ("f32_fp64ls", torch.float32, rgs.RGS_FP64_LS),
                            ("f32_fp64fine", torch.float32, rgs.RGS_FP64_FINE), ("f32_df", torch.float32, 0),
                            ("bf16_fp64ls", torch.bfloat16, rgs.RGS_FP64_LS),
                            ("bf16_fp64fine", torch.bfloat16, rgs.RGS_FP64_FINE), ("bf16_df", torch.bfloat16, 0)):
        g = run_qr(h, sk, to_gpu(A), qdtype=qd, qscale=True, flags=flags)
        out[name] = metrics(g["R"], g["Q"] * g["qscale"][None, :], g["info"]["delta"])
    print(f"oracle FP64: ||A-QR||/||A|| {rel(A, Qref @ ref.R):.3e}  cond(Q) {np.linalg.cond(Qref):.3f}  "
          f"Delta_m {ref.delta:.3e}")
    for name, v in list(emu.items()) + list(out.items()):
        print(f"{name:>14}: ||R-R_or||/||R_or|| {v['R']:.3e}  ||A-QR||/||A|| {v['A-QR']:.3e}  "
              f"cond(Q) {v['condQ']:.3f}  Delta_m {v['delta']:.3e}")
    assert out["f64"]["R"] <= 1e-11 and out["f64"]["A-QR"] <= 1e-13
    for name, v in out.items():
        if name == "f64":
            continue
        e = emu[name.split("_")[0]]
        assert v["R"] <= 10 * e["R"] and v["A-QR"] <= 10 * e["A-QR"], name
        assert v["condQ"] <= 10 * e["condQ"], name
        assert e["delta"] / 10 <= v["delta"] <= 10 * e["delta"], name


# ------------------------------------------------------------------ status, modes, edge cases
def test_breakdown_reported_with_column(h):
    n, m, k = 2000, 6, 30
    A = synth.gdw_matrix(n, m, 10.0, 5).numpy().T.copy()
    A[:, 4] = 2.0 * A[:, 1] - A[:, 0]
    sk = rgs.rgs_sketch_create(h, "gaussian", n, k, 3)
    with pytest.raises(rgs.RgsError) as e:
        run_qr(h, sk, to_gpu(A))
    assert e.value.status == rgs.RGS_ERR_BREAKDOWN
    assert e.value.info["breakdown_col"] == 4
    # the handle stays usable afterwards
    A[:, 4] = np.random.default_rng(0).standard_normal(n)
    run_qr(h, sk, to_gpu(A))


@pytest.mark.parametrize("kind,qdtype", [("srht", torch.float32), ("gaussian", torch.float64)])
def test_nonfinite_input_reported(h, kind, qdtype):
    """A NaN in column 3 of W: the sketched norm of that column is not finite, the call returns
    RGS_ERR_NONFINITE naming the column, and the handle stays usable."""
    n, m, k = 3000, 8, 40
    A = synth.gdw_matrix(n, m, 10.0, 6).numpy().T.copy()
    A[100, 3] = np.nan
    sk = rgs.rgs_sketch_create(h, kind, n, k, 2)
    with pytest.raises(rgs.RgsError) as e:
        run_qr(h, sk, to_gpu(A), qdtype=qdtype)
    assert e.value.status == rgs.RGS_ERR_NONFINITE
    assert "column 3" in str(e.value)
    A[100, 3] = 0.5
    g = run_qr(h, sk, to_gpu(A), qdtype=qdtype)
    assert np.all(np.isfinite(g["R"]))


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
@pytest.mark.parametrize("qdtype,qscale,pin", [(torch.float64, False, True), (torch.float32, True, True),
                                               (torch.float32, True, False), (torch.bfloat16, False, True)])
def test_host_pointers_match_device_path(h, kind, qdtype, qscale, pin):
    """Host buffers (copied in column chunks behind the factorization for the SRHT) give the
    device path's result bit for bit; m = 21 leaves a ragged last chunk."""
    n, m, k = 5000, 21, 64
    A = synth.gdw_matrix(n, m, 1e4, 6).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, kind, n, k, 4)
    d = run_qr(h, sk, to_gpu(A), qdtype, qscale)
    Wh = torch.from_numpy(A.T.copy()).T
    if pin:
        Wh = Wh.pin_memory()
    Qh = rgs.colmajor_empty(n, m, dtype=qdtype, device="cpu", pin=pin)
    Rh = rgs.colmajor_empty(m, m, device="cpu", pin=pin)
    qs = torch.empty(m, dtype=torch.float64).pin_memory() if qscale else None
    for _ in range(2):                               # the second call reuses the staging buffers
        Qh.zero_()
        rgs.rgs_qr(h, sk, Wh, Qh, Rh, qscale=qs)
        assert np.array_equal(Rh.numpy(), d["R"]) and np.array_equal(Qh.double().numpy(), d["Q"])
        if qscale:
            assert np.array_equal(qs.numpy(), d["qscale"])


def test_deterministic_reruns(h):
    n, m, k = 9000, 30, 90
    A = to_gpu(synth.gdw_matrix(n, m, 1e5, 7).numpy().T.copy())
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 6)
    a, b = run_qr(h, sk, A, torch.float32), run_qr(h, sk, A, torch.float32)
    assert np.array_equal(a["R"], b["R"]) and np.array_equal(a["Q"], b["Q"])


def test_invalid_arguments_rejected(h):
    n, m = 500, 10
    sk = rgs.rgs_sketch_create(h, "gaussian", n, 8, 1)           # k < m
    W = rgs.colmajor_empty(n, m)
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_qr(h, sk, W, rgs.colmajor_empty(n, m), rgs.colmajor_empty(m, m))
    assert e.value.status == rgs.RGS_ERR_INVALID_ARG
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_sketch_create(h, "srht", 100, 129, 1)            # k > s = 128
    assert e.value.status == rgs.RGS_ERR_INVALID_ARG


@pytest.mark.parametrize("qdtype", [torch.float32, torch.bfloat16])
def test_double_float_sketch_accuracy(h, qdtype):
    """S must equal Theta applied to the stored basis: the double-float transform's error, stated."""
    n, m, k = 50000, 24, 96
    A = synth.gdw_matrix(n, m, 1e4, 12).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 3)
    g = run_qr(h, sk, to_gpu(A), qdtype=qdtype, qscale=True)
    Qrep = g["Q"] * g["qscale"][None, :]                   # the represented basis Q' diag(sigma)
    exact = Sketch("srht", n, k, 3).apply(Qrep)
    err = rel(g["S"], exact)
    print(f"double-float sketch ({qdtype}): ||S - Theta Q||/||S|| = {err:.3e}")
    assert err <= 1e-13


def test_fp64_fine_flag_close_to_double_float(h):
    """FP32 storage: the double-float transform and least squares against all-FP64 fine
    arithmetic (RGS_QR_FP64_FINE) on the same input."""
    n, m, k = 30000, 20, 80
    A = to_gpu(synth.gdw_matrix(n, m, 1e3, 13).numpy().T.copy())
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 2)
    R1, R2 = rgs.colmajor_empty(m, m), rgs.colmajor_empty(m, m)
    rgs.rgs_qr(h, sk, A, rgs.colmajor_empty(n, m, dtype=torch.float32), R1)
    rgs.rgs_qr(h, sk, A, rgs.colmajor_empty(n, m, dtype=torch.float32), R2, flags=rgs.RGS_QR_FP64_FINE)
    d = rel(R1.cpu().numpy(), R2.cpu().numpy())
    print(f"FP32 storage, double-float vs FP64 fine arithmetic: ||dR||/||R|| = {d:.3e}")
    assert d <= 1e-9


def test_objects_may_outlive_their_handle():
    """Destroying the handle first, then the sketch, then exiting must not crash (separate process)."""
    import subprocess
    import sys
    code = (
        "import torch, paper_2011_05090_gb300 as rgs\n"
        "h = rgs.rgs_create()\n"
        "sk = rgs.rgs_sketch_create(h, 'srht', 4096, 64, 1)\n"
        "a = rgs.rgs_arnoldi_create(h, sk, 4096, 8)\n"
        "rgs.load().rgs_destroy(h.ptr); h.ptr = None\n"
        "del a, sk\n"
        "h2 = rgs.rgs_create(); sk2 = rgs.rgs_sketch_create(h2, 'gaussian', 100, 8, 2)\n"
        "print('ok')\n")
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-2000:]


# ------------------------------------------------------------------ the bench workload, full size
@pytest.mark.parametrize("fine", ["ls64", "df"])
def test_c2_full_size_sampled_parity(h, fine):
    """The 2^20 x 500 factorization of the benchmark (cond 1e10, SRHT k = 2000, FP32 basis, the
    bench's tuned launch shape; FP64 least squares as timed by the bench, and double-float),
    checked on sampled columns against what the oracle computes one column at a time from the
    GPU's own outputs: the sketches Theta q'_i (steps 4-6), the sketched least-squares solutions
    (step 2, oracle Householder on the computed S), the FP32 update chain (step 3, oracle
    emulation), plus Delta_m and ||W - QR|| as properties."""
    n, m, k = 1 << 20, 500, 2000
    W = synth.gdw_matrix(n, m, 1e10, 0, device="cuda").T
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 0)
    rgs.rgs_autotune_update(h, sk, m // 2, torch.float32)
    Q = rgs.colmajor_empty(n, m, dtype=torch.float32)
    R = rgs.colmajor_empty(m, m)
    S = rgs.colmajor_empty(k, m)
    qs = torch.empty(m, dtype=torch.float64, device="cuda")
    info = rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, S=S, flags=FINE[fine])
    torch.cuda.synchronize()
    Rh, Sh, sig = R.cpu().numpy(), S.cpu().numpy(), qs.cpu().numpy()
    osk = Sketch("srht", n, k, 0)
    cols = [0, 1, 7, 100, 250, 499]
    Wc = W[:, cols].cpu().numpy()
    Qc = Q[:, cols].double().cpu().numpy()
    P, Sq = osk.apply(Wc), osk.apply(Qc)
    for c, i in enumerate(cols):
        r_or = np.linalg.norm(Sq[:, c])                      # r_ii = ||Theta q'_i||
        assert abs(Rh[i, i] - r_or) <= 1e-12 * r_or, i
        assert rel(Sh[:, i], Sq[:, c] / r_or) <= 1e-12, i    # s_i
        if i > 0:
            x = orgs.ls_householder(Sh[:, :i], P[:, c])      # step 2 on the computed S
            assert rel(Rh[:i, i], x) <= 1e-10, i
    # step 3: the FP32 chain q'_i = fl32(w_i) - sum_j c_j q'_j, c_j = fl32(R(j, i) sigma_j), one
    # rounding per fused multiply-add: bit-identical on every row
    for i in (7, 100):
        Qp = Q[:, :i].double().cpu().numpy()
        ref = orgs.update_fp32(W[:, i].cpu().numpy(), Qp, Rh[:i, i] * sig[:i])
        got = Q[:, i].double().cpu().numpy()
        same = np.mean(got == ref)
        print(f"column {i}: step-3 chain bit-identical in {same:.6f} of the rows, "
              f"rel diff {rel(got, ref):.2e}")
        assert np.array_equal(got, ref), (i, np.flatnonzero(got != ref)[:8])
    # properties of the whole factorization
    d = np.linalg.norm(np.eye(m) - Sh.T @ Sh)
    assert abs(d - info["delta"]) <= 1e-8 * d
    E = W - (Q.double() * qs[None, :]) @ R
    err = (torch.linalg.norm(E) / torch.linalg.norm(W)).item()
    del E
    print(f"full size: ||W - QR||/||W|| = {err:.3e}, Delta_m = {info['delta']:.3e}")
    assert err <= 1e-6


@pytest.mark.parametrize("scale", [2.0 ** 100, 2.0 ** -80])
def test_double_float_least_squares_on_scaled_inputs(h, scale):
    """FP32 basis (double-float least squares, FP64 squared norms), W scaled by 2^100 (1.3e30) or
    2^-80 (8.3e-25): the steps commute with a power-of-two scaling while no value leaves FP32's
    exponent range, so R scales by the same factor (to 1e-12: the runs are not bit-identical, a
    difference of 1e-14 to 1e-12 in R was measured) and the basis agrees to FP32 rounding (such a
    difference can flip the FP32 rounding of a step-3 coefficient); an overflow, underflow or
    loss of the double-float low words would show as orders of magnitude more."""
    n, m, k = 20000, 30, 120
    A = synth.gdw_matrix(n, m, 1e6, 14).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 5)
    ref = run_qr(h, sk, to_gpu(A), qdtype=torch.float32, qscale=True)
    g = run_qr(h, sk, to_gpu(A * scale), qdtype=torch.float32, qscale=True)
    Qr = ref["Q"] * ref["qscale"][None, :]
    Qg = g["Q"] * g["qscale"][None, :]
    assert np.all(np.isfinite(g["R"])) and np.all(np.isfinite(Qg))
    print(f"scale {scale:.3e}: R {rel(g['R'] / scale, ref['R']):.2e}, Q {rel(Qg, Qr):.2e}, "
          f"bit-identical R: {np.array_equal(g['R'], ref['R'] * scale)}")
    assert rel(g["R"] / scale, ref["R"]) <= 1e-12
    assert rel(Qg, Qr) <= 1e-6


# ------------------------------------------------------------------ unique precision (Sec. 5.1)
def test_unique_precision_within_emulated_oracle(h):
    """RGS_FP32_FINE (FP32 transform sums and least squares, FP32 basis) against the oracle's
    unique-precision emulation: errors within 10x of the emulation's."""
    n, m, k = 20000, 40, 120
    A = synth.gdw_matrix(n, m, 1e6, 3).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 8)
    g = run_qr(h, sk, to_gpu(A), qdtype=torch.float32, qscale=True, flags=rgs.RGS_FP32_FINE)
    Qg = g["Q"] * g["qscale"][None, :]
    emu = orgs.rgs_qr(A, Sketch("srht", n, k, 8), storage="f32", fine="f32")
    exact = orgs.rgs_qr(A, Sketch("srht", n, k, 8))
    e_gpu, e_emu = rel(A, Qg @ g["R"]), rel(A, emu.Q @ emu.R)
    r_gpu, r_emu = rel(g["R"], exact.R), rel(emu.R, exact.R)
    print(f"unique FP32: ||A-QR||/||A|| gpu {e_gpu:.3e} emulated {e_emu:.3e}; ||R-R_fp64||/||R_fp64|| gpu "
          f"{r_gpu:.3e} emulated {r_emu:.3e}; cond(Q) gpu {np.linalg.cond(Qg):.3f} emulated {np.linalg.cond(emu.Q):.3f}")
    assert e_gpu <= 10 * e_emu and r_gpu <= 10 * r_emu
    assert np.linalg.cond(Qg) <= 10 * np.linalg.cond(emu.Q)
    with pytest.raises(rgs.RgsError):                       # FP64 basis: not the unique-precision setting
        run_qr(h, sk, to_gpu(A), qdtype=torch.float64, flags=rgs.RGS_FP32_FINE)


def test_unique_precision_degrades_where_mixed_precision_does_not(h):
    """Sec. 5.1 on the f_mu functions (P-SRHT, n not a power of two): past i = 150, where W_i is
    numerically singular, the unique-FP32 basis loses conditioning and the mixed-precision one
    (FP32 step 3, FP64 elsewhere) stays near 1 + O(epsilon)."""
    n, m, k = 100000, 250, 1500
    W = synth.f_mu_matrix(n, m, device="cuda").T
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 6)
    out = {}
    for name, flags in (("unique", rgs.RGS_FP32_FINE), ("mixed", rgs.RGS_FP64_FINE)):
        Q = rgs.colmajor_empty(n, m, dtype=torch.float32)
        R = rgs.colmajor_empty(m, m)
        qs = torch.empty(m, dtype=torch.float64, device="cuda")
        rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, flags=flags)
        Qb = Q.double() * qs[None, :]
        out[name] = [float(torch.linalg.cond(Qb[:, :i]).item()) for i in (100, 250)]
    print(f"cond(Q_100), cond(Q_250): unique FP32 {out['unique']}, mixed precision {out['mixed']}")
    assert abs(out["unique"][0] - out["mixed"][0]) <= 0.02 * out["mixed"][0]
    assert out["mixed"][1] < 3.0 and out["unique"][1] > 5 * out["mixed"][1]


def test_c2_full_size_errors_vs_fp64_oracle(h):
    """The bench's 2^20 x 500 factorization (cond 1e10, SRHT k = 2000) against the C oracle run in
    full on the host cores: FP64 (the reference R) and its FP32-storage emulation.  The errors of
    the FP32 basis (FP64 and double-float least squares) and of the BF16 basis are stated against
    the FP64 oracle, and the FP32 ones must lie within 10x of the emulation's."""
    import os
    n, m, k = 1 << 20, 500, 2000
    W = synth.gdw_matrix(n, m, 1e10, 0, device="cuda").T
    Wh = W.cpu().numpy()
    c_oracle.set_threads(len(os.sched_getaffinity(0)))
    csk = c_oracle.CSketch("srht", n, k, 0)
    ref = c_oracle.rgs_qr(Wh, csk)
    emu = c_oracle.rgs_qr(Wh, csk, storage="f32")
    nW = np.linalg.norm(Wh)
    e_emu = np.linalg.norm(Wh - (emu.Qp * emu.sigma[None, :]) @ emu.R) / nW
    r_emu = rel(emu.R, ref.R)
    del emu
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 0)
    out = {}
    for name, qd, flags in (("f32_fp64ls", torch.float32, rgs.RGS_FP64_LS), ("f32_df", torch.float32, 0),
                            ("bf16_fp64ls", torch.bfloat16, rgs.RGS_FP64_LS)):
        Q = rgs.colmajor_empty(n, m, dtype=qd)
        R = rgs.colmajor_empty(m, m)
        qs = torch.empty(m, dtype=torch.float64, device="cuda")
        info = rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, flags=flags)
        torch.cuda.synchronize()
        E = W - (Q.double() * qs[None, :]) @ R
        out[name] = (rel(R.cpu().numpy(), ref.R), (torch.linalg.norm(E) / torch.linalg.norm(W)).item(), info["delta"])
        del Q, E
    print(f"FP64 oracle at full size: Delta_m {ref.delta:.3e}; FP32 emulation: ||R-R_or||/||R_or|| {r_emu:.3e}, "
          f"||W-QR||/||W|| {e_emu:.3e}")
    for name, (r, e, d) in out.items():
        print(f"{name}: ||R-R_or||/||R_or|| {r:.3e}  ||W-QR||/||W|| {e:.3e}  Delta_m {d:.3e}")
    for name in ("f32_fp64ls", "f32_df"):
        assert out[name][0] <= 10 * r_emu and out[name][1] <= 10 * e_emu
    assert out["bf16_fp64ls"][1] <= 1e-2


# ------------------------------------------------------------------ step 2 by Richardson (Sec. 2.3)
@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_richardson_least_squares_matches_oracle(h, kind):
    """RGS_LS_RICHARDSON: step 2 by two Richardson sweeps on the normal equations, FP64 basis,
    against the oracle's ls="richardson" (the NumPy and C oracles bound the rounding-order floor)."""
    n, m, k = 20000, 30, 120
    A = synth.gdw_matrix(n, m, 1e2, 31).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, kind, n, k, 4)
    g = run_qr(h, sk, to_gpu(A), qdtype=torch.float64, flags=rgs.RGS_LS_RICHARDSON)
    ref = orgs.rgs_qr(A, Sketch(kind, n, k, 4), ls="richardson", sweeps=2)
    refc = c_oracle.rgs_qr(A, c_oracle.CSketch(kind, n, k, 4), ls="richardson", sweeps=2)
    hh = orgs.rgs_qr(A, Sketch(kind, n, k, 4))
    floor = max(1e-12, 10 * rel(refc.R, ref.R))
    print(f"{kind}: ||R-R_or||/||R_or|| {rel(g['R'], ref.R):.3e} (floor {floor:.1e}); Richardson vs Householder "
          f"oracle {rel(ref.R, hh.R):.3e}; Delta_m gpu {g['info']['delta']:.3e} oracle {ref.delta:.3e}")
    assert rel(g["R"], ref.R) <= floor
    assert abs(g["info"]["delta"] - ref.delta) <= 1e-8 + 1e-6 * ref.delta


def test_richardson_with_fp32_basis_within_emulated_oracle(h):
    """FP32 basis with FP64 least squares by Richardson against the oracle's FP32 emulation with
    the same solver; without FP64 least squares the flag is rejected."""
    n, m, k = 20000, 30, 120
    A = synth.gdw_matrix(n, m, 1e2, 32).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 5)
    g = run_qr(h, sk, to_gpu(A), qdtype=torch.float32, qscale=True, flags=rgs.RGS_LS_RICHARDSON | rgs.RGS_FP64_LS)
    Qg = g["Q"] * g["qscale"][None, :]
    emu = orgs.rgs_qr(A, Sketch("srht", n, k, 5), ls="richardson", sweeps=2, storage="f32")
    exact = orgs.rgs_qr(A, Sketch("srht", n, k, 5), ls="richardson", sweeps=2)
    e_gpu, e_emu = rel(A, Qg @ g["R"]), rel(A, emu.Q @ emu.R)
    r_gpu, r_emu = rel(g["R"], exact.R), rel(emu.R, exact.R)
    print(f"Richardson FP32 basis: ||A-QR|| gpu {e_gpu:.3e} emulated {e_emu:.3e}; ||R-R_fp64|| gpu {r_gpu:.3e} "
          f"emulated {r_emu:.3e}")
    assert e_gpu <= 10 * e_emu and r_gpu <= 10 * r_emu
    with pytest.raises(rgs.RgsError):
        run_qr(h, sk, to_gpu(A), qdtype=torch.float32, flags=rgs.RGS_LS_RICHARDSON)
