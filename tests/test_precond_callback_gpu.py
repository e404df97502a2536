"""GPU parity of a caller's right preconditioner (RGS_PRECOND_CALLBACK: the route for incomplete
factorisations such as the ILU(0) of Sec. 5.3).  The test's M is block Jacobi over blocks of 32
consecutive unknowns (one grid line of a 32-wide grid: line relaxation), a linear map applied
with torch on the handle's stream.  One cycle against ``oracle/gmres.py`` with the same M,
flexible and not; convergence with FP32 and BF16 bases; a nonlinear M under the fallback rule;
the failure path of a callback that raises."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import paper_2011_05090_gb300 as rgs
import synth
from oracle import gmres as og
from oracle.sketch import Sketch

pytestmark = pytest.mark.gpu

BS = 32


@pytest.fixture(scope="module")
def h():
    from paper_2011_05090_gb300 import build
    build.build()
    return rgs.rgs_create()


def dev(v):
    return torch.tensor(np.asarray(v), dtype=torch.float64, device="cuda")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def system(N, seed):
    csr, _ = synth.diffusion_2d(N, 1.5, 4, seed)
    return csr, sp.csr_matrix((csr[2], csr[1], csr[0]))


def block_inverses(A):
    n = A.shape[0]
    assert n % BS == 0
    return np.stack([np.linalg.inv(A[i:i + BS, i:i + BS].toarray()) for i in range(0, n, BS)])


def oracle_m(inv):
    return lambda v: (inv @ v.reshape(-1, BS, 1)).reshape(-1)


class LineJacobi:
    """z = blockdiag(A_bb)^{-1} v on the device; records the (v, z) dtypes of every call."""

    def __init__(self, inv):
        self.inv = torch.tensor(inv, device="cuda")
        self.calls = []

    def __call__(self, v, z):
        self.calls.append((v.dtype, z.dtype))
        z.copy_(torch.bmm(self.inv, v.double().view(-1, BS, 1)).view(-1))


@pytest.mark.parametrize("flexible", [False, True])
def test_callback_one_cycle_matches_oracle(h, flexible):
    csr, A = system(32, 1)
    n, m, k = A.shape[0], 20, 70
    b = synth.rhs(n, 3)
    _, C = rgs.csr_to_device(*csr)
    inv = block_inverses(A)
    for kind in ("srht", "gaussian"):
        M = LineJacobi(inv)
        sk = rgs.rgs_sketch_create(h, kind, n, k, 5)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        rgs.rgmres_set_preconditioner(h, "callback", apply=M, flexible=flexible)
        try:
            rgs.rgmres_solve(h, sk, C, dev(b), x, restart=m, max_cycles=1, qdtype=torch.float64, fixed_steps=True)
        finally:
            rgs.rgmres_set_preconditioner(h, "none")
        ref = og.rgmres(A, b, Sketch(kind, n, k, 5), restart=m, max_cycles=1, fixed_steps=True,
                        precond=oracle_m(inv), flexible=flexible)
        xs = x.cpu().numpy()
        assert ref.true_residuals[1] < 0.5 * ref.true_residuals[0]     # M is doing work
        assert rel(xs, ref.x) <= 1e-10, kind
        # m products (columns 0 .. m-1), and M (Q y) once at the end when not flexible
        assert len(M.calls) == m + (0 if flexible else 1)
        assert all(c == (torch.float64, torch.float64) for c in M.calls)


@pytest.mark.parametrize("qdtype", [torch.float32, torch.bfloat16])
def test_callback_line_jacobi_beats_point_jacobi_and_none(h, qdtype):
    csr, A = system(64, 2)
    n = A.shape[0]
    b = synth.rhs(n, 4)
    _, C = rgs.csr_to_device(*csr)
    M = LineJacobi(block_inverses(A))
    sk = rgs.rgs_sketch_create(h, "srht", n, 120, 6)
    steps = {}
    # a BF16 basis without a preconditioner needs far more than 400 restarts on this system
    pcs = ("none", "jacobi", "callback") if qdtype == torch.float32 else ("jacobi", "callback")
    for pc in pcs:
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        rgs.rgmres_set_preconditioner(h, pc, apply=M if pc == "callback" else None)
        try:
            res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=40, rtol=1e-8, max_cycles=400, qdtype=qdtype)
        finally:
            rgs.rgmres_set_preconditioner(h, "none")
        xs = x.cpu().numpy()
        assert res["converged"] and np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8, pc
        assert res["fallback_cycle"] == -1
        steps[pc] = res["total_steps"]
    print(steps)
    assert steps["callback"] < steps["jacobi"] < steps.get("none", np.inf)
    # the basis vectors arrive in the storage type, Q y in FP64; z is FP32 for these bases
    assert {c[0] for c in M.calls} == {qdtype, torch.float64}
    assert {c[1] for c in M.calls} == {torch.float32}


def test_nonlinear_callback_falls_back(h):
    # z = ||v|| c for a fixed field c: every z_j is a multiple of c, so after a cycle the true
    # residual stops decreasing; with nonlinear = 1 the solver switches M off and converges
    csr, A = system(32, 6)
    n = A.shape[0]
    b = synth.rhs(n, 8)
    _, C = rgs.csr_to_device(*csr)
    c = dev(np.random.default_rng(2).standard_normal(n))

    def const_dir(v, z):
        z.copy_(c * v.double().norm())

    sk = rgs.rgs_sketch_create(h, "srht", n, 100, 5)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    rgs.rgmres_set_preconditioner(h, "callback", apply=const_dir, flexible=True, nonlinear=True)
    try:
        res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=30, rtol=1e-8, max_cycles=400, qdtype=torch.float32)
    finally:
        rgs.rgmres_set_preconditioner(h, "none")
    xs = x.cpu().numpy()
    assert res["fallback_cycle"] >= 1
    assert res["converged"] and np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8


def test_callback_exception_fails_the_solve_and_the_handle_recovers(h):
    csr, A = system(32, 3)
    n = A.shape[0]
    b = synth.rhs(n, 9)
    _, C = rgs.csr_to_device(*csr)
    sk = rgs.rgs_sketch_create(h, "srht", n, 80, 7)

    def planted(v, z):
        raise ZeroDivisionError("planted failure")

    rgs.rgmres_set_preconditioner(h, "callback", apply=planted, flexible=False)
    try:
        with pytest.raises(rgs.RgsError) as ei:
            rgs.rgmres_solve(h, sk, C, dev(b), torch.zeros(n, dtype=torch.float64, device="cuda"),
                             restart=20, max_cycles=3)
    finally:
        rgs.rgmres_set_preconditioner(h, "none")
    assert ei.value.status == rgs.RGS_ERR_CALLBACK
    assert isinstance(ei.value.__cause__, ZeroDivisionError)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = rgs.rgmres_solve(h, sk, C, dev(b), x, restart=40, rtol=1e-8, max_cycles=400)
    assert res["converged"] and np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b) <= 1e-8


def test_callback_argument_checks(h):
    with pytest.raises(ValueError):
        rgs.rgmres_set_preconditioner(h, "callback")
    with pytest.raises(rgs.RgsError):           # a nonlinear M needs the flexible method
        rgs.rgmres_set_preconditioner(h, "callback", apply=lambda v, z: None, flexible=False, nonlinear=True)
    rgs.rgmres_set_preconditioner(h, "none")
