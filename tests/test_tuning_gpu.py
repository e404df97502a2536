"""Launch-shape tuning: the autotuners pick among candidates that compute the same quantities."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import paper_2011_05090_gb300 as rgs
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2011_05090_gb300 import build
    build.build()
    return rgs.rgs_create()


def to_gpu(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T)).cuda().T


def qr_R(h, sk, A):
    n, m = A.shape
    Q = rgs.colmajor_empty(n, m, dtype=torch.float32)
    R = rgs.colmajor_empty(m, m)
    rgs.rgs_qr(h, sk, to_gpu(A), Q, R)
    torch.cuda.synchronize()
    return R.cpu().numpy()


def test_tuning_roundtrip_and_checks(h):
    t0 = rgs.rgs_get_tuning(h)
    rgs.rgs_set_tuning(h, 3, 1, 1e6)
    assert rgs.rgs_get_tuning(h) == {"upd_blocks_per_sm": 3, "batch_blocks_per_sm": 1, "batch_min_team_work": 1e6,
                                     "ls_blocks": 0, "batch_rows_per_thread": 4}
    rgs.rgs_set_tuning(h, 3, 1, 1e6, 0, 2)
    assert rgs.rgs_get_tuning(h)["batch_rows_per_thread"] == 2
    for bad in [(0, 1, 1e6), (5, 1, 1e6), (2, 5, 1e6), (2, 1, 0.0), (2, 1, 1e6, 0, 3)]:
        with pytest.raises(rgs.RgsError):
            rgs.rgs_set_tuning(h, *bad)
    rgs.rgs_set_tuning(h, t0["upd_blocks_per_sm"], t0["batch_blocks_per_sm"], t0["batch_min_team_work"],
                       t0["ls_blocks"], t0["batch_rows_per_thread"])


def test_update_autotune_keeps_the_factorization(h):
    n, m, k = 1 << 16, 40, 160
    A = synth.gdw_matrix(n, m, 1e8, 4).numpy().T.copy()
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 2)
    ref = {}
    for c in (2, 4):
        rgs.rgs_set_tuning(h, c, 0, 524288.0)
        ref[c] = qr_R(h, sk, A)
    assert np.linalg.norm(ref[2] - ref[4]) <= 1e-13 * np.linalg.norm(ref[4])
    out = rgs.rgs_autotune_update(h, sk, 64)
    print(out)
    assert out["upd_blocks_per_sm"] in (2, 3, 4) and all(t > 0 for t in out["ms"])
    assert out["ms"][out["upd_blocks_per_sm"] - 2] == min(out["ms"])
    R = qr_R(h, sk, A)
    assert np.linalg.norm(R - ref[4]) <= 1e-13 * np.linalg.norm(ref[4])


def test_batched_autotune_then_solve(h):
    g = np.random.default_rng(5)
    csrs, As, bs, keep, ms_, ks = [], [], [], [], [], []
    for i in range(12):
        nx, ny = int(g.integers(20, 90)), int(g.integers(20, 90))
        csr = synth.convdiff_2d(nx, ny, float(g.uniform(1, 60)), float(g.uniform(0, 6)))
        arrays, C = rgs.csr_to_device(*csr)
        keep.append(arrays)
        csrs.append(C)
        As.append(sp.csr_matrix((csr[2], csr[1], csr[0])))
        bs.append(torch.tensor(synth.rhs(nx * ny, i), device="cuda"))
        m = int(g.integers(20, 50))
        ms_.append(m)
        ks.append(2 * m)
    out = rgs.rgs_autotune_batched(h, csrs, bs, ms_, ks, cycles=1)
    print(out)
    assert 1 <= out["batch_blocks_per_sm"] <= 4 and out["batch_min_team_work"] in (131072.0, 524288.0, 2097152.0)
    assert out["batch_rows_per_thread"] in (2, 4) and len(out["ms"]) == 12
    assert min(t for t in out["ms"] if t > 0) > 0
    xs = [torch.zeros(b.numel(), dtype=torch.float64, device="cuda") for b in bs]
    res = rgs.rgmres_solve_batched(h, csrs, bs, xs, ms_, ks, rtol=1e-8, max_cycles=300)
    for A, b, x, r in zip(As, bs, xs, res):
        bb = b.cpu().numpy()
        assert r["converged"] and np.linalg.norm(bb - A @ x.cpu().numpy()) <= 1e-8 * np.linalg.norm(bb)
