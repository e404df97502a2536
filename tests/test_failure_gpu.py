"""The device-side wait timeout, exercised without hanging or faulting the GPU.

Every grid and team barrier of the library's kernels gives up after a clock-cycle budget,
records RGS_ERR_TIMEOUT, raises the abort word and lets every CTA leave at its next barrier.
rgs_set_wait_budget(h, 1) makes that budget one cycle, so the first CTA that has to wait at
all gives up: the timeout path then runs on purpose in the real kernels (the cooperative
least-squares kernel of QR and RGMRES, the team barriers of the batched solver).  Each call
must return RGS_ERR_TIMEOUT, and the handle must stay usable: with the default budget back,
the same calls return results identical to those of a run that never timed out.
"""
import numpy as np
import pytest
import torch

import paper_2011_05090_gb300 as rgs
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2011_05090_gb300 import build
    build.build()
    return rgs.rgs_create()


def _qr(h, sk, W, qd, flags=0):
    n, m = W.shape
    Q = rgs.colmajor_empty(n, m, dtype=qd)
    R = rgs.colmajor_empty(m, m)
    qs = torch.empty(m, dtype=torch.float64, device="cuda")
    rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, flags=flags)
    torch.cuda.synchronize()
    return R.cpu().numpy(), Q.double().cpu().numpy(), qs.cpu().numpy()


@pytest.mark.parametrize("qd,flags", [(torch.float32, 0), (torch.float32, rgs.RGS_FP64_FINE),
                                      (torch.float64, 0)])
def test_qr_wait_timeout_reported_and_handle_usable(h, qd, flags):
    n, m, k = 1 << 16, 24, 96
    W = synth.gdw_matrix(n, m, 1e6, 3, device="cuda").T
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 1)
    ref = _qr(h, sk, W, qd, flags)
    try:
        rgs.rgs_set_wait_budget(h, 1)
        with pytest.raises(rgs.RgsError) as e:
            _qr(h, sk, W, qd, flags)
        assert e.value.status == rgs.RGS_ERR_TIMEOUT
    finally:
        rgs.rgs_set_wait_budget(h, 0)
    again = _qr(h, sk, W, qd, flags)
    for a, b in zip(ref, again):
        assert np.array_equal(a, b)


def test_rgmres_wait_timeout_reported_and_handle_usable(h):
    csr = synth.convdiff_2d(60, 50, 20.0, 0.7)
    n = 60 * 50
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    b = torch.tensor(synth.rhs(n, 3), device="cuda")
    sk = rgs.rgs_sketch_create(h, "srht", n, 80, 2)

    def solve():
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        r = rgs.rgmres_solve(h, sk, C, b, x, restart=30, rtol=1e-8, max_cycles=50, qdtype=torch.float32)
        return r, x.cpu().numpy()

    r0, x0 = solve()
    try:
        rgs.rgs_set_wait_budget(h, 1)
        with pytest.raises(rgs.RgsError) as e:
            solve()
        assert e.value.status == rgs.RGS_ERR_TIMEOUT
    finally:
        rgs.rgs_set_wait_budget(h, 0)
    r1, x1 = solve()
    assert r0["converged"] and r1["converged"] and np.array_equal(x0, x1)


def test_batched_wait_timeout_reported_and_handle_usable(h):
    """Two 256 x 256 systems: each is solved by a team of several CTAs (team barriers)."""
    insts = []
    for i in range(2):
        csr = synth.convdiff_2d(256, 256, 30.0 + i, 0.5 + i)
        arrays, C = rgs.csr_to_device(*csr)
        insts.append((arrays, C, torch.tensor(synth.rhs(256 * 256, 40 + i), device="cuda")))

    def solve():
        xs = [torch.zeros(256 * 256, dtype=torch.float64, device="cuda") for _ in insts]
        res = rgs.rgmres_solve_batched(h, [I[1] for I in insts], [I[2] for I in insts], xs, [30, 30], [60, 60],
                                       max_cycles=2, fixed_steps=True, qdtype=torch.float32, sketch_seed=3)
        return res, [x.cpu().numpy() for x in xs]

    r0, x0 = solve()
    try:
        rgs.rgs_set_wait_budget(h, 1)
        with pytest.raises(rgs.RgsError) as e:
            solve()
        assert e.value.status == rgs.RGS_ERR_TIMEOUT
    finally:
        rgs.rgs_set_wait_budget(h, 0)
    r1, x1 = solve()
    for a, b in zip(x0, x1):
        assert np.array_equal(a, b)
