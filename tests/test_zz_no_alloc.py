"""rgs_sketch_apply_noalloc, the sketch for callers that cannot allocate device memory during a
call, against rgs_sketch_apply (which grows a handle-owned workspace with cudaMalloc) and against
the CPU oracle's sketch.

Both are called through the C ABI on the same inputs, twice in a row, so the second call also
shows that whatever the first call left in the shared scratch array does not leak into it.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2011_05090_gb300 as rgs
from oracle.sketch import Sketch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2011_05090_gb300 import build
    build.build()
    return rgs.rgs_create()


def colmajor(a):
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().T


@pytest.mark.parametrize("kind,n,k,ncols", [("srht", 1 << 20, 2000, 2), ("srht", 70001, 300, 5),
                                            ("gaussian", 10000, 300, 3), ("srht", 1000, 64, 1)])
def test_noalloc_matches_sketch_apply_on_consecutive_calls(h, kind, n, k, ncols):
    sk = rgs.rgs_sketch_create(h, kind, n, k, 23)
    rng = np.random.default_rng(n + k)
    for _ in range(2):
        X = colmajor(rng.standard_normal((n, ncols)))
        Y0 = rgs.rgs_sketch_apply(h, sk, X)
        Y1 = rgs.colmajor_empty(k, ncols)
        Y1.fill_(float("nan"))
        rgs.rgs_sketch_apply_noalloc(h, sk, X, Y1)
        torch.cuda.synchronize()
        err = (Y1 - Y0).abs().max().item()
        assert err <= 1e-13 * X.norm(dim=0).max().item()
    # the oracle's Theta X on the last input
    want = Sketch(kind, n, k, 23).apply(X.cpu().numpy())
    got = Y1.cpu().numpy()
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


def test_noalloc_more_columns_than_one_launch_takes(h):
    """70,000 columns (k = 2): launched in groups of at most 65,535 columns."""
    n, k, ncols = 64, 2, 70000
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 4)
    X = colmajor(np.random.default_rng(9).standard_normal((n, ncols)))
    Y0 = rgs.rgs_sketch_apply(h, sk, X)
    Y1 = rgs.colmajor_empty(k, ncols)
    Y1.fill_(float("nan"))
    rgs.rgs_sketch_apply_noalloc(h, sk, X, Y1)
    torch.cuda.synchronize()
    want = Sketch("srht", n, k, 4).apply(X.cpu().numpy())
    assert np.abs(Y1.cpu().numpy() - want).max() <= 1e-13 * np.abs(want).max()
    assert np.abs(Y0.cpu().numpy() - want).max() <= 1e-13 * np.abs(want).max()


def test_noalloc_rejects_wrong_dtype_device_and_host_pointers(h):
    n, k = 1000, 16
    sk = rgs.rgs_sketch_create(h, "gaussian", n, k, 2)
    Y = rgs.colmajor_empty(k, 1)
    for X in (torch.zeros(n, 1, dtype=torch.float32, device="cuda"), torch.zeros(n, 1, dtype=torch.float64)):
        with pytest.raises(ValueError):
            rgs.rgs_sketch_apply_noalloc(h, sk, X, Y)
        with pytest.raises(ValueError):
            rgs.rgs_sketch_apply(h, sk, X, Y)
    # straight through the C ABI with a host array: rejected before any launch
    Xh = np.zeros(n)
    st = rgs.load().rgs_sketch_apply_noalloc(h.ptr, sk.ptr, 1, Xh.ctypes.data_as(ctypes.c_void_p), n,
                                            ctypes.c_void_p(Y.data_ptr()), k)
    assert st == rgs.RGS_ERR_INVALID_ARG


def test_noalloc_rejects_sizes_beyond_the_scratch(h):
    k, n = 2000, 4096
    ncols = rgs.RGS_NOALLOC_SCRATCH_BYTES // 8 // k + 1
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 1)
    X = rgs.colmajor_empty(n, ncols)
    Y = rgs.colmajor_empty(k, ncols)
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_sketch_apply_noalloc(h, sk, X, Y)
    assert e.value.status == rgs.RGS_ERR_INVALID_ARG and "scratch" in str(e.value)
