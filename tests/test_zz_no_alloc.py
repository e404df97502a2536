"""rgs_sketch_apply_noalloc, the sketch for callers that cannot allocate device memory during a
call, against rgs_sketch_apply (which grows a handle-owned workspace with cudaMalloc).

Both are called through the C ABI on the same inputs, twice in a row, so the second call also
shows that whatever the first call left in the shared scratch array does not leak into it.
"""
import numpy as np
import pytest
import torch

import paper_2011_05090_gb300 as rgs

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


def test_noalloc_rejects_sizes_beyond_the_scratch(h):
    k, n = 2000, 4096
    ncols = rgs.RGS_NOALLOC_SCRATCH_BYTES // 8 // k + 1
    sk = rgs.rgs_sketch_create(h, "srht", n, k, 1)
    X = rgs.colmajor_empty(n, ncols)
    Y = rgs.colmajor_empty(k, ncols)
    with pytest.raises(rgs.RgsError) as e:
        rgs.rgs_sketch_apply_noalloc(h, sk, X, Y)
    assert e.value.status == rgs.RGS_ERR_INVALID_ARG and "scratch" in str(e.value)
