"""The N > 1 paths on CPU ranks (gloo, world size 2): the bench's replica timing (max over ranks,
whole-job rate) and the row-sharded sketch identity that a row-partitioned RGS would use (each
rank sketches its rows, one all-reduce of k values gives Theta w)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from oracle.sketch import Sketch, fwht

WORLD = 2


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)


def _timing(rank, port, q):
    _init(rank, port)
    ms = [10.0, 25.0][rank]
    m = bench.max_over_ranks(ms, WORLD, "cpu")
    q.put((rank, m, bench.job_rate(1e9, WORLD, m)))
    dist.destroy_process_group()


def _srht_shard(rank, port, q):
    # n = s = 2^12 rows split in two halves; H_s = [[H, H], [H, -H]] (Sylvester), so row j of
    # H_s D x is  sum_r (-1)^(popcount(j_hi & r)) (H_{s/2} D_r x_r)[j_lo]
    _init(rank, port)
    n, k, seed = 1 << 12, 64, 3
    sk = Sketch("srht", n, k, seed)
    x = np.random.default_rng(7).standard_normal(n)
    half = n // 2
    rows = slice(rank * half, (rank + 1) * half)
    z = fwht(sk.signs[rows] * x[rows])
    j = np.asarray(sk.rows)
    sign = np.where((j // half) & rank, -1.0, 1.0)
    part = torch.tensor(sign * z[j % half] / np.sqrt(k))
    dist.all_reduce(part)
    # Gaussian: column blocks of Theta, summed the same way
    gk = Sketch("gaussian", n, k, seed)
    gpart = torch.tensor(gk.dense()[:, rows] @ x[rows])
    dist.all_reduce(gpart)
    q.put((rank, part.numpy(), sk.apply(x), gpart.numpy(), gk.apply(x)))
    dist.destroy_process_group()


def _run(fn):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=fn, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(WORLD)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out, key=lambda t: t[0])


def test_replica_timing_takes_the_slowest_rank():
    out = _run(_timing)
    for rank, m, rate in out:
        assert m == 25.0
        assert rate == pytest.approx(2 * 1e9 / 0.025)


def test_row_sharded_sketch_equals_the_full_sketch():
    for rank, part, full, gpart, gfull in _run(_srht_shard):
        assert np.allclose(part, full, rtol=1e-12, atol=1e-12)
        assert np.allclose(gpart, gfull, rtol=1e-12, atol=1e-12)
