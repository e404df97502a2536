#!/usr/bin/env python
"""Benchmark of randomized Gram-Schmidt QR (Alg. 2) on one or more GB300 GPUs.

Workload (one "step" = one full rgs_qr call):
    A = G D W with n = 2^20 rows, m = 500 columns, D log-spaced from 1 to 1e-10,
    G iid N(0,1), W Haar orthogonal; SRHT sketch with k = 2000 over 2^20;
    basis stored in FP32 with FP32 update arithmetic, sketches / least squares
    in FP64.  Inputs (4.2 GB) are far larger than L2 (129 MB), so no flush is
    needed between steps.

Metric: whole-job algorithmic HBM throughput of the QR in GB/s, i.e.
    bytes = 8 n m                    (step 1, one pass over W)
          + sum_i [4 n i + 8 n + 4 n] (steps 3-4: read Q'_{i-1}, read w_i, write q'_i)
divided by the measured time.  With --gpus N (torchrun), every rank factors
its own independent matrix (weak scaling, no collective on the data path).

The second half of the metric is reported in the same line ("rgmres"): restarted
RGMRES(100) with RGS-Arnoldi (SRHT k = 400, FP32 basis, FP64 least squares and
restart residual) against FP64 CGS2-GMRES(100) on the same GPU, time to a relative
residual of 1e-8 on a 3D convection-diffusion operator: 128^3 grid (n = 2,097,152,
7-point CSR, FP64 values), log-normal diffusion (sigma = 1, correlation length 8
cells), Peclet number 50, iid N(0,1) right-hand side.

--impl reference times the CPU oracle (oracle/c/rgs_oracle.c) on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RGS-QR HBM GB/s (% peak); RGMRES time-to-1e-8 vs FP64 CGS2-GMRES same GB300"
N_ROWS, M_COLS, K_SKETCH, COND, SEED = 1 << 20, 500, 2000, 1e10, 0
WORKLOAD = "rgs_qr n=1048576 m=500 cond=1e10 srht k=2000 q=f32"


def qr_bytes(n, m, esz=4, wbytes=8):
    upd = sum(esz * n * i + wbytes * n + esz * n for i in range(m))
    return wbytes * n * m + upd, upd


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_traffic():
    """Mean per-launch DRAM traffic (bytes) of the fused update kernel over the m = 500 step, from the
    committed ncu summary (measured on one launch, scaled by the launch's algorithmic bytes)."""
    path = os.path.join(ROOT, "profiles", "rgs_update_sketch_c2.txt")
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("traffic_bytes_per_launch_full_step:"):
                    return float(line.split(":")[1])
    except OSError:
        pass
    return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) >= 9:
                        rows.append(p)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def f(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [f(r[1]) for r in rows if f(r[1]) is not None]
        mx = [f(r[2]) for r in rows if f(r[2]) is not None]
        pw = [f(r[3]) for r in rows if f(r[3]) is not None]
        loaded = [s for s, p in zip(sm, pw) if p is not None and p > 0.5 * max(pw)] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_sample_gbps(A_cols_host, n, k, storage="f32"):
    """Time the C oracle on the first columns of the workload; returns (GB/s, seconds, columns)."""
    from oracle import c_oracle
    c_oracle.build()
    sk = c_oracle.CSketch("srht", n, k, SEED)
    msub = A_cols_host.shape[1]
    t0 = time.perf_counter()
    c_oracle.rgs_qr(A_cols_host, sk, ls="householder", storage=storage)
    dt = time.perf_counter() - t0
    total, _ = qr_bytes(n, msub)
    return total / dt / 1e9, dt, msub


def run_reference(args):
    """The CPU oracle as it stands, on a bounded sample of the workload (host cores)."""
    import torch
    import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    msub = 40
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A = synth.gdw_matrix(N_ROWS, M_COLS, COND, SEED, device=dev)[:msub].cpu().numpy().T.copy()
    for _ in range(args.warmup):
        cpu_sample_gbps(A, N_ROWS, K_SKETCH)
    vals, secs = [], []
    for _ in range(args.steps):
        v, dt, _ = cpu_sample_gbps(A, N_ROWS, K_SKETCH)
        vals.append(v)
        secs.append(dt)
    total, _ = qr_bytes(N_ROWS, msub)
    value = total * len(secs) / sum(secs) / 1e9
    sample = f"first {msub} of {M_COLS} columns of the workload (n=2^20, SRHT k=2000, f32 storage emulation)"
    out = {"metric": METRIC, "value": value, "unit": "GB/s", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "sample_columns": msub},
           "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_gmres_c3(rgs, h, N=128, max_cycles=400, solvers=("rgmres", "cgs2")):
    """Time-to-1e-8 of RGMRES (FP32 basis) and FP64 CGS2-GMRES on the 3D convection-diffusion system."""
    import torch
    import synth
    csr = synth.convdiff_3d(N, 50.0, 1.0, 8, 0)
    n = N ** 3
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    b = torch.tensor(synth.rhs(n, 0), device="cuda")
    sk = rgs.rgs_sketch_create(h, "srht", n, 400, 0)
    # warm-up on a few cycles (kernels loaded, allocator primed)
    xw = torch.zeros(n, dtype=torch.float64, device="cuda")
    rgs.rgmres_solve(h, sk, C, b, xw, restart=100, max_cycles=1)
    rgs.cgs2_gmres_solve(h, C, b, xw.zero_(), restart=100, max_cycles=1)
    out = {"config": "convdiff3d 128^3 n=2097152 nnz=%d Pe=50 sigma=1 corr=8 restart=100 rtol=1e-8" % len(csr[1])}
    runs = (("rgmres_f32_srht400", "rgmres", lambda x: rgs.rgmres_solve(h, sk, C, b, x, restart=100, rtol=1e-8,
                                                                    max_cycles=max_cycles, qdtype=torch.float32)),
            ("cgs2_gmres_f64", "cgs2", lambda x: rgs.cgs2_gmres_solve(h, C, b, x, restart=100, rtol=1e-8,
                                                                     max_cycles=max_cycles)))
    for name, key, fn in runs:
        if key not in solvers:
            continue
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fn(x)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"seconds": dt, "converged": res["converged"], "rel_residual": res["rel_residual"],
                     "cycles": res["cycles"], "arnoldi_steps": res["total_steps"],
                     "us_per_step": 1e6 * dt / max(1, res["total_steps"])}
    if "rgmres_f32_srht400" in out and "cgs2_gmres_f64" in out:
        a, c = out["rgmres_f32_srht400"], out["cgs2_gmres_f64"]
        out["speedup_vs_cgs2_fp64"] = c["seconds"] / a["seconds"]
    return out


def run_gmres_profile(args):
    """Profiling case: the 128^3 RGMRES and/or CGS2 solve for a few cycles only (no bench line)."""
    import paper_2011_05090_gb300 as rgs
    from paper_2011_05090_gb300 import build as libbuild
    libbuild.build()
    h = rgs.rgs_create()
    print(json.dumps(run_gmres_c3(rgs, h, max_cycles=args.gmres_cycles, solvers=tuple(args.gmres_only.split(",")))),
          flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2011_05090_gb300 as rgs
    import synth
    from paper_2011_05090_gb300 import build as libbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        libbuild.build()
    if world > 1:
        dist.barrier()

    n, m, k = N_ROWS, (args.cols or M_COLS), K_SKETCH
    W = synth.gdw_matrix(n, m, COND, SEED + rank, device="cuda").T          # (n, m) column-major
    h = rgs.rgs_create()
    sk = rgs.rgs_sketch_create(h, "srht", n, k, SEED)
    Q = rgs.colmajor_empty(n, m, dtype=torch.float32)
    R = rgs.colmajor_empty(m, m)
    qs = torch.empty(m, dtype=torch.float64, device="cuda")
    flags = rgs.RGS_QR_TIMINGS

    for _ in range(args.warmup):
        rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, flags=flags)
    torch.cuda.synchronize()

    infos = []
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        start.record()
        for _ in range(args.steps):
            infos.append(rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, flags=flags))
        stop.record()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = start.elapsed_time(stop)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    total, upd = qr_bytes(n, m)
    value = world * total * args.steps / (ms_max * 1e-3) / 1e9

    # dominant kernel: the fused update + sketch, timed per launch on the library's stream
    upd_ms = sum(i["update_ms"] for i in infos) / len(infos)
    peak, peak_kind = peaks()
    achieved = upd / (upd_ms * 1e-3) / 1e9
    traffic_full = profile_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_full if (traffic_full and m == M_COLS) else None,
                "kernel": "update_sketch_kernel<float,SRHT>",
                "bytes_per_launch": upd / m, "launches_per_step": m,
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured" else "fallback 6.8 TB/s"}
    phases = {"sketch_P_ms": sum(i["sketch_ms"] for i in infos) / len(infos), "update_ms": upd_ms,
              "ls_ms": sum(i["ls_ms"] for i in infos) / len(infos)}
    launches = sum(i["launches"] for i in infos)
    last = infos[-1]

    # end to end through the same C entry point with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        Wh = torch.empty(m, n, dtype=torch.float64, pin_memory=True)
        Wh.copy_(W.T)
        Wh = Wh.T
        Qh = rgs.colmajor_empty(n, m, dtype=torch.float32, pin=True)
        Rh = rgs.colmajor_empty(m, m, pin=True)
        qh = torch.empty(m, dtype=torch.float64, pin_memory=True)
        rgs.rgs_qr(h, sk, Wh, Qh, Rh, qscale=qh)
        torch.cuda.synchronize()
        e_steps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(e_steps):
            rgs.rgs_qr(h, sk, Wh, Qh, Rh, qscale=qh)
        torch.cuda.synchronize()
        e_s = (time.perf_counter() - t0) / e_steps
        e2e = {"value": world * total / e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": 8 * n * m,
               "d2h_bytes_per_step": 4 * n * m + 8 * m * m + 8 * m, "ms_per_step": 1e3 * e_s}

    gm = None
    if rank == 0 and not args.no_gmres:
        gm = run_gmres_c3(rgs, h)

    cpu = None
    if rank == 0 and not args.no_cpu:
        msub = 100
        v, dt, _ = cpu_sample_gbps(W[:, :msub].cpu().numpy(), n, k)
        cpu = {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"first {msub} of {m} columns (n=2^20, SRHT k=2000, f32 storage emulation), {dt:.1f} s"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
               "config": {"workload": WORKLOAD if m == M_COLS else f"profiling case m={m}", "n": n, "m": m, "k": k, "sketch": "srht", "qtype": "f32",
                          "cond": COND, "l2": "inputs 4.2 GB > L2, no flush", "parallelism": f"replicas{world}"},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk.summary(), "phases_ms": phases,
               "certificates": {"delta": last["delta"], "delta_tilde": last["delta_tilde"]},
               "rgmres": gm,
               "hbm_frac_whole_job": value / world / peak}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-gmres", action="store_true")
    ap.add_argument("--gmres-only", default="", help="profiling cases only: 'rgmres', 'cgs2' or both")
    ap.add_argument("--gmres-cycles", type=int, default=400)
    ap.add_argument("--cols", type=int, default=0, help="profiling cases only: override m (the bench line is m=500)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.gmres_only:
        run_gmres_profile(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
