#!/usr/bin/env python
"""Benchmark of randomized Gram-Schmidt QR (Alg. 2) on one or more GB300 GPUs.

Workload (one "step" = one full rgs_qr call):
    A = G D W with n = 2^20 rows, m = 500 columns, D log-spaced from 1 to 1e-10,
    G iid N(0,1), W Haar orthogonal; SRHT sketch with k = 2000 over 2^20;
    basis stored in FP32 with FP32 update arithmetic; the sketched least squares
    (steps 2, 5, 6) in FP64 (RGS_FP64_LS); the SRHT's transform sums in double-float
    (FP32 pairs, about 2^-48: finer than the FP32 accumulation the workload allows).
    The same factorization with everything fine in FP64 ("fp64_fine") and with
    double-float least squares ("double_float_fine") is reported beside it.  Inputs (4.2 GB) are far larger than L2 (129 MB), so no
    flush is needed between steps.

Metric: whole-job algorithmic HBM throughput of the QR in GB/s, i.e.
    bytes = 8 n m                    (step 1, one pass over W)
          + sum_i [4 n i + 8 n + 4 n] (steps 3-4: read Q'_{i-1}, read w_i, write q'_i)
divided by the measured time.  With --gpus N (torchrun), every rank factors
its own independent matrix (weak scaling, no collective on the data path).

The second half of the metric is reported in the same line ("rgmres"): restarted
RGMRES(100) with RGS-Arnoldi (SRHT k = 400, FP32 basis; FP64 least squares, Givens and
restart residual; double-float sketch sums and products) against FP64 CGS2-GMRES(100) on the same
GPU, time to a relative residual of 1e-8 on a 3D convection-diffusion operator: 128^3
grid (n = 2,097,152, 7-point CSR, FP64 values), log-normal diffusion (sigma = 1,
correlation length 8 cells), Peclet number 50, iid N(0,1) right-hand side.  The
all-FP64-fine, all-double-float and BF16-basis variants are reported beside it.

"c1": the small FP64 factorization (n = 10,000, m = 100, cond 1e8, Gaussian k = 300),
latency-bound, reported as time per call.

"embedding_certificate": Sec. 3.2's a posteriori certificate omega_bar (eps* = 0.05) for the
factorization's basis and for one RGS-Arnoldi cycle's basis on the 128^3 operator.

"batched" in the same line: 256 independent 2D convection-diffusion RGMRES solves in one
persistent launch (rgmres_solve_batched, FP32 basis, Gaussian k = 2 restart) against the
same 256 systems solved one after another with FP64 CGS2-GMRES, at the full sizes (sides
64..512) for two fixed cycles each, and to 1e-8 on sides 16..64.

--c5 N prints a separate line for the learned preconditioner on N x N diffusion grids:
training-data harvest from plain RGMRES, training with the library's kernels, and held-out
solves with the learned (flexible), Jacobi and no preconditioner.

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
    """(total, update-pass) algorithmic bytes of one factorization.  Total: 8 n m (step 1 reads W)
    + sum_i 4 n (i + 3) (steps 3-4 read Q'_{i-1} and w_i, write q'_i).  With the SRHT the update
    pass of column i also reads w_{i+1} for its step-1 sketch, so the update launches carry
    8 n (m - 1) of the step-1 bytes and one separate sketch reads w_1."""
    steps34 = sum(esz * n * i + wbytes * n + esz * n for i in range(m))
    return wbytes * n * m + steps34, steps34 + wbytes * n * (m - 1)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_traffic(variant="fp64_fine"):
    """Mean per-launch DRAM traffic (bytes) of the fused update kernel over the m = 500 step, from the
    committed ncu summary of the same kernel variant (measured on one launch, scaled by the launch's
    algorithmic bytes); None when no capture of that variant is committed."""
    path = os.path.join(ROOT, "profiles", "rgs_update_sketch_c2.txt")
    key = f"traffic_bytes_per_launch_full_step_{variant}:"
    try:
        with open(path) as f:
            for line in f:
                if line.startswith(key):
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


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_sample_gbps(A_cols_host, n, k, storage="f32", threads=0):
    """Time the C oracle on the first columns of the workload with `threads` threads (0: all host
    cores); returns (GB/s, seconds, columns, threads used)."""
    from oracle import c_oracle
    c_oracle.build()
    used = c_oracle.set_threads(threads if threads > 0 else host_cores())
    sk = c_oracle.CSketch("srht", n, k, SEED)
    msub = A_cols_host.shape[1]
    t0 = time.perf_counter()
    c_oracle.rgs_qr(A_cols_host, sk, ls="householder", storage=storage)
    dt = time.perf_counter() - t0
    total, _ = qr_bytes(n, msub)
    return total / dt / 1e9, dt, msub, used


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
    used = 1
    for _ in range(args.steps):
        v, dt, _, used = cpu_sample_gbps(A, N_ROWS, K_SKETCH)
        vals.append(v)
        secs.append(dt)
    total, _ = qr_bytes(N_ROWS, msub)
    value = total * len(secs) / sum(secs) / 1e9
    sample = (f"first {msub} of {M_COLS} columns of the workload (n=2^20, SRHT k=2000, f32 storage emulation), "
              f"C oracle -O3 with OpenMP on {used} host threads")
    out = {"metric": METRIC, "value": value, "unit": "GB/s", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "sample_columns": msub},
           "cpu_baseline": {"value": value, "unit": "GB/s", "cores": used, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_gmres_c3(rgs, h, N=128, max_cycles=400, solvers=("rgmres", "rgmres_f64", "rgmres_df", "rgmres_bf16",
                                                          "cgs2")):
    """Time-to-1e-8 of RGMRES (FP32 basis; FP64 least squares, and the all-FP64 and all-double-float
    fine arithmetics beside it) and FP64 CGS2-GMRES on the 3D convection-diffusion system."""
    import torch
    import synth
    csr = synth.convdiff_3d(N, 50.0, 1.0, 8, 0)
    n = N ** 3
    (rp, ci, va), C = rgs.csr_to_device(*csr)
    b = torch.tensor(synth.rhs(n, 0), device="cuda")
    sk = rgs.rgs_sketch_create(h, "srht", n, 400, 0)
    # warm-up on a few cycles (kernels loaded, allocator primed)
    xw = torch.zeros(n, dtype=torch.float64, device="cuda")
    rgs.rgmres_solve(h, sk, C, b, xw, restart=100, max_cycles=1, ls64=True)
    rgs.rgmres_solve(h, sk, C, b, xw.zero_(), restart=100, max_cycles=1, fine64=True)
    rgs.rgmres_solve(h, sk, C, b, xw.zero_(), restart=100, max_cycles=1)
    rgs.cgs2_gmres_solve(h, C, b, xw.zero_(), restart=100, max_cycles=1)
    out = {"config": "convdiff3d 128^3 n=2097152 nnz=%d Pe=50 sigma=1 corr=8 restart=100 rtol=1e-8" % len(csr[1])}

    def rg(qd, fine64=False, ls64=False):
        return lambda x: rgs.rgmres_solve(h, sk, C, b, x, restart=100, rtol=1e-8, max_cycles=max_cycles, qdtype=qd,
                                          fine64=fine64, ls64=ls64)
    runs = (("rgmres_f32_fp64ls_srht400", "rgmres", rg(torch.float32, ls64=True)),
            ("rgmres_f32_fp64fine_srht400", "rgmres_f64", rg(torch.float32, fine64=True)),
            ("rgmres_f32_df_srht400", "rgmres_df", rg(torch.float32)),
            ("rgmres_bf16_fp64ls_srht400", "rgmres_bf16", rg(torch.bfloat16, ls64=True)),
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
    c = out.get("cgs2_gmres_f64")
    for name, key in (("rgmres_f32_fp64ls_srht400", "speedup_vs_cgs2_fp64"),
                      ("rgmres_f32_fp64fine_srht400", "speedup_vs_cgs2_fp64_all_fp64_fine"),
                      ("rgmres_f32_df_srht400", "speedup_vs_cgs2_fp64_double_float")):
        if c and name in out:
            out[key] = c["seconds"] / out[name]["seconds"]
    return out


def run_certificates(rgs, h, W, sk, n, m, k):
    """Sec. 3.2's embedding certificate omega_bar (eps* = 0.05, Phi an SRHT of Theta's size with
    another seed) for (a) the basis of the 2^20 x 500 factorization and (b) the Arnoldi basis of one
    RGMRES(100) cycle on the 128^3 convection-diffusion operator (FP32 bases, FP64 least squares)."""
    import torch
    import synth
    out = {}
    Q = rgs.colmajor_empty(n, m, dtype=torch.float32)
    R = rgs.colmajor_empty(m, m)
    S = rgs.colmajor_empty(k, m)
    qs = torch.empty(m, dtype=torch.float64, device="cuda")
    rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, S=S, flags=rgs.RGS_FP64_LS)
    phi = rgs.rgs_sketch_create(h, "srht", n, k, 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c = rgs.rgs_certify_embedding(h, sk, phi, Q, 0.05, vscale=qs, VTheta=S)
    torch.cuda.synchronize()
    out["qr_2e20x500_srht2000"] = {**c, "eps_star": 0.05, "ms": 1e3 * (time.perf_counter() - t0)}
    del Q, S
    N = 128
    csr = synth.convdiff_3d(N, 50.0, 1.0, 8, 0)
    n3 = N ** 3
    arrays, C = rgs.csr_to_device(*csr)
    b = torch.tensor(synth.rhs(n3, 0), device="cuda")
    th3 = rgs.rgs_sketch_create(h, "srht", n3, 400, 0)
    ph3 = rgs.rgs_sketch_create(h, "srht", n3, 400, 1)
    a = rgs.rgs_arnoldi_create(h, th3, n3, 101, torch.float32, ls64=True)
    rgs.rgs_arnoldi_start(h, a, b)
    for _ in range(100):
        rgs.rgs_arnoldi_step(h, a, csr=C)
    _, _, qs3 = rgs.rgs_arnoldi_get(h, a)
    Q3 = rgs.rgs_arnoldi_basis(a, 101)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c3 = rgs.rgs_certify_embedding(h, th3, ph3, Q3, 0.05, vscale=torch.tensor(qs3, device="cuda"))
    torch.cuda.synchronize()
    out["arnoldi_128cube_srht400_101cols"] = {**c3, "eps_star": 0.05, "ms": 1e3 * (time.perf_counter() - t0)}
    return out


def run_c1(rgs, h, reps=20):
    """The small FP64 factorization (n = 10,000, m = 100, cond 1e8, Gaussian k = 300 seed 0):
    latency-bound, so the time per call is reported (mean of `reps` calls after warm-up)."""
    import torch
    import synth
    n, m, k = 10000, 100, 300
    W = synth.gdw_matrix(n, m, 1e8, 0).cuda().T                  # (n, m) column-major
    sk = rgs.rgs_sketch_create(h, "gaussian", n, k, 0)
    Q = rgs.colmajor_empty(n, m)
    R = rgs.colmajor_empty(m, m)
    for _ in range(3):
        info = rgs.rgs_qr(h, sk, W, Q, R)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(reps):
        info = rgs.rgs_qr(h, sk, W, Q, R)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    E = W - Q @ R
    err = (torch.linalg.norm(E) / torch.linalg.norm(W)).item()
    return {"config": "rgs_qr n=10000 m=100 cond=1e8 gaussian k=300 seed 0, f64 basis", "ms_per_call": ms,
            "calls": reps, "delta": info["delta"], "delta_tilde": info["delta_tilde"], "rel_err_A_minus_QR": err,
            "launches_per_call": info["launches"]}


def c4_instances(rgs, NB, lo, hi, seed0):
    """The batched workload: 2D upwind convection-diffusion, sides uniform in [lo, hi], Peclet
    U[1, 100] at an angle U[0, 2 pi), restart U{30..80}, Gaussian k = 2 restart, b iid N(0,1)."""
    import torch
    import synth
    insts = []
    for i in range(NB):
        g = np.random.default_rng(seed0 + i)
        nx, ny = int(g.integers(lo, hi + 1)), int(g.integers(lo, hi + 1))
        ang, pe, m = float(g.uniform(0, 2 * np.pi)), float(g.uniform(1, 100)), int(g.integers(30, 81))
        csr = synth.convdiff_2d(nx, ny, pe, ang)
        arrays, C = rgs.csr_to_device(*csr)
        insts.append({"n": nx * ny, "m": m, "C": C, "arrays": arrays,
                      "b": torch.tensor(synth.rhs(nx * ny, seed0 + i), device="cuda")})
    return insts


def run_batched_c4(rgs, h):
    """256 instances in one persistent launch (FP32 basis) against 256 sequential FP64 CGS2-GMRES
    solves: (a) at the full sizes (sides 64..512) for two fixed cycles per instance (most of these
    unpreconditioned solves need tens of thousands of steps to reach 1e-8), (b) time to 1e-8 on
    sides 16..64, where every instance converges."""
    import torch

    def batched(insts, **kw):
        xs = [torch.zeros(I["n"], dtype=torch.float64, device="cuda") for I in insts]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = rgs.rgmres_solve_batched(h, [I["C"] for I in insts], [I["b"] for I in insts], xs,
                                       [I["m"] for I in insts], [2 * I["m"] for I in insts], sketch_seed=1,
                                       qdtype=torch.float32, **kw)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, res

    def sequential_cgs2(insts, **kw):
        dt, steps, conv = 0.0, 0, 0
        for I in insts:
            x = torch.zeros(I["n"], dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = rgs.cgs2_gmres_solve(h, I["C"], I["b"], x, restart=I["m"], **kw)
            torch.cuda.synchronize()
            dt += time.perf_counter() - t0
            steps += r["total_steps"]
            conv += r["converged"]
        return dt, steps, conv

    out = {}
    full = c4_instances(rgs, 256, 64, 512, 0)
    batched(full[:8], max_cycles=1, fixed_steps=True)                      # warm-up
    out["tuning"] = rgs.rgs_autotune_batched(h, [I["C"] for I in full], [I["b"] for I in full],
                                             [I["m"] for I in full], [2 * I["m"] for I in full], cycles=1,
                                             sketch_seed=1)
    with Clocks(0) as clk:
        dt, res = batched(full, max_cycles=2, fixed_steps=True)
    steps = sum(r["total_steps"] for r in res)
    ct, cs, _ = sequential_cgs2(full, max_cycles=2, fixed_steps=True)
    out["full_fixed_2_cycles"] = {
        "config": "256 x convdiff2d sides U[64,512] Pe U[1,100] restart U{30..80} gaussian k=2m, 2 fixed cycles",
        "sum_n": sum(I["n"] for I in full), "arnoldi_steps": steps, "batched_f32_s": dt,
        "batched_steps_per_s": steps / dt, "sequential_cgs2_f64_s": ct, "speedup": ct / dt,
        "clocks": clk.summary()}
    del full
    small = c4_instances(rgs, 256, 16, 64, 1000)
    dt, res = batched(small, max_cycles=400, rtol=1e-8)
    ct, cs, cconv = sequential_cgs2(small, max_cycles=400, rtol=1e-8)
    out["small_to_1e-8"] = {
        "config": "256 x convdiff2d sides U[16,64], same draws otherwise, rtol 1e-8",
        "batched_f32_s": dt, "converged": sum(r["converged"] for r in res),
        "arnoldi_steps": sum(r["total_steps"] for r in res), "sequential_cgs2_f64_s": ct,
        "cgs2_converged": cconv, "cgs2_steps": cs, "speedup": ct / dt, "launches": 1}
    return out


def run_c4_full(args):
    """The batched workload at its configured sizes (256 systems, sides U[64, 512]) solved to a
    relative residual of 1e-8 under a cycle cap: the batched solver (one persistent launch, FP32
    basis, autotuned shape) against the same 256 systems solved one after another with FP64
    CGS2-GMRES; converged counts, Arnoldi steps, times and the residuals reached."""
    import torch
    import paper_2011_05090_gb300 as rgs
    from paper_2011_05090_gb300 import build as libbuild
    libbuild.build()
    h = rgs.rgs_create()
    cap = args.c4_full
    full = c4_instances(rgs, 256, 64, 512, 0)
    Cs, bs = [I["C"] for I in full], [I["b"] for I in full]
    ms, ks = [I["m"] for I in full], [2 * I["m"] for I in full]
    tuning = rgs.rgs_autotune_batched(h, Cs, bs, ms, ks, cycles=1, sketch_seed=1)
    xs = [torch.zeros(I["n"], dtype=torch.float64, device="cuda") for I in full]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = rgs.rgmres_solve_batched(h, Cs, bs, xs, ms, ks, rtol=1e-8, max_cycles=cap, sketch_seed=1,
                                   qdtype=torch.float32)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    cg_s, cg_conv, cg_steps, cg_res = 0.0, 0, 0, []
    for I in full:
        x = torch.zeros(I["n"], dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = rgs.cgs2_gmres_solve(h, I["C"], I["b"], x, restart=I["m"], rtol=1e-8, max_cycles=cap)
        torch.cuda.synchronize()
        cg_s += time.perf_counter() - t0
        cg_conv += r["converged"]
        cg_steps += r["total_steps"]
        cg_res.append(r["rel_residual"])
    bres = [r["rel_residual"] for r in res]
    out = {"metric": "batched RGMRES time to 1e-8, 256 convection-diffusion systems at full size",
           "config": f"256 x convdiff2d sides U[64,512] Pe U[1,100] restart U{{30..80}} gaussian k=2m, rtol 1e-8, "
                     f"cap {cap} cycles", "sum_n": sum(I["n"] for I in full), "tuning": tuning,
           "batched_f32": {"seconds": tb, "converged": sum(r["converged"] for r in res),
                           "arnoldi_steps": sum(r["total_steps"] for r in res),
                           "median_rel_residual": float(np.median(bres)), "max_rel_residual": float(np.max(bres))},
           "sequential_cgs2_f64": {"seconds": cg_s, "converged": cg_conv, "arnoldi_steps": cg_steps,
                                   "median_rel_residual": float(np.median(cg_res)),
                                   "max_rel_residual": float(np.max(cg_res))},
           "speedup": cg_s / tb}
    print(json.dumps(out), flush=True)


def run_learned_c5(rgs, h, N=256, ell=16.0, nfields=40, rhs_per_field=8, cycles=3, steps=1500, ntest=3,
                   max_cycles=400, batch=16, nval=0, eval_every=1000):
    """Learned preconditioner: harvest restart residuals of plain RGMRES(50) solves on nfields
    diffusion problems (kappa = exp(1.5 g), correlation ell; right-hand sides from white noise to
    smooth), train the conv net with the residual-norm loss, then solve held-out fields with
    flexible RGMRES(50) + the net, Jacobi RGMRES(50) and plain RGMRES(50) (FP32 basis,
    Gaussian k = 100)."""
    import torch
    import synth
    from paper_2011_05090_gb300 import learned
    n = N * N
    sk = rgs.rgs_sketch_create(h, "gaussian", n, 100, 1)
    cap = nfields * rhs_per_field * cycles
    inputs = torch.zeros(cap, 2, N, N, device="cuda")
    stencils = torch.zeros(nfields, 5, N, N, device="cuda")
    field_of = torch.zeros(cap, dtype=torch.int64, device="cuda")
    t0 = time.perf_counter()
    w = 0
    for f in range(nfields):
        csr, lk = synth.diffusion_2d(N, 1.5, ell, 1000 + f)
        arrays, C = rgs.csr_to_device(*csr)
        stencils[f] = learned.stencil_from_csr(h, C, N, N)
        g = np.random.default_rng(f)
        for j in range(rhs_per_field):
            corr = float(g.choice([0.0, 1.0, 2.0, 4.0, 8.0])) * N / 32
            b = synth.gaussian_field((N, N), corr, g.integers(1 << 30)).ravel() if corr else g.standard_normal(n)
            got = learned.harvest(h, sk, C, torch.tensor(lk, device="cuda"), torch.tensor(b, device="cuda"),
                                  inputs, start=w, cycles=cycles, restart=50)
            field_of[w:w + got] = f
            w += got
    torch.cuda.synchronize()
    harvest_s = time.perf_counter() - t0
    net = rgs.rgs_convnet_create(h, N, N, batch, seed=7)
    t0 = time.perf_counter()
    scores = None
    if nval:
        # model selection on validation fields (seeds 800000..), distinct from training and test fields
        val = []
        for f in range(nval):
            csr, lk = synth.diffusion_2d(N, 1.5, ell, 800000 + f)
            arrays, C = rgs.csr_to_device(*csr)
            val.append((C, torch.tensor(synth.rhs(n, 55 + f), device="cuda"), torch.tensor(lk, device="cuda"),
                        arrays))
        losses, scores = learned.train_selected(h, net, inputs[:w], steps, stencils, field_of[:w], sk,
                                                [(c, b_, l_) for c, b_, l_, _ in val], eval_every=eval_every,
                                                batch=batch, lr=1e-3, max_cycles=max_cycles // 3)
    else:
        losses = learned.train(h, net, inputs[:w], steps, stencils, field_of[:w], batch=batch, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del inputs
    res = {"none": [], "jacobi": [], "learned": []}
    for f in range(ntest):
        csr, lk = synth.diffusion_2d(N, 1.5, ell, 900000 + f)
        arrays, C = rgs.csr_to_device(*csr)
        b = torch.tensor(synth.rhs(n, 77 + f), device="cuda")
        lkd = torch.tensor(lk, device="cuda")
        for pc in res:
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            r = learned.solve(h, sk, C, b, x, restart=50, rtol=1e-8, max_cycles=max_cycles, precond=pc, net=net,
                              logkappa=lkd)
            torch.cuda.synchronize()
            res[pc].append({"seconds": time.perf_counter() - t1, "steps": r["total_steps"],
                            "converged": r["converged"], "rel_residual": r["rel_residual"],
                            "fallback_cycle": r["fallback_cycle"]})
    summary = {k: {"converged": sum(e["converged"] for e in v), "mean_steps": float(np.mean([e["steps"] for e in v])),
                   "mean_seconds": float(np.mean([e["seconds"] for e in v])),
                   "median_rel_residual": float(np.median([e["rel_residual"] for e in v]))} for k, v in res.items()}
    return {"config": f"diffusion2d {N}^2 sigma=1.5 corr={ell} RGMRES(50) gaussian k=100 f32, cap {max_cycles} cycles",
            "training": {"fields": nfields, "inputs": w, "harvest_s": harvest_s, "steps": steps, "batch": batch,
                         "train_s": train_s, "ms_per_step": 1e3 * train_s / steps, "validation": scores,
                         "validation_fields": nval,
                         "loss_first_50": float(np.mean(losses[:50])), "loss_last_50": float(np.mean(losses[-50:]))},
            "held_out_fields": ntest, "summary": summary, "per_field": res}


def run_ex1(args):
    """Sec. 5.1, Ex. 1: the f_mu functions, n = 10^6 points, m = 300 parameters, P-SRHT sketches of
    k = 1500 and 5000 rows (10^6 is not a power of two).  RGS through rgs_qr with an FP32 basis in
    the unique-precision setting (RGS_FP32_FINE: everything in FP32) and in the paper's mixed
    precision (RGS_FP64_FINE: step 3 in FP32, everything else in FP64).  For i = 10, 20, ..., 300:
    cond(Q_i) and ||W_i - Q_i R_i||_F / ||W_i||_F (Q_i, R_i the leading blocks of the final factors,
    which RGS never changes after column i).  The C oracle's emulation of the mixed-precision run
    (FP32 step 3 with one rounding per fused multiply-add, FP64 elsewhere) is tabulated beside it."""
    import torch
    import paper_2011_05090_gb300 as rgs
    import synth
    from paper_2011_05090_gb300 import build as libbuild
    libbuild.build()
    h = rgs.rgs_create()
    n, m = 1000000, 300
    W = synth.f_mu_matrix(n, m, device="cuda").T                      # (n, m) column-major
    grid = list(range(10, m + 1, 10))

    def curves(Qb, R, Wd):
        G = (Qb.T @ Qb).cpu().numpy()
        cond = []
        for i in grid:
            ev = np.linalg.eigvalsh(G[:i, :i])              # cond(Q_i)^2 from the Gram matrix
            cond.append(float(np.sqrt(ev[-1] / ev[0])))
        E = Wd - Qb @ R
        ce = torch.cumsum((E * E).sum(dim=0), 0).cpu().numpy()
        cw = torch.cumsum((Wd * Wd).sum(dim=0), 0).cpu().numpy()
        err = [float(np.sqrt(ce[i - 1] / cw[i - 1])) for i in grid]
        return cond, err

    out = {"experiment": "Sec. 5.1 Ex. 1: f_mu(x) = sin(10(mu+x)) / (cos(100(mu-x)) + 1.1)",
           "config": {"n": n, "m": m, "sketch": "P-SRHT (s = 2^20)", "basis": "f32", "i": grid}, "runs": {}}
    for k in (1500, 5000):
        sk = rgs.rgs_sketch_create(h, "srht", n, k, 0)
        for name, flags in (("unique_fp32", rgs.RGS_FP32_FINE), ("mixed_fp32_fp64", rgs.RGS_FP64_FINE)):
            Q = rgs.colmajor_empty(n, m, dtype=torch.float32)
            R = rgs.colmajor_empty(m, m)
            qs = torch.empty(m, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, flags=flags)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            cond, err = curves(Q.double() * qs[None, :], R, W)
            out["runs"][f"k{k}_{name}"] = {"ms": 1e3 * dt, "delta": info["delta"], "cond_Q": cond, "rel_err": err}
            del Q
    if not args.no_cpu:
        from oracle import c_oracle
        c_oracle.build()
        c_oracle.set_threads(host_cores())
        Wh = W.cpu().numpy()
        for k in (1500,):
            t0 = time.perf_counter()
            ref = c_oracle.rgs_qr(Wh, c_oracle.CSketch("srht", n, k, 0), storage="f32")
            dt = time.perf_counter() - t0
            Qb = torch.tensor(ref.Qp * ref.sigma[None, :], device="cuda")
            cond, err = curves(Qb, torch.tensor(ref.R, device="cuda"), W)
            out["runs"][f"k{k}_mixed_fp32_fp64_oracle"] = {"s": dt, "cores": host_cores(), "delta": ref.delta,
                                                            "cond_Q": cond, "rel_err": err}
    r = out["runs"]
    out["checks"] = {
        "mixed_cond_max": max(max(r["k1500_mixed_fp32_fp64"]["cond_Q"]), max(r["k5000_mixed_fp32_fp64"]["cond_Q"])),
        "unique_cond_final_k1500": r["k1500_unique_fp32"]["cond_Q"][-1],
        "unique_cond_final_k5000": r["k5000_unique_fp32"]["cond_Q"][-1],
        "k5000_does_not_help_unique": r["k5000_unique_fp32"]["cond_Q"][-1] >= r["k1500_unique_fp32"]["cond_Q"][-1]}
    print(json.dumps(out), flush=True)


def run_profile_case(args):
    """Small cases for ncu captures (no bench line): 'update' and 'c2' run the QR workload (below);
    'convnet' runs three training steps and one
    forward pass of the network on a batch of four 256 x 256 grids; 'batched' runs 16 instances
    (sides 32..64) of the batched solver for two fixed cycles; 'ls' runs one RGS QR of a 2^16 x 500
    matrix with an SRHT of k = 2000 rows, an FP32 basis and FP64 least squares (the least-squares
    launches have the bench workload's k, m and arithmetic; only the row count is smaller)."""
    import torch
    import synth
    import paper_2011_05090_gb300 as rgs
    from paper_2011_05090_gb300 import build as libbuild
    from paper_2011_05090_gb300 import learned
    libbuild.build()
    h = rgs.rgs_create()
    if args.profile_case == "convnet":
        N, B = 256, 4
        net = rgs.rgs_convnet_create(h, N, N, B, seed=1)
        g = torch.Generator(device="cpu")
        g.manual_seed(0)
        x = torch.randn(B, 2, N, N, generator=g).cuda()
        csr, _ = synth.diffusion_2d(N, 1.5, 16, 0)
        arrays, C = rgs.csr_to_device(*csr)
        S = learned.stencil_from_csr(h, C, N, N).expand(B, 5, N, N).contiguous()
        for _ in range(3):
            rgs.rgs_convnet_train_step(h, net, x, x[:, 0].contiguous(), lr=1e-3, stencil=S)
        rgs.rgs_convnet_forward(h, net, x)
    elif args.profile_case in ("update", "c2"):
        # 'update': one factorization of the first 128 columns of the 2^20-row workload (update
        # launch j + 1 is column j; launch 0 sketches w_1); 'c2': two factorizations of the full
        # 2^20 x 500 workload (the second one's 1004 launches follow the first one's)
        n, k = 1 << 20, 2000
        m = 128 if args.profile_case == "update" else 500
        W = synth.gdw_matrix(n, m, 1e10, 0, device="cuda").T
        sk = rgs.rgs_sketch_create(h, "srht", n, k, 0)
        Q = rgs.colmajor_empty(n, m, dtype=torch.float32)
        R = rgs.colmajor_empty(m, m)
        qs = torch.empty(m, dtype=torch.float64, device="cuda")
        for _ in range(1 if args.profile_case == "update" else 2):
            rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, flags=rgs.RGS_FP64_LS)
    elif args.profile_case == "ls":
        n, m, k = 1 << 16, 500, 2000
        W = synth.gdw_matrix(n, m, 1e10, 0).T.to("cuda")
        sk = rgs.rgs_sketch_create(h, "srht", n, k, 0)
        Q = rgs.colmajor_empty(n, m, dtype=torch.float32)
        R = rgs.colmajor_empty(m, m)
        qs = torch.empty(m, dtype=torch.float64, device="cuda")
        rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, flags=rgs.RGS_FP64_LS)
    else:
        insts = c4_instances(rgs, 16, 32, 64, 0)
        xs = [torch.zeros(I["n"], dtype=torch.float64, device="cuda") for I in insts]
        rgs.rgmres_solve_batched(h, [I["C"] for I in insts], [I["b"] for I in insts], xs, [I["m"] for I in insts],
                                 [2 * I["m"] for I in insts], max_cycles=2, fixed_steps=True, qdtype=torch.float32)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case}), flush=True)


def run_gmres_profile(args):
    """Profiling case: the 128^3 RGMRES and/or CGS2 solve for a few cycles only (no bench line)."""
    import paper_2011_05090_gb300 as rgs
    from paper_2011_05090_gb300 import build as libbuild
    libbuild.build()
    h = rgs.rgs_create()
    print(json.dumps(run_gmres_c3(rgs, h, max_cycles=args.gmres_cycles, solvers=tuple(args.gmres_only.split(",")))),
          flush=True)


def max_over_ranks(ms, world, device):
    """The slowest rank's timed region (the whole job ends when it does)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms_max):
    """Whole-job throughput: the units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


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
    fine = rgs.RGS_FP64_LS                    # least-squares steps 2, 5, 6 in FP64 for the FP32 basis
    flags = rgs.RGS_QR_TIMINGS | fine
    tuning = rgs.rgs_autotune_update(h, sk, m // 2, torch.float32)     # launch shape of the update pass

    for _ in range(args.warmup):
        rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, flags=flags)
    torch.cuda.synchronize()

    # The timed region runs without per-launch events (they cost about 3 us of stream time per
    # launch); the same K steps are then run again with CUDA events around every launch on the
    # library's stream, and the per-kernel durations (roofline, phase split) come from that pass.
    infos, tinfos = [], []
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    istart, istop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        start.record()
        for _ in range(args.steps):
            infos.append(rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, flags=fine))
        stop.record()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        istart.record()
        for _ in range(args.steps):
            tinfos.append(rgs.rgs_qr(h, sk, W, Q, R, qscale=qs, flags=flags))
        istop.record()
        torch.cuda.synchronize()
    ms_max = max_over_ranks(start.elapsed_time(stop), world, "cuda")
    total, upd = qr_bytes(n, m)
    value = job_rate(total * args.steps, world, ms_max) / 1e9

    # dominant kernel: the fused update + sketch, timed per launch on the library's stream
    upd_ms = sum(i["update_ms"] for i in tinfos) / len(tinfos)
    peak, peak_kind = peaks()
    achieved = upd / (upd_ms * 1e-3) / 1e9
    traffic_full = profile_traffic("double_float")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_full if (traffic_full and m == M_COLS) else None,
                "kernel": "update_sketch_kernel<float,SRHT,double-float transform>",
                "bytes_per_launch": upd / m, "launches_per_step": m,
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured" else "fallback 6.8 TB/s",
                "timing": "CUDA events around each launch on the library stream, over the K steps that follow "
                          "the timed region (same inputs, same launch sequence)"}
    phases = {"sketch_P_ms": sum(i["sketch_ms"] for i in tinfos) / len(tinfos), "update_ms": upd_ms,
              "ls_ms": sum(i["ls_ms"] for i in tinfos) / len(tinfos),
              "instrumented_ms_per_step": istart.elapsed_time(istop) / args.steps}
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
        for _ in range(max(3, args.warmup)):            # the same warm-up as the device-timed value
            rgs.rgs_qr(h, sk, Wh, Qh, Rh, qscale=qh, flags=fine)
        torch.cuda.synchronize()
        # each call copies W in and Q', R, sigma out (pinned host buffers) and returns after its
        # stream synchronisation; the value is the mean over the same K steps as the device-timed
        # value, the median beside it (host-link bandwidth on a shared machine varies by call)
        e_times = []
        if world > 1:
            dist.barrier()
        for _ in range(args.steps):
            t0 = time.perf_counter()
            rgs.rgs_qr(h, sk, Wh, Qh, Rh, qscale=qh, flags=fine)
            e_times.append(time.perf_counter() - t0)
        e_s = max_over_ranks(1e3 * sum(e_times) / len(e_times), world, "cuda") * 1e-3   # slowest rank
        e2e = {"value": world * total / e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": 8 * n * m,
               "d2h_bytes_per_step": 4 * n * m + 8 * m * m + 8 * m, "ms_per_step": 1e3 * e_s,
               "ms_per_step_median": 1e3 * statistics.median(e_times), "steps": len(e_times),
               "ms_steps": [round(1e3 * t, 1) for t in e_times]}
        del Wh, Qh

    # the same factorization with the other fine arithmetics: everything fine in FP64, and
    # everything fine in double-float (FP32 pairs, about 2^-48 per operation); time, throughput,
    # certificates and the difference from the headline's R
    variants = {}
    if rank == 0:
        Rref = R.clone()
        Rd = rgs.colmajor_empty(m, m)
        for vname, vflags in (("fp64_fine", rgs.RGS_FP64_FINE), ("double_float_fine", 0),
                              ("richardson_fp64ls", rgs.RGS_FP64_LS | rgs.RGS_LS_RICHARDSON)):
            rgs.rgs_qr(h, sk, W, Q, Rd, qscale=qs, flags=vflags)
            torch.cuda.synchronize()
            start.record()
            for _ in range(3):
                iv = rgs.rgs_qr(h, sk, W, Q, Rd, qscale=qs, flags=vflags)
            stop.record()
            torch.cuda.synchronize()
            td = start.elapsed_time(stop) / 3e3
            variants[vname] = {"ms": 1e3 * td, "GB/s": total / td / 1e9, "hbm_frac": total / td / 1e9 / peaks()[0],
                               "delta": iv["delta"], "delta_tilde": iv["delta_tilde"],
                               "rel_diff_R_vs_headline": (torch.linalg.norm(Rd - Rref) / torch.linalg.norm(Rref)).item()}
            if vflags & rgs.RGS_LS_RICHARDSON:
                # Sec. 2.3's normal-equations alternative on this ill-conditioned matrix: its
                # least-squares time and the factorization error it leaves
                ti = rgs.rgs_qr(h, sk, W, Q, Rd, qscale=qs, flags=vflags | rgs.RGS_QR_TIMINGS)
                E = W - (Q.double() * qs[None, :]) @ Rd
                variants[vname]["ls_ms"] = ti["ls_ms"]
                variants[vname]["rel_err_W_minus_QR"] = (torch.linalg.norm(E) / torch.linalg.norm(W)).item()
                del E
        del Rd, Rref

    # the BF16-storage variant of the same factorization (FP64 least squares): time, throughput,
    # certificates
    bf16 = None
    if rank == 0:
        Qb = rgs.colmajor_empty(n, m, dtype=torch.bfloat16)
        rgs.rgs_qr(h, sk, W, Qb, R, qscale=qs, flags=fine)
        torch.cuda.synchronize()
        start.record()
        for _ in range(3):
            ib = rgs.rgs_qr(h, sk, W, Qb, R, qscale=qs, flags=fine)
        stop.record()
        torch.cuda.synchronize()
        tb = start.elapsed_time(stop) / 3e3
        total_b, _ = qr_bytes(n, m, esz=2)
        bf16 = {"ms": 1e3 * tb, "GB/s": total_b / tb / 1e9, "algorithmic_bytes": total_b,
                "delta": ib["delta"], "delta_tilde": ib["delta_tilde"]}
        del Qb

    gm = None
    if rank == 0 and not args.no_gmres:
        gm = run_gmres_c3(rgs, h)
    batched = None
    if rank == 0 and not args.no_batched:
        batched = run_batched_c4(rgs, h)
    c1 = run_c1(rgs, h) if rank == 0 else None
    certs = run_certificates(rgs, h, W, sk, n, m, k) if (rank == 0 and m == M_COLS) else None

    cpu = None
    if rank == 0 and not args.no_cpu:
        # the C oracle (-O3, OpenMP over independent rows and butterflies) on all host cores, and
        # on one core beside it, each on a sample of the first columns of the same matrix
        msub = 100
        Wc = W[:, :msub].cpu().numpy()
        v, dt, _, used = cpu_sample_gbps(Wc, n, k, threads=0)
        v1, dt1, _, _ = cpu_sample_gbps(Wc[:, :40].copy(), n, k, threads=1)
        cpu = {"value": v, "unit": "GB/s", "cores": used, "kind": "oracle",
               "sample": f"first {msub} of {m} columns (n=2^20, SRHT k=2000, f32 storage emulation), "
                         f"{dt:.1f} s on {used} threads",
               "single_thread": {"value": v1, "unit": "GB/s", "cores": 1,
                                 "sample": f"first 40 of {m} columns, {dt1:.1f} s"}}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
               "dtype_detail": "basis and update in f32 (u_crs); sketched least squares (steps 2, 5, 6), squared "
                               "norms, R and the scales in f64 (RGS_FP64_LS); SRHT transform sums in double-float "
                               "(f32 pairs, ~2^-48)",
               "data": "synthetic",
               "config": {"workload": WORKLOAD if m == M_COLS else f"profiling case m={m}", "n": n, "m": m, "k": k, "sketch": "srht", "qtype": "f32",
                          "cond": COND, "l2": "inputs 4.2 GB > L2, no flush", "parallelism": f"replicas{world}",
                          "tuning": tuning},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk.summary(), "phases_ms": phases,
               "certificates": {"delta": last["delta"], "delta_tilde": last["delta_tilde"]},
               "rgmres": gm, "batched": batched, "bf16_basis": bf16, "fine_variants": variants, "c1": c1,
               "embedding_certificate": certs,
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
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--profile-case", choices=["convnet", "batched", "ls", "update", "c2"], default="",
                    help="small case for an ncu capture only (no bench line)")
    ap.add_argument("--c5", type=int, default=0, metavar="N",
                    help="only the learned-preconditioner workload on N x N grids (one JSON line)")
    ap.add_argument("--c5-steps", type=int, default=1500)
    ap.add_argument("--c5-fields", type=int, default=40)
    ap.add_argument("--c5-test", type=int, default=3)
    ap.add_argument("--c5-cycles", type=int, default=400)
    ap.add_argument("--c5-val", type=int, default=0, help="validation fields for model selection (0: none)")
    ap.add_argument("--c5-eval-every", type=int, default=1000)
    ap.add_argument("--ex1", action="store_true", help="only the reproduction of Sec. 5.1's Ex. 1 (one JSON line)")
    ap.add_argument("--c4-full", type=int, default=0, metavar="CAP",
                    help="only the 256-system batch at full size to 1e-8 under a cap of CAP cycles (one JSON line)")
    args = ap.parse_args()
    if args.ex1:
        run_ex1(args)
    elif args.c4_full:
        run_c4_full(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.profile_case:
        run_profile_case(args)
    elif args.c5:
        import paper_2011_05090_gb300 as rgs
        from paper_2011_05090_gb300 import build as libbuild
        libbuild.build()
        h = rgs.rgs_create()
        out = run_learned_c5(rgs, h, N=args.c5, ell=args.c5 / 16.0, nfields=args.c5_fields, steps=args.c5_steps,
                             ntest=args.c5_test, max_cycles=args.c5_cycles, nval=args.c5_val,
                             eval_every=args.c5_eval_every)
        print(json.dumps({"metric": "learned preconditioner: iterations and time to 1e-8", **out}), flush=True)
    elif args.gmres_only:
        run_gmres_profile(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
