"""RGS-Arnoldi (Alg. 3), randomized GMRES (Eq. hls) and CGS2-GMRES, in NumPy FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Alg. 3 (Sec. 4.1): w_1 = b, then RGS iteration 1; for i = 2..m, w_i = A q_{i-1}
(u_fine) and RGS iteration i.  Its R factor gives the Hessenberg matrix
H_m = R_m(1:m, 2:m) with A Q_{m-1} = Q_m H_m.

Randomized GMRES (Sec. 4.2): y = argmin_z || H_m z - r_11 e_1 ||, x = Q_{m-1} y;
this minimises the sketched residual || Theta (A x - b) || over K_{m-1}
(Eq. hls2).  The Hessenberg least-squares problem is solved here by
``numpy.linalg.lstsq`` (the library stands in for the Givens rotations the
paper uses; both are backward stable on this small dense problem).

Restarting (not in the paper, whose GMRES is a single cycle): cycle c starts
Alg. 3 from w_1 = r = b - A x (FP64), adds Q_{j} y to x, and recomputes the
true FP64 residual.  ``restart`` is the largest number of Arnoldi steps
(products with A) per cycle, so a cycle's basis has restart + 1 columns.

A restart cycle that leaves the true residual without a relative decrease of 2^-10 draws a new
Theta for the following cycles, the r-th such draw with seed + r * 0x9E3779B97F4A7C15 (mod 2^64)
and the caller's kind, n and k.  Each cycle minimises the sketched residual only; after many
cycles with one Theta the residual is no longer independent of it and can settle where Theta sees
little of it, when the cycles stop making progress.  (A rule of the restarted solver, like
restarting itself; ``refresh=False`` turns it off.)

Right preconditioning (Sec. 5, Ex. 3 applies A P): with ``precond`` given,
the operator is A M and x += M (Q y); with ``flexible=True`` each
z_j = M(q_j) is stored and x += Z y (a nonlinear M is allowed).

CGS2-GMRES: the same restarted GMRES on an l2-orthonormal Arnoldi basis built
with the projector (I - Q Q^T)^2 (Sec. 1.2), everything in FP64; the
comparator whose passes over Q the paper counts (Sec. 2.4).
"""
from __future__ import annotations

import numpy as np

from .sketch import Sketch
from .rgs import (BREAKDOWN_FACTOR, U_FINE, ls_householder, ls_richardson,
                  round_storage, update_fp32)


class ArnoldiCycle:
    pass


def rgs_arnoldi(matvec, w1, sketch, steps, ls="householder", sweeps=2, storage="f64",
                precond=None, stop=None):
    """Alg. 3 with up to ``steps`` products by the operator; returns the cycle state.

    ``matvec(v)`` is A v in FP64.  ``precond(v)`` (optional) is M v; then
    w_{i+1} = A M q_i and Z holds M q_i.  ``stop(rho, j)`` may end the cycle
    early given the sketched-residual estimate rho after j steps.
    """
    n = w1.shape[0]
    mcols = steps + 1
    k = sketch.k
    Qp = np.zeros((n, mcols))
    Q = np.zeros((n, mcols))
    Z = np.zeros((n, steps)) if precond is not None else None
    sigma = np.zeros(mcols)
    R = np.zeros((mcols, mcols))
    S = np.zeros((k, mcols))
    P = np.zeros((k, mcols))
    rho = []
    j_done = 0
    happy = False
    w = w1
    for i in range(mcols):
        if i > 0:
            v = Q[:, i - 1]
            if precond is not None:
                Z[:, i - 1] = precond(v)
                v = Z[:, i - 1]
            w = matvec(v)                                    # Alg. 3 step 3
        p = sketch.apply(w)                                  # Alg. 2 step 1
        P[:, i] = p
        x = ls_householder(S[:, :i], p) if ls == "householder" else ls_richardson(S[:, :i], p, sweeps)
        if storage == "f64":
            qp = w - Q[:, :i] @ x
        else:
            qp = update_fp32(w, Qp[:, :i], x * sigma[:i])
        qp = round_storage(qp, storage)
        sp = sketch.apply(qp)
        r = np.linalg.norm(sp)
        R[:i, i] = x
        R[i, i] = r
        if i > 0:
            j_done = i
            H = R[: i + 1, 1 : i + 1]
            g = np.zeros(i + 1)
            g[0] = R[0, 0]
            y, *_ = np.linalg.lstsq(H, g, rcond=None)
            rho.append(float(np.linalg.norm(H @ y - g)))
        if not r > BREAKDOWN_FACTOR * U_FINE * np.linalg.norm(p):
            if i == 0:
                raise RuntimeError("zero right-hand side")
            happy = True                                     # invariant Krylov space
            break
        S[:, i] = sp / r
        Qp[:, i] = qp
        sigma[i] = 1.0 / r
        Q[:, i] = qp * sigma[i]
        if i > 0 and stop is not None and stop(rho[-1], i):
            break
    out = ArnoldiCycle()
    out.steps = j_done
    out.Q, out.Qp, out.sigma, out.R, out.S, out.P, out.Z = Q, Qp, sigma, R, S, P, Z
    out.rho = np.array(rho)
    out.happy = happy
    j = j_done
    if j > 0:
        H = R[: j + 1, 1 : j + 1]
        if happy:
            H = H[:j, :]
        g = np.zeros(H.shape[0])
        g[0] = R[0, 0]
        out.y, *_ = np.linalg.lstsq(H, g, rcond=None)
    else:
        out.y = np.zeros(0)
    return out


class SolveResult:
    pass


REFRESH_STRIDE = 0x9E3779B97F4A7C15


def refresh_seed(seed, r):
    """Seed of the r-th redrawn Theta of a restarted solve."""
    return (int(seed) + int(r) * REFRESH_STRIDE) % (1 << 64)


def rgmres(A, b, sketch, restart, tol=1e-8, max_cycles=50, x0=None, ls="householder",
           sweeps=2, storage="f64", precond=None, flexible=False, inner_factor=0.5,
           fixed_steps=False, refresh=True):
    """Restarted randomized GMRES with RGS-Arnoldi; ``A`` is anything with ``A @ v``.

    Inner stop (unless ``fixed_steps``): sketched residual estimate
    <= threshold, initially inner_factor * tol * ||Theta b||; a cycle that stopped on it
    but left the true residual above tol multiplies the threshold of the following cycles by
    inner_factor * tol / (true relative residual).  Outer stop: ||b - A x|| <= tol ||b||.
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    sb = np.linalg.norm(sketch.apply(b))
    base_seed = sketch.seed
    res = SolveResult()
    res.true_residuals = []
    res.steps = []
    res.rho = []
    matvec = lambda v: A @ v
    r = b - A @ x
    res.true_residuals.append(float(np.linalg.norm(r) / bnorm))
    converged = res.true_residuals[-1] <= tol
    cycles = 0
    thr = inner_factor * tol * sb
    res.refreshes = 0
    while not converged and cycles < max_cycles:
        tr = res.true_residuals
        if refresh and cycles > 0 and not (tr[-1] < tr[-2] * (1.0 - 2.0 ** -10)):
            res.refreshes += 1
            sketch = Sketch(sketch.kind, sketch.n, sketch.k, refresh_seed(base_seed, res.refreshes))
        stop = None if fixed_steps else (lambda rho, j, thr=thr: rho <= thr)
        cyc = rgs_arnoldi(matvec, r, sketch, restart, ls, sweeps, storage,
                          precond=precond, stop=stop)
        j = cyc.steps
        if precond is None:
            dx = cyc.Q[:, :j] @ cyc.y
        elif flexible:
            dx = cyc.Z[:, :j] @ cyc.y
        else:
            dx = precond(cyc.Q[:, :j] @ cyc.y)
        x = x + dx
        r = b - A @ x
        res.true_residuals.append(float(np.linalg.norm(r) / bnorm))
        res.steps.append(j)
        res.rho.append(cyc.rho)
        cycles += 1
        converged = res.true_residuals[-1] <= tol
        if not converged and j < restart:
            thr *= min(1.0, inner_factor * tol / res.true_residuals[-1])
    res.x = x
    res.cycles = cycles
    res.converged = converged
    return res


def cgs2_arnoldi(matvec, r0, steps, stop=None):
    """l2 Arnoldi with CGS2: h = V^T w, w -= V h, twice; returns V, H, y, beta."""
    n = r0.shape[0]
    V = np.zeros((n, steps + 1))
    H = np.zeros((steps + 1, steps))
    beta = np.linalg.norm(r0)
    V[:, 0] = r0 / beta
    j_done = 0
    rho = []
    for j in range(steps):
        w = matvec(V[:, j])
        h1 = V[:, : j + 1].T @ w
        w = w - V[:, : j + 1] @ h1
        h2 = V[:, : j + 1].T @ w
        w = w - V[:, : j + 1] @ h2
        H[: j + 1, j] = h1 + h2
        hn = np.linalg.norm(w)
        H[j + 1, j] = hn
        j_done = j + 1
        Hj = H[: j + 2, : j + 1]
        g = np.zeros(j + 2)
        g[0] = beta
        y, *_ = np.linalg.lstsq(Hj, g, rcond=None)
        rho.append(float(np.linalg.norm(Hj @ y - g)))
        if not hn > BREAKDOWN_FACTOR * U_FINE * np.linalg.norm(h1):
            break
        V[:, j + 1] = w / hn
        if stop is not None and stop(rho[-1], j + 1):
            break
    Hj = H[: j_done + 1, :j_done]
    g = np.zeros(j_done + 1)
    g[0] = beta
    y, *_ = np.linalg.lstsq(Hj, g, rcond=None)
    return V[:, :j_done], H, y, np.array(rho)


def cgs2_gmres(A, b, restart, tol=1e-8, max_cycles=50, x0=None, inner_factor=0.5, fixed_steps=False):
    """Restarted FP64 GMRES with a CGS2 Arnoldi basis."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    res = SolveResult()
    res.true_residuals = []
    res.steps = []
    r = b - A @ x
    res.true_residuals.append(float(np.linalg.norm(r) / bnorm))
    converged = res.true_residuals[-1] <= tol
    cycles = 0
    thr = inner_factor * tol * bnorm
    while not converged and cycles < max_cycles:
        stop = None if fixed_steps else (lambda rho, j, thr=thr: rho <= thr)
        V, H, y, rho = cgs2_arnoldi(lambda v: A @ v, r, restart, stop)
        x = x + V[:, : len(y)] @ y
        r = b - A @ x
        res.true_residuals.append(float(np.linalg.norm(r) / bnorm))
        res.steps.append(len(y))
        cycles += 1
        converged = res.true_residuals[-1] <= tol
        if not converged and len(y) < restart:
            thr *= min(1.0, inner_factor * tol / res.true_residuals[-1])
    res.x = x
    res.cycles = cycles
    res.converged = converged
    return res
