"""Training data, training and use of the learned right preconditioner (flexible RGMRES).

The network is trained on residuals that plain restarted RGMRES produces itself.  After restart
cycle j of a solve of A x = b, the residual r_j = b - A x_j and the error e_j = A^{-1} r_j form
the pair (r_j, e_j) that shows the map r -> A^{-1} r a right preconditioner M approximates.
The loss measures the error of M(r_j) in the residual norm,
||A (M(r_j) - e_j)|| = ||A M(r_j) - r_j||, so it needs r_j and A but never e_j itself; it is
what a right preconditioner must make small (an error that is small in the plain norm but
rough is amplified by A and makes a useless preconditioner).  A solve started from a
white-noise right-hand side yields residuals from white noise (r_0 = b) to smooth (late
cycles), the range of vectors a flexible solver later applies M to.  Arnoldi basis vectors
of the cycles can be added as further inputs.

Inputs are scaled to unit root mean square, rms(v) = ||v|| / sqrt(n), like the network's
input inside the solver (rgs_convnet_input); the operators travel as 5-point stencils (centre,
west, east, north, south coefficients of each row; rgs_csr_to_stencil).

Everything numerical runs in librgs (the solver, the products with A, the network's forward,
backward and Adam kernels); this module only moves tensors between those calls.
"""
from __future__ import annotations

import math

import torch

from . import (rgmres_set_preconditioner, rgmres_solve, rgs_arnoldi_basis, rgs_arnoldi_create, rgs_arnoldi_start,
               rgs_arnoldi_step, rgs_convnet_input, rgs_convnet_train_step, rgs_csr_residual, rgs_csr_to_stencil)


def stencil_from_csr(h, csr, H, W):
    """(5, H, W) FP32 coefficients of a 5-point operator on an H x W grid (x fastest) from its CSR
    (the library's rgs_csr_to_stencil); raises if a row reaches another neighbour."""
    return rgs_csr_to_stencil(h, csr, H, W)


def harvest(h, sk, csr, logkappa, b, inputs, start=0, cycles=100, restart=50, qdtype=torch.float32,
            basis_cols=()):
    """Run plain RGMRES(restart) on A x = b from x = 0 and write, for j = 0, 1, ..., the input
    (r_j / rms(r_j), log kappa) of every restart residual into inputs[start:] (N x 2 x H x W
    FP32), followed, for each column index c in ``basis_cols``, by the c-th Arnoldi basis vector
    of an RGS-Arnoldi process started from r_j.  Stops after ``cycles`` residuals, when the
    solve reaches 1e-10, or when ``inputs`` is full.  Returns the number of rows written."""
    H, W = logkappa.shape
    lk = logkappa.reshape(-1).double().contiguous()
    x = torch.zeros_like(b)
    N = inputs.shape[0]
    w = start
    arn = None
    if basis_cols:
        arn = rgs_arnoldi_create(h, sk, H * W, max(basis_cols) + 1, qdtype)

    def put(v, nonzero=True):
        nonlocal w
        if w >= N or not nonzero:
            return False
        rgs_convnet_input(h, v, lk, inputs[w].view(2, H * W))
        w += 1
        return True

    for j in range(cycles):
        r, rnorm = rgs_csr_residual(h, csr, x, b)
        if not put(r, rnorm > 0):
            break
        if arn is not None:
            rgs_arnoldi_start(h, arn, r)
            for _ in range(max(basis_cols)):
                rgs_arnoldi_step(h, arn, csr=csr)
            Q = rgs_arnoldi_basis(arn, max(basis_cols) + 1)
            for c in basis_cols:
                if not put(Q[:, c].double().contiguous()):
                    break
        res = rgmres_solve(h, sk, csr, b, x, restart=restart, rtol=1e-10, max_cycles=1, qdtype=qdtype)
        if res["converged"] or w >= N:
            break
    return w - start


def train(h, net, inputs, steps, stencils, field_of, batch=16, lr=1e-3, lr_final=1e-5, seed=0, log_every=0):
    """Adam on random minibatches of ``inputs`` for ``steps`` steps with the residual-norm loss
    mean_b ||A_b net(x_b) - r_b||^2 / ||r_b||^2 (r_b = channel 0 of x_b, A_b =
    stencils[field_of[b]]), the learning rate decaying along a cosine from ``lr`` to
    ``lr_final``.  Returns the per-step losses."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    N = inputs.shape[0]
    losses = []
    for t in range(steps):
        idx = torch.randint(0, N, (batch,), generator=g).to(inputs.device)
        xb = inputs.index_select(0, idx).contiguous()
        rb = xb[:, 0].contiguous()
        sb = stencils.index_select(0, field_of.index_select(0, idx)).contiguous()
        a = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * t / max(steps - 1, 1)))
        losses.append(rgs_convnet_train_step(h, net, xb, rb, lr=a, stencil=sb))
        if log_every and (t % log_every == 0 or t == steps - 1):
            print(f"step {t}: loss {losses[-1]:.4f} (lr {a:.2e})", flush=True)
    return losses


def validation_score(h, sk, systems, net, restart=50, max_cycles=100):
    """Cost of flexible RGMRES with the network on validation systems [(csr, b, log kappa)]: the
    Arnoldi steps to 1e-8, or for a solve that stops short, the step budget times
    (1 + log10(residual reached / 1e-8)).  Lower is better."""
    score = 0.0
    for csr, b, lk in systems:
        x = torch.zeros_like(b)
        r = solve(h, sk, csr, b, x, restart=restart, rtol=1e-8, max_cycles=max_cycles, precond="learned", net=net,
                  logkappa=lk)
        if r["converged"]:
            score += r["total_steps"]
        else:
            rel = max(r["rel_residual"], 1e-8) if r["rel_residual"] == r["rel_residual"] else 1.0
            score += restart * max_cycles * (1.0 + math.log10(rel / 1e-8))
    return score


def train_selected(h, net, inputs, steps, stencils, field_of, sk, val_systems, eval_every=1000, batch=16, lr=1e-3,
                   lr_final=1e-5, seed=0, restart=50, max_cycles=100, log=False):
    """train() in rounds of eval_every steps on one learning-rate schedule, scoring the network on
    the validation systems after each round and keeping the parameters of the best round (the
    training loss tracks the solver's behaviour only loosely).  Returns (losses, scores)."""
    from . import rgs_convnet_get_params, rgs_convnet_set_params
    losses, scores = [], []
    best, best_p = float("inf"), None
    done = 0
    while done < steps:
        n = min(eval_every, steps - done)
        # the slice [done, done + n) of one cosine schedule over all steps
        a0 = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * done / max(steps - 1, 1)))
        a1 = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * (done + n - 1) / max(steps - 1, 1)))
        losses += train(h, net, inputs, n, stencils, field_of, batch=batch, lr=a0, lr_final=a1, seed=seed + done)
        done += n
        sc = validation_score(h, sk, val_systems, net, restart=restart, max_cycles=max_cycles)
        scores.append((done, sc))
        if log:
            print(f"step {done}: loss {sum(losses[-50:]) / min(50, len(losses)):.4f}, validation cost {sc:.0f}",
                  flush=True)
        if sc < best:
            best, best_p = sc, rgs_convnet_get_params(h, net)
    if best_p is not None:
        rgs_convnet_set_params(h, net, best_p)
    return losses, scores


def solve(h, sk, csr, b, x, restart=50, rtol=1e-8, max_cycles=1000, qdtype=torch.float32, precond="none",
          net=None, logkappa=None):
    """rgmres_solve with the right preconditioner ``precond`` ("none", "jacobi" or "learned";
    the learned one runs flexible), restoring "none" afterwards."""
    if precond == "learned":
        lk = logkappa.reshape(-1).to(torch.float64).contiguous()
        rgmres_set_preconditioner(h, "learned", net, lk, flexible=True)
    else:
        rgmres_set_preconditioner(h, precond)
    try:
        return rgmres_solve(h, sk, csr, b, x, restart=restart, rtol=rtol, max_cycles=max_cycles, qdtype=qdtype)
    finally:
        rgmres_set_preconditioner(h, "none")
