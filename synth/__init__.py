"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws inputs; it contains none of the RGS / GMRES arithmetic.
The shapes follow the paper's experiments (Sec. 5): tall matrices with m << n
and a prescribed singular-value decay for QR, and sparse PDE operators for
GMRES (the paper's SiO2 matrix and cloak model are not available, so
convection-diffusion stencils stand in for them).
"""
from __future__ import annotations

import numpy as np
import torch


def _gen(device, seed):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def haar_orthogonal(m, seed, device="cpu"):
    """Haar-distributed m x m orthogonal matrix (QR of a Gaussian with the signs of diag(R))."""
    g = _gen("cpu", seed)
    X = torch.randn(m, m, generator=g, dtype=torch.float64)
    Qh, Rh = torch.linalg.qr(X)
    d = torch.sign(torch.diagonal(Rh))
    d[d == 0] = 1.0
    return (Qh * d[None, :]).to(device)


def gdw_matrix(n, m, cond, seed, device="cpu"):
    """A = G D W: G iid N(0,1) (n x m), D = diag(logspace(0, -log10(cond), m)), W Haar.

    Returned as a torch FP64 tensor of shape (m, n): row j holds column j of A,
    i.e. A is stored column-major with leading dimension n.
    """
    g = _gen(device, seed)
    Gt = torch.randn(m, n, generator=g, dtype=torch.float64, device=device)   # G^T
    d = torch.logspace(0.0, -float(np.log10(cond)), m, dtype=torch.float64, device=device)
    W = haar_orthogonal(m, seed + 7919, device)
    # A^T = W^T D G^T
    return (W.T * d[None, :]) @ Gt


def f_mu_matrix(n, m, device="cpu"):
    """Sec. 5.1 test functions f_mu(x) = sin(10(mu+x)) / (cos(100(mu-x)) + 1.1) on an even grid.

    Returned column-major as a tensor of shape (m, n).
    """
    x = torch.linspace(0.0, 1.0, n, dtype=torch.float64, device=device)
    mu = torch.linspace(0.0, 1.0, m, dtype=torch.float64, device=device)
    return torch.sin(10.0 * (mu[:, None] + x[None, :])) / (torch.cos(100.0 * (mu[:, None] - x[None, :])) + 1.1)
