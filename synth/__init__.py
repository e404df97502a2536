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


def gaussian_field(shape, corr_len, seed):
    """Zero-mean, unit-variance Gaussian random field: white noise smoothed by a Gaussian kernel.

    The kernel's standard deviation is corr_len / sqrt(2) cells, so the field's
    correlation function is exp(-d^2 / (2 corr_len^2)) (periodic FFT convolution).
    """
    rng = np.random.default_rng(int(seed))
    noise = rng.standard_normal(shape)
    k = [np.fft.fftfreq(s) for s in shape]
    grids = np.meshgrid(*k, indexing="ij")
    sd = corr_len / np.sqrt(2.0)
    filt = np.exp(-2.0 * np.pi ** 2 * sd ** 2 * sum(g ** 2 for g in grids))
    f = np.real(np.fft.ifftn(np.fft.fftn(noise) * filt))
    f -= f.mean()
    std = f.std()
    return f / std if std > 0 else f


def convdiff_csr(shape, kappa, velocity):
    """Upwind finite-volume matrix of -div(kappa grad u) + v . grad u on the unit box.

    ``shape`` = interior cells per axis (last axis fastest in the row ordering), h = 1/(N+1),
    homogeneous Dirichlet boundary; face diffusivities are harmonic means; the
    convection term is first-order upwind.  Returns (rowptr, colind, val) as
    int32 / int32 / FP64 with column indices ascending in each row.
    """
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    kappa = np.asarray(kappa, dtype=np.float64).reshape(shape)
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    diag = np.zeros(shape)
    rows, cols, vals = [], [], []
    for ax in range(d):
        h = 1.0 / (shape[ax] + 1)
        v = float(velocity[ax])
        for side in (-1, 1):
            nb_k = np.roll(kappa, -side, axis=ax)
            inside = np.ones(shape, dtype=bool)
            sl = [slice(None)] * d
            sl[ax] = slice(-1, None) if side == 1 else slice(0, 1)
            inside[tuple(sl)] = False
            kf = np.where(inside, 2.0 * kappa * nb_k / (kappa + nb_k), kappa) / h ** 2
            diag += kf
            conv = 0.0
            if v > 0 and side == -1:
                conv = v / h          # v (u_i - u_{i-1}) / h
            elif v < 0 and side == 1:
                conv = -v / h         # v (u_{i+1} - u_i) / h
            diag += conv
            nb = np.roll(idx, -side, axis=ax)
            rows.append(idx[inside])
            cols.append(nb[inside])
            vals.append(-(kf[inside] + conv))
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    r = np.concatenate([a.ravel() for a in rows])
    c = np.concatenate([a.ravel() for a in cols])
    v = np.concatenate([a.ravel() for a in vals])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr.astype(np.int32), c.astype(np.int32), v


def convdiff_3d(N, peclet, sigma, corr_len, seed):
    """3D variable-coefficient convection-diffusion on an N^3 grid (7-point stencil).

    kappa = exp(sigma g) with g a unit-variance Gaussian field of correlation length
    ``corr_len`` cells; constant velocity of magnitude ``peclet`` along (1,1,1)/sqrt(3)
    (Peclet number with unit length and unit reference diffusivity).
    """
    g = gaussian_field((N, N, N), corr_len, seed)
    v = peclet * np.ones(3) / np.sqrt(3.0)
    return convdiff_csr((N, N, N), np.exp(sigma * g), v)


def convdiff_2d(nx, ny, peclet, angle, kappa=None):
    """2D convection-diffusion (5-point) with velocity peclet * (cos a, sin a)."""
    kap = np.ones((nx, ny)) if kappa is None else kappa
    v = peclet * np.array([np.cos(angle), np.sin(angle)])
    return convdiff_csr((nx, ny), kap, v)


def rhs(n, seed):
    """Right-hand side with iid N(0,1) entries."""
    return np.random.default_rng(int(seed) + 1_000_003).standard_normal(n)


def csr_dense(csr, n=None):
    rowptr, colind, val = csr
    n = len(rowptr) - 1 if n is None else n
    A = np.zeros((n, n))
    for r in range(n):
        A[r, colind[rowptr[r]:rowptr[r + 1]]] += val[rowptr[r]:rowptr[r + 1]]
    return A


def diffusion_2d(N, sigma, corr_len, seed):
    """-div(kappa grad u) = f on an N x N grid, kappa = exp(sigma g), g a unit-variance Gaussian
    field of correlation length ``corr_len`` cells (seed).  The finite-volume matrix is scaled
    by h^2 so that its entries are O(kappa).  Returns ((rowptr, colind, val), log kappa (N x N))."""
    g = gaussian_field((N, N), corr_len, seed)
    rowptr, colind, val = convdiff_csr((N, N), np.exp(sigma * g), np.zeros(2))
    h = 1.0 / (N + 1)
    return (rowptr, colind, val * h * h), sigma * g
