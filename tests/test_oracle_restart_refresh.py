"""Pins of the restarted solver's Theta refresh (a rule of restarting, which the paper does not
use: its GMRES runs one cycle), CPU only.

A residual an SRHT cannot see: for n a power of two, v = D H e_j with row j not sampled gives
Theta v = P H D D H e_j / sqrt(k) = (n / sqrt(k)) P e_j = 0, as H H = n I and D D = I.  From an
x0 with b - A x0 = v plus a small visible part, every cycle with that Theta minimises the visible
part only, so the true residual stays at ||v|| (checked with ``refresh=False``).  With the rule, the
first cycle without a relative decrease of 2^-10 draws a new Theta (seed + 0x9E3779B97F4A7C15),
which sees v, and the solve converges.
"""
import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import gmres as og
from oracle.sketch import Sketch


def stalled_start(N=32, k=60, seed=3):
    """A (n = N^2 = 2^10), b, the sketch and an x0 whose residual Theta barely sees."""
    csr, _ = synth.diffusion_2d(N, 1.5, 4, 1)
    A = sp.csr_matrix((csr[2], csr[1], csr[0]))
    n = A.shape[0]
    sk = Sketch("srht", n, k, seed)
    sampled = set(int(r) for r in sk.rows)
    j = next(c for c in range(n) if c not in sampled)
    v = sk.signs * scipy.linalg.hadamard(n)[:, j]
    b = synth.rhs(n, 5)
    bn = np.linalg.norm(b)
    rng = np.random.default_rng(7)
    r0 = 1e-2 * bn * v / np.linalg.norm(v) + 1e-6 * bn * rng.standard_normal(n) / np.sqrt(n)
    x0 = spla.spsolve(A.tocsc(), b - r0)
    return A, b, sk, x0, v


def test_null_space_vector_is_invisible():
    A, b, sk, x0, v = stalled_start()
    assert np.abs(sk.apply(v)).max() <= 1e-12 * np.linalg.norm(v)
    other = Sketch("srht", sk.n, sk.k, og.refresh_seed(sk.seed, 1))
    assert np.linalg.norm(other.apply(v)) >= 0.1 * np.linalg.norm(v)


def test_fixed_theta_stalls_on_an_invisible_residual():
    A, b, sk, x0, _ = stalled_start()
    res = og.rgmres(A, b, sk, restart=20, tol=1e-8, max_cycles=6, x0=x0, refresh=False)
    tr = res.true_residuals
    assert not res.converged and res.refreshes == 0
    assert tr[-1] >= 0.9 * tr[0]                       # ||v|| untouched: no cycle makes progress


def test_refresh_after_the_first_stalled_cycle_converges():
    A, b, sk, x0, _ = stalled_start()
    res = og.rgmres(A, b, sk, restart=20, tol=1e-8, max_cycles=300, x0=x0)
    tr = res.true_residuals
    assert tr[1] >= (1.0 - 2.0 ** -10) * tr[0]          # cycle 1 stalls, so a new Theta is drawn
    assert tr[2] < 0.5 * tr[1]                          # ... which sees the residual
    assert res.converged and res.refreshes >= 1
    assert np.linalg.norm(b - A @ res.x) <= 1e-8 * np.linalg.norm(b)


def test_refresh_seed_is_the_stated_stride_mod_2_64():
    assert og.refresh_seed(5, 1) == 5 + 0x9E3779B97F4A7C15
    assert og.refresh_seed(2 ** 64 - 1, 1) == 0x9E3779B97F4A7C15 - 1
    assert og.refresh_seed(7, 3) == (7 + 3 * 0x9E3779B97F4A7C15) % 2 ** 64
