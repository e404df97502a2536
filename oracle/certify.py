"""A posteriori certification of the epsilon-embedding property (Sec. 3.2), in NumPy FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Theta is an epsilon-embedding for V (n x m) when | ||Theta x||^2 - ||x||^2 | <= epsilon ||x||^2
for every x in range(V) (Sec. 2.2).  The smallest such epsilon is

    omega = max(1 - s_min^2, s_max^2 - 1),   s = singular values of Theta U,

with U an orthonormal basis of range(V) (computable only with access to V itself).  The
certificate of Sec. 3.2 (Prop. cert01) needs only the two sketches V^Theta = Theta V and
V^Phi = Phi V with a second sketch Phi drawn independently of V and Theta: with X such that
V^Phi X is orthonormal,

    omega_bar = max(1 - (1 - eps*) s_min^2, (1 + eps*) s_max^2 - 1),   s = sing. values of V^Theta X,

and Theta is an omega_bar-embedding for V with probability at least 1 - delta* when Phi is an
(eps*, delta*, 1) oblivious embedding.  X is taken here as R^{-1} from the Householder QR of
V^Phi (LAPACK), and the singular values come from LAPACK's SVD.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def omega_exact(V, theta_apply):
    """omega for V (n x m) and the sketch ``theta_apply`` (an n-row block -> k-row block)."""
    U, _ = np.linalg.qr(np.asarray(V, dtype=np.float64))
    s = np.linalg.svd(theta_apply(U), compute_uv=False)
    return float(max(1.0 - s[-1] ** 2, s[0] ** 2 - 1.0))


def omega_bar(VTheta, VPhi, eps_star=0.05):
    """Prop. cert01: the certificate from the sketches V^Theta (k x m) and V^Phi (k' x m).
    Returns (omega_bar, s_min, s_max) with s the singular values of V^Theta X."""
    VTheta = np.asarray(VTheta, dtype=np.float64)
    VPhi = np.asarray(VPhi, dtype=np.float64)
    _, R = np.linalg.qr(VPhi)                                # V^Phi = Q R, so X = R^{-1}
    Z = scipy.linalg.solve_triangular(R, VTheta.T, trans="T", lower=False).T   # V^Theta R^{-1}
    s = np.linalg.svd(Z, compute_uv=False)
    smin, smax = float(s[-1]), float(s[0])
    wb = max(1.0 - (1.0 - eps_star) * smin ** 2, (1.0 + eps_star) * smax ** 2 - 1.0)
    return float(wb), smin, smax


def cert2_bound(omega, eps_prime, eps_star=0.05):
    """Prop. cert2: omega_bar <= (1 + eps*) (1 - eps')^{-1} (1 + omega) - 1 when Phi is an
    eps'-embedding for V."""
    return (1.0 + eps_star) * (1.0 + omega) / (1.0 - eps_prime) - 1.0
