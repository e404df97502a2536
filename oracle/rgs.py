"""Randomized Gram-Schmidt QR (Alg. 2), written step by step in NumPy FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Alg. 2 (Sec. 2.3), for i = 1..m:
  1. p_i = Theta w_i                                     (u_fine)
  2. R(1:i-1, i) = argmin_y || S_{i-1} y - p_i ||          (u_fine)
  3. q'_i = w_i - Q_{i-1} R(1:i-1, i)                     (u_crs)
  4. s'_i = Theta q'_i                                    (u_fine)
  5. r_ii = || s'_i ||                                    (u_fine)
  6. s_i = s'_i / r_ii                                    (u_fine)
  7. q_i = q'_i / r_ii                                    (u_fine)
  8. Delta_m = ||I - S^T S||_F, Delta~_m = ||P - S R||_F / ||P||_F.

Least-squares solvers for step 2 (Sec. 2.3):
  * ``"householder"``: the QR factorisation by Householder reflections used in
    the paper's experiments (Sec. 5); here LAPACK's via ``numpy.linalg.qr``
    followed by a triangular solve;
  * ``"richardson"``: the normal equations S^T S x = S^T p solved by a few
    Richardson sweeps x <- x + S^T (p - S x) from x = 0, which the paper
    proposes when S is of moderate size.

Precision model (Sec. 2.3, the assumptions of Sec. 3 on Delta q_i): W and Q are
held in the working (storage) precision u_crs; step 3 runs in u_crs; everything
else in FP64.  Step 7 is required to carry only u_fine error, so the basis is
kept as the stored q'_i together with the FP64 factor 1/r_ii (``Qp``, ``sigma``);
the FP64 product ``Q = Qp * sigma`` is the basis the algorithm defines.
Storage ``"f32"``/``"bf16"`` rounds q'_i to that format and runs step 3 as an
FP32 fused multiply-add chain summed over j = 1..i-1 in order, each multiply-add
rounded once (``fma32``: the FP32 product is exact in FP64, the difference is
carried exactly as a TwoSum pair and that pair is rounded to FP32 once).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

U_FINE = 2.0 ** -53
BREAKDOWN_FACTOR = 16.0


class BreakdownError(RuntimeError):
    def __init__(self, column):
        super().__init__(f"RGS breakdown at column {column}")
        self.column = column


def round_bf16(x):
    """Round FP64 values to bfloat16 (round to nearest even), returned as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_storage(x, storage):
    if storage == "f64":
        return np.asarray(x, dtype=np.float64)
    if storage == "f32":
        return np.asarray(x, dtype=np.float32).astype(np.float64)
    if storage == "bf16":
        return round_bf16(x)
    raise ValueError(storage)


def ls_householder(S, p):
    """argmin ||S y - p|| by Householder QR of S (LAPACK geqrf) and back substitution."""
    if S.shape[1] == 0:
        return np.zeros(0)
    Qh, Rh = np.linalg.qr(S, mode="reduced")
    return scipy.linalg.solve_triangular(Rh, Qh.T @ p, lower=False)


def ls_richardson(S, p, sweeps=2):
    """Richardson sweeps x <- x + S^T (p - S x) on the normal equations, from x = 0."""
    x = np.zeros(S.shape[1])
    for _ in range(sweeps):
        x = x + S.T @ (p - S @ x)
    return x


def fma32(acc, c, q):
    """One FP32 fused multiply-add acc - c q, rounded once to FP32 (round to nearest even).

    acc, c, q hold FP32 values (as FP64 arrays).  The product c q has at most 48 significant
    bits, so it is exact in FP64.  The difference acc - c q is carried exactly as the
    unevaluated pair (s, e) of Knuth's TwoSum (s = fl64(acc - c q), e the rounding error).
    Rounding that pair to FP32: s rounds correctly unless s lies exactly halfway between two
    FP32 neighbours (both are FP64 numbers, so no FP32 rounding boundary lies strictly between
    the exact value and s); there the sign of e says on which side the exact value lies, and
    e = 0 is a true tie, which FP32 conversion resolves to even.
    """
    acc = np.asarray(acc, dtype=np.float64)
    prod = np.asarray(c, dtype=np.float64) * np.asarray(q, dtype=np.float64)
    s = acc - prod
    bb = s - acc
    e = (acc - (s - bb)) + (-prod - bb)
    r = s.astype(np.float32)
    rd = r.astype(np.float64)
    toward = np.where(s > rd, np.float32(np.inf), np.float32(-np.inf)).astype(np.float32)
    other = np.nextafter(r, toward)
    od = other.astype(np.float64)
    tie = (e != 0.0) & (rd != s) & (0.5 * (rd + od) == s)
    pick_other = tie & ((e > 0.0) == (od > rd))
    return np.where(pick_other, other, r).astype(np.float64)


def update_fp32(w, Qp, c):
    """Step 3 in FP32: acc = fl32(w); acc = fma32(-c_j, q'_j, acc) for j = 1..i-1, with
    c_j = fl32(c) and every multiply-add rounded once, as a fused multiply-add does."""
    acc = np.asarray(w, dtype=np.float32).astype(np.float64)
    c32 = np.asarray(c, dtype=np.float32).astype(np.float64)
    for j in range(Qp.shape[1]):
        acc = fma32(acc, c32[j], Qp[:, j])
    return acc


class QRResult:
    pass


def ls_householder_f32(S, p):
    """argmin ||S y - p|| with every operation in FP32 (LAPACK sgeqrf and an FP32 triangular solve)."""
    if S.shape[1] == 0:
        return np.zeros(0)
    Qh, Rh = np.linalg.qr(np.asarray(S, dtype=np.float32), mode="reduced")
    y = scipy.linalg.solve_triangular(Rh, Qh.T @ np.asarray(p, dtype=np.float32), lower=False)
    return np.asarray(y, dtype=np.float32).astype(np.float64)


def rgs_qr(W, sketch, ls="householder", sweeps=2, storage="f64", P=None, fine="f64"):
    """Alg. 2 on the n x m matrix W with sketch ``sketch`` (an ``oracle.sketch.Sketch``).

    fine="f32" is the unique-precision setting of Sec. 5.1 (u_fine = u_crs = FP32, with an FP32
    basis): the sketches, the least-squares problem, r_ii, s_i and 1/r_ii in FP32 arithmetic.
    Returns an object with Q (FP64 basis), Qp (stored q'), sigma (1/r_ii), R, S,
    P, delta (Delta_m), delta_tilde (Delta~_m).
    """
    W = np.asarray(W, dtype=np.float64)
    n, m = W.shape
    up = fine == "f32"
    if up and storage == "f64":
        raise ValueError("the unique-precision setting needs an FP32 or BF16 basis")
    if P is None:
        P = sketch.apply_f32(W) if up else sketch.apply(round_storage(W, "f64"))   # step 1, all columns
    k = P.shape[0]
    if m > k:
        raise ValueError("Alg. 2 needs m <= k")
    Qp = np.zeros((n, m))
    Q = np.zeros((n, m))
    sigma = np.zeros(m)
    R = np.zeros((m, m))
    S = np.zeros((k, m))
    for i in range(m):
        p = P[:, i]
        if up:
            x = ls_householder_f32(S[:, :i], p)              # step 2 in FP32
        elif ls == "householder":
            x = ls_householder(S[:, :i], p)                  # step 2
        elif ls == "richardson":
            x = ls_richardson(S[:, :i], p, sweeps)
        else:
            raise ValueError(ls)
        if storage == "f64":
            qp = W[:, i] - Q[:, :i] @ x                      # step 3
        else:
            qp = update_fp32(W[:, i], Qp[:, :i], x * sigma[:i])
        qp = round_storage(qp, storage)
        if up:
            sp = sketch.apply_f32(qp)                        # step 4 in FP32
            r = float(np.linalg.norm(sp.astype(np.float32)))  # step 5: FP32 norm
            # the breakdown rule keeps its FP64 threshold: it detects exactly dependent columns,
            # and numerically dependent ones continue, as in Sec. 5.1's unique-precision run
            if not r > BREAKDOWN_FACTOR * U_FINE * float(np.linalg.norm(p.astype(np.float32))):
                raise BreakdownError(i)
            S[:, i] = (sp.astype(np.float32) / np.float32(r)).astype(np.float64)   # step 6
            sigma[i] = float(np.float32(1.0) / np.float32(r))
        else:
            sp = sketch.apply(qp)                            # step 4
            r = np.linalg.norm(sp)                           # step 5
            if not r > BREAKDOWN_FACTOR * U_FINE * np.linalg.norm(p):
                raise BreakdownError(i)
            S[:, i] = sp / r                                 # step 6
            sigma[i] = 1.0 / r
        Qp[:, i] = qp
        Q[:, i] = qp * sigma[i]                              # step 7
        R[:i, i] = x
        R[i, i] = r
    out = QRResult()
    out.Q, out.Qp, out.sigma, out.R, out.S, out.P = Q, Qp, sigma, R, S, P
    out.delta, out.delta_tilde = certificates(S, R, P)
    return out


def certificates(S, R, P):
    """Step 8: Delta_m = ||I - S^T S||_F and Delta~_m = ||P - S R||_F / ||P||_F."""
    m = S.shape[1]
    delta = np.linalg.norm(np.eye(m) - S.T @ S, "fro")
    delta_tilde = np.linalg.norm(P - S @ R, "fro") / np.linalg.norm(P, "fro")
    return float(delta), float(delta_tilde)
