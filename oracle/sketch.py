"""Sketching matrices Theta (k x n) of the paper, applied on the CPU in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.1 defines the two families used here:

* Gaussian (the paper's experiments note no difference from Rademacher, Sec. 5):
  i.i.d. N(0, 1/k) entries; "gaussian_bf16" is the same draws rounded to bfloat16 before
  the 1/sqrt(k) scale (the sketch of the batched solver);
* (P-)SRHT: for s the power of two with n <= s < 2n, Theta is the first n
  columns of (1/sqrt(k)) * P * H_s * D, with D a diagonal of random signs, H_s
  the (unnormalised, +-1) Walsh-Hadamard matrix of order s and P a uniform
  sub-sample of k of its s rows.

The Walsh-Hadamard transform is written out as the textbook in-place butterfly
(log2 s stages of (a, b) -> (a + b, a - b)), natural (Sylvester) ordering,
H_s[a, b] = (-1)^popcount(a & b).
"""
from __future__ import annotations

import numpy as np

from . import philox


def next_pow2(n):
    s = 1
    while s < n:
        s *= 2
    return s


def fwht(x, dtype=np.float64):
    """Unnormalised Walsh-Hadamard transform along axis 0 (length must be a power of two), every
    butterfly computed in ``dtype``."""
    y = np.array(x, dtype=dtype, copy=True)
    s = y.shape[0]
    if s & (s - 1):
        raise ValueError("length must be a power of two")
    h = 1
    while h < s:
        y = y.reshape((s // (2 * h), 2, h) + y.shape[1:])
        a = y[:, 0].copy()
        b = y[:, 1].copy()
        y[:, 0] = a + b
        y[:, 1] = a - b
        y = y.reshape((s,) + y.shape[3:])
        h *= 2
    return y


class Sketch:
    """A seeded sketching matrix Theta; ``apply(X)`` returns Theta @ X in FP64."""

    def __init__(self, kind, n, k, seed):
        if kind not in ("gaussian", "gaussian_bf16", "srht"):
            raise ValueError(kind)
        self.kind, self.n, self.k, self.seed = kind, int(n), int(k), int(seed)
        if kind == "gaussian":
            self._theta = philox.gaussian_theta(self.k, self.n, self.seed)
        elif kind == "gaussian_bf16":
            from .rgs import round_bf16
            self._theta = round_bf16(philox.gaussian_normals(self.k, self.n, self.seed)) / np.sqrt(self.k)
        else:
            self.s = next_pow2(self.n)
            if self.k > self.s:
                raise ValueError("SRHT needs k <= s")
            self.signs = philox.srht_signs(self.n, self.seed)
            self.rows = philox.srht_sample(self.s, self.k, self.seed)

    def apply(self, X):
        X = np.asarray(X, dtype=np.float64)
        vec = X.ndim == 1
        if vec:
            X = X[:, None]
        if X.shape[0] != self.n:
            raise ValueError("row count mismatch")
        if self.kind in ("gaussian", "gaussian_bf16"):
            Y = self._theta @ X
        else:
            Z = np.zeros((self.s, X.shape[1]))
            Z[: self.n] = self.signs[:, None] * X
            Y = fwht(Z)[self.rows] / np.sqrt(self.k)
        return Y[:, 0] if vec else Y

    def apply_f32(self, X):
        """Theta @ X with every operation in FP32 (the unique-precision setting of Sec. 5.1): X
        rounded to FP32, Theta's Gaussian entries rounded to FP32 and an FP32 product, or the
        SRHT's signs, FP32 butterflies and an FP32 1/sqrt(k) scale.  Returned as FP64."""
        X = np.asarray(X, dtype=np.float64)
        vec = X.ndim == 1
        if vec:
            X = X[:, None]
        if X.shape[0] != self.n:
            raise ValueError("row count mismatch")
        X32 = X.astype(np.float32)
        if self.kind in ("gaussian", "gaussian_bf16"):
            Y = self._theta.astype(np.float32) @ X32
        else:
            Z = np.zeros((self.s, X.shape[1]), dtype=np.float32)
            Z[: self.n] = self.signs.astype(np.float32)[:, None] * X32
            Y = fwht(Z, np.float32)[self.rows] * np.float32(1.0 / np.sqrt(self.k))
        Y = Y.astype(np.float64)
        return Y[:, 0] if vec else Y

    def dense(self):
        """Theta as an explicit k x n FP64 matrix (small n only)."""
        return self.apply(np.eye(self.n))
