"""Philox4x32-10 counter-based generator, and the seeded sketch entries drawn from it.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper only asks that the sketching matrix come from "a seeded random
number generator" so that any block of Theta can be produced without storage
or communication (Sec. 2.1 on Rademacher/P-SRHT; Sec. 2.4 on distributed
architectures).  Philox4x32-10 is restated here from its published definition
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11): a 4x32-bit counter and a 2x32-bit key; each of ten rounds multiplies
counter words 0 and 2 by two fixed odd constants, keeps the 64-bit products'
high and low halves, XORs the high halves with the other two counter words and
the round key, and permutes; the key is bumped by two Weyl constants between
rounds.

Stream layout used by both the oracle and the GPU library (a reading of the
paper's "seeded generator"; the paper fixes none):

* key = (seed mod 2^32, seed div 2^32)
* Gaussian Theta entry (row l, column c):  counter (c, l >> 1, 0, 0);
  u1, u2 from words (x0,x1) and (x2,x3) as 53-bit midpoint uniforms;
  Box-Muller radius sqrt(-2 ln u1), angle 2*pi*u2; even rows take the cosine,
  odd rows the sine; the entry is divided by sqrt(k) so that E||Theta x||^2 =
  ||x||^2.
* SRHT sign of column c: bit (c mod 128) of the four words at counter
  (c >> 7, 0, 0, 1); a set bit means -1.
* SRHT row sample: key64(c) = x0 * 2^32 + x1 at counter (c, 0, 0, 2) for every
  c < s; the k indices with the smallest (key64, c) are kept, in ascending
  index order.  This is a uniform draw without replacement.
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

STREAM_GAUSS = 0
STREAM_SRHT_SIGN = 1
STREAM_SRHT_SAMPLE = 2


def philox4x32_10(ctr, key):
    """Apply Philox4x32-10 to counters ``ctr`` (shape (..., 4), uint32) under ``key`` (2 ints).

    Returns an array of the same shape holding the four output words.
    """
    c = np.asarray(ctr, dtype=np.uint64) & np.uint64(MASK32)
    c0, c1, c2, c3 = (c[..., j].copy() for j in range(4))
    k0 = np.uint64(int(key[0]) & MASK32)
    k1 = np.uint64(int(key[1]) & MASK32)
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    mask = np.uint64(MASK32)
    sh = np.uint64(32)
    for rnd in range(10):
        if rnd > 0:
            k0 = np.uint64((int(k0) + PHILOX_W0) & MASK32)
            k1 = np.uint64((int(k1) + PHILOX_W1) & MASK32)
        p0 = m0 * c0          # < 2^64, exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> sh, p0 & mask
        hi1, lo1 = p1 >> sh, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def _key(seed):
    seed = int(seed)
    return (seed & MASK32, (seed >> 32) & MASK32)


def _u53(hi, lo):
    """Midpoint 53-bit uniform in (0,1) from two 32-bit words."""
    v = ((hi.astype(np.uint64) << np.uint64(32)) | lo.astype(np.uint64)) >> np.uint64(11)
    return (v.astype(np.float64) + 0.5) * 2.0 ** -53


def gaussian_theta(k, n, seed, col0=0, ncols=None):
    """Columns [col0, col0+ncols) of the k x n Gaussian sketch with N(0, 1/k) entries (FP64)."""
    return gaussian_normals(k, n, seed, col0, ncols) / np.sqrt(k)


def gaussian_normals(k, n, seed, col0=0, ncols=None):
    """The N(0, 1) draws behind the Gaussian sketch: entry (l, c) from counter (c, l >> 1, 0, 0),
    Box-Muller (cosine for even l, sine for odd l)."""
    if ncols is None:
        ncols = n - col0
    cols = np.arange(col0, col0 + ncols, dtype=np.uint64)
    pairs = np.arange((k + 1) // 2, dtype=np.uint64)
    ctr = np.zeros((len(pairs), len(cols), 4), dtype=np.uint64)
    ctr[..., 0] = cols[None, :]
    ctr[..., 1] = pairs[:, None]
    ctr[..., 3] = STREAM_GAUSS
    x = philox4x32_10(ctr, _key(seed))
    u1 = _u53(x[..., 0], x[..., 1])
    u2 = _u53(x[..., 2], x[..., 3])
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    out = np.empty((2 * len(pairs), len(cols)))
    out[0::2] = rad * np.cos(ang)
    out[1::2] = rad * np.sin(ang)
    return out[:k]


def srht_signs(n, seed):
    """Rademacher diagonal D of the SRHT: array of +-1.0 of length n."""
    c = np.arange(n, dtype=np.uint64)
    blocks = np.arange((n + 127) // 128, dtype=np.uint64)
    ctr = np.zeros((len(blocks), 4), dtype=np.uint64)
    ctr[:, 0] = blocks
    ctr[:, 3] = STREAM_SRHT_SIGN
    x = philox4x32_10(ctr, _key(seed)).astype(np.uint64)
    word = x[(c >> np.uint64(7)).astype(np.int64), ((c & np.uint64(127)) >> np.uint64(5)).astype(np.int64)]
    bit = (word >> (c & np.uint64(31))) & np.uint64(1)
    return np.where(bit == 1, -1.0, 1.0)


def srht_sample(s, k, seed):
    """k distinct row indices of the s x s Hadamard matrix, uniform without replacement, ascending."""
    if not 0 < k <= s:
        raise ValueError("need 0 < k <= s")
    c = np.arange(s, dtype=np.uint64)
    ctr = np.zeros((s, 4), dtype=np.uint64)
    ctr[:, 0] = c
    ctr[:, 3] = STREAM_SRHT_SAMPLE
    x = philox4x32_10(ctr, _key(seed)).astype(np.uint64)
    key64 = (x[:, 0] << np.uint64(32)) | x[:, 1]
    order = np.lexsort((c, key64))       # primary key64, ties by index
    return np.sort(order[:k]).astype(np.int64)
