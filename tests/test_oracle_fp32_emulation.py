"""Pin of the oracle's FP32 step-3 emulation against exact rational arithmetic (CPU only).

Step 3 of Alg. 2 runs in the working precision u_crs (Sec. 2.3); for an FP32 basis that is a
chain of FP32 fused multiply-adds acc <- acc - c_j q'_j.  Each of them rounds the exact value
acc - c_j q'_j once to FP32 (round to nearest, ties to even).  The reference here computes that
exact value as a ``fractions.Fraction`` and picks the nearest FP32 number by comparing exact
distances to the neighbours, so it shares nothing with the TwoSum construction of the oracles.
The constructed near-tie cases are ones where rounding first to FP64 and then to FP32 lands on
an FP32 midpoint and resolves it the wrong way, so a double-rounding emulation fails them.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import c_oracle, rgs

F32 = np.float32


def round_f32_exact(x: Fraction) -> float:
    """Nearest FP32 number to the rational x, ties to even (mantissa's last bit 0)."""
    d = np.float32(float(x))          # float(Fraction) is correctly rounded to FP64
    cands = {float(np.nextafter(d, F32(-np.inf))), float(d), float(np.nextafter(d, F32(np.inf)))}
    best = None
    for c in sorted(cands):
        dist = abs(Fraction(c) - x)
        even = (int(np.array(c, dtype=np.float32).view(np.uint32)) & 1) == 0
        key = (dist, not even)
        if best is None or key < best[0]:
            best = (key, c)
    return best[1]


def exact_fma32(acc, c, q):
    return round_f32_exact(Fraction(float(acc)) - Fraction(float(c)) * Fraction(float(q)))


def double_rounded(acc, c, q):
    """The emulation that rounds to FP64 first: what a wrong oracle would compute."""
    return float(F32(float(acc) - float(c) * float(q)))


def _random_triples(n, seed):
    g = np.random.default_rng(seed)
    acc = (g.standard_normal(n) * np.exp2(g.integers(-20, 20, n))).astype(np.float32)
    c = (g.standard_normal(n) * np.exp2(g.integers(-30, 10, n))).astype(np.float32)
    q = (g.standard_normal(n) * np.exp2(g.integers(-30, 10, n))).astype(np.float32)
    return acc.astype(np.float64), c.astype(np.float64), q.astype(np.float64)


def _near_ties(n, seed):
    """acc - c q = (a midpoint between acc and an FP32 neighbour) +- a tiny amount, where the
    tiny amount (h a^2 2^-46 for h half an FP32 ulp of acc) is below half an FP64 ulp."""
    g = np.random.default_rng(seed)
    accs, cs, qs = [], [], []
    for t in range(n):
        acc = F32(g.standard_normal() * 2.0 ** int(g.integers(-10, 10)))
        if acc == 0:
            continue
        e = np.frexp(np.float64(acc))[1]          # |acc| in [2^(e-1), 2^e)
        h = 2.0 ** (e - 1 - 24)                   # half an FP32 ulp of acc
        a = int(g.integers(1, 64))
        c = F32(1.0 + a * 2.0 ** -23)             # c q = h (1 - a^2 2^-46)
        q = F32(h * (1.0 - 2 * a * 2.0 ** -24))
        sign = 1.0 if (t % 2 == 0) else -1.0      # toward zero or away from zero
        accs.append(float(acc))
        cs.append(float(c) * sign * np.sign(float(acc)))
        qs.append(float(q))
    # exact ties: c q equal to half an ulp of acc
    for t in range(32):
        acc = F32((1.0 + int(g.integers(0, 1 << 23)) * 2.0 ** -23) * 2.0 ** int(g.integers(-5, 5)))
        e = np.frexp(np.float64(acc))[1]
        accs.append(float(acc))
        cs.append(1.0 if t % 2 else -1.0)
        qs.append(2.0 ** (e - 1 - 24))
    return np.array(accs), np.array(cs), np.array(qs)


@pytest.mark.parametrize("which", ["numpy", "c"])
def test_fma32_matches_exact_rounding(which):
    acc, c, q = _random_triples(3000, 1)
    a2, c2, q2 = _near_ties(500, 2)
    acc, c, q = np.concatenate([acc, a2]), np.concatenate([c, c2]), np.concatenate([q, q2])
    want = np.array([exact_fma32(a, b, d) for a, b, d in zip(acc, c, q)])
    if which == "numpy":
        got = rgs.fma32(acc, c, q)
    else:
        got = np.array([c_oracle.update_fp32(np.array([a]), np.array([[d]]), np.array([b]))[0]
                        for a, b, d in zip(acc, c, q)])
    assert np.array_equal(got, want)


def test_near_tie_cases_catch_double_rounding():
    """The constructed cases are discriminating: rounding through FP64 gets many of them wrong."""
    acc, c, q = _near_ties(500, 2)
    want = np.array([exact_fma32(a, b, d) for a, b, d in zip(acc, c, q)])
    naive = np.array([double_rounded(a, b, d) for a, b, d in zip(acc, c, q)])
    assert np.count_nonzero(naive != want) > 100


@pytest.mark.parametrize("which", ["numpy", "c"])
def test_update_chain_matches_exact_chain(which):
    """Step 3 over several columns: fl32(w), then one exactly rounded multiply-add per column,
    with c_j rounded to FP32 first."""
    g = np.random.default_rng(3)
    n, ncols = 40, 25
    w = g.standard_normal(n)
    Qp = g.standard_normal((n, ncols)).astype(np.float32).astype(np.float64) * np.exp2(g.integers(-12, 4, ncols))
    cc = g.standard_normal(ncols) * np.exp2(g.integers(-12, 4, ncols))
    want = np.empty(n)
    for r in range(n):
        acc = float(F32(w[r]))
        for j in range(ncols):
            acc = exact_fma32(acc, float(F32(cc[j])), Qp[r, j])
        want[r] = acc
    got = rgs.update_fp32(w, Qp, cc) if which == "numpy" else c_oracle.update_fp32(w, Qp, cc)
    assert np.array_equal(got, want)
