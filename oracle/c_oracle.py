"""ctypes front end of the plain-C oracle (``oracle/c/rgs_oracle.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  ``build()`` compiles
the C file with gcc into ``oracle/c/build/``; the arrays passed in and out are
NumPy FP64 / int32 arrays in column-major order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "c", "rgs_oracle.c")
_OUT = os.path.join(_HERE, "c", "build", "librgs_oracle.so")
_lib = None


def build(force=False):
    """Compile the C oracle: -O3, no architecture-specific flags, no contraction of a multiply and
    an add into a fused multiply-add (so x86 and Arm builds round alike), OpenMP over independent
    loops when the compiler has it (results do not depend on the thread count)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        base = ["gcc", "-O3", "-std=c99", "-ffp-contract=off", "-D_DEFAULT_SOURCE", "-fPIC", "-shared"]
        tmp = _OUT + ".tmp"
        try:
            subprocess.check_call(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + [_SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def set_threads(n):
    """Threads of the C oracle's parallel loops (0: the OpenMP default); returns the count in use."""
    return int(lib().orc_set_threads(int(n)))


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        P = ctypes.c_void_p
        L.orc_philox.argtypes = [P, P, P]
        L.orc_sketch_new.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64]
        L.orc_sketch_new.restype = P
        L.orc_sketch_free.argtypes = [P]
        L.orc_sketch_apply.argtypes = [P, P, P]
        L.orc_sketch_rows.argtypes = [P]
        L.orc_sketch_rows.restype = P
        L.orc_sketch_signs.argtypes = [P]
        L.orc_sketch_signs.restype = P
        L.orc_rgs_qr.argtypes = [P, ctypes.c_int64, ctypes.c_int, P, ctypes.c_int64, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, P, P, P, P, P, P]
        L.orc_rgmres.argtypes = [P, ctypes.c_int64, P, P, P, P, P, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, P, P]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_update_fp32.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, ctypes.c_int64, P, P]
        L.orc_cgs2_gmres.argtypes = [ctypes.c_int64, P, P, P, P, P, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def update_fp32(w, Qp, c):
    """Step 3 in FP32 (one rounding per fused multiply-add term), the C oracle's emulation."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    Qp = np.asfortranarray(Qp, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    n, ncols = Qp.shape
    out = np.empty(n)
    lib().orc_update_fp32(n, ncols, _p(w), _p(Qp), max(1, n), _p(c), _p(out))
    return out


KIND = {"gaussian": 0, "srht": 1}
LS = {"householder": 0, "richardson": 1}
STORAGE = {"f64": 0, "f32": 1, "bf16": 2}


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c), _p(k), _p(out))
    return out


class CSketch:
    """Theta built by the C oracle."""

    def __init__(self, kind, n, k, seed):
        self.kind, self.n, self.k, self.seed = kind, int(n), int(k), int(seed)
        self.h = lib().orc_sketch_new(KIND[kind], self.n, self.k, self.seed)
        if not self.h:
            raise ValueError("invalid sketch shape")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_sketch_free(self.h)
            self.h = None

    def rows(self):
        ptr = lib().orc_sketch_rows(self.h)
        return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_int64)), (self.k,)).copy()

    def signs(self):
        ptr = lib().orc_sketch_signs(self.h)
        return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_double)), (self.n,)).copy()

    def apply(self, X):
        X = np.asarray(X, dtype=np.float64)
        vec = X.ndim == 1
        Xc = np.asfortranarray(X[:, None] if vec else X)
        Y = np.zeros((self.k, Xc.shape[1]), order="F")
        for c in range(Xc.shape[1]):
            col = np.ascontiguousarray(Xc[:, c])
            out = np.zeros(self.k)
            lib().orc_sketch_apply(self.h, _p(col), _p(out))
            Y[:, c] = out
        return Y[:, 0] if vec else Y


class CQR:
    pass


def rgs_qr(W, sketch, ls="householder", sweeps=2, storage="f64"):
    """Alg. 2 through the C oracle; W is an (n, m) array."""
    W = np.asfortranarray(W, dtype=np.float64)
    n, m = W.shape
    k = sketch.k
    Qp = np.zeros((n, m), order="F")
    sigma = np.zeros(m)
    R = np.zeros((m, m), order="F")
    S = np.zeros((k, m), order="F")
    P = np.zeros((k, m), order="F")
    certs = np.zeros(2)
    st = lib().orc_rgs_qr(sketch.h, n, m, _p(W), n, LS[ls], sweeps, STORAGE[storage],
                          _p(Qp), _p(sigma), _p(R), _p(S), _p(P), _p(certs))
    if st != 0:
        raise RuntimeError(f"C oracle rgs_qr status {st}")
    out = CQR()
    out.Qp, out.sigma, out.R, out.S, out.P = Qp, sigma, R, S, P
    out.Q = Qp * sigma[None, :]
    out.delta, out.delta_tilde = float(certs[0]), float(certs[1])
    return out


class CSolve:
    pass


def rgmres(csr, b, sketch, restart, tol=1e-8, max_cycles=50, x0=None, ls="householder", sweeps=2,
           storage="f64", fixed_steps=False, inner_factor=0.5):
    """Restarted RGS-GMRES through the C oracle; csr = (rowptr, colind, val) int32/int32/FP64."""
    rowptr, colind, val = (np.ascontiguousarray(a) for a in csr)
    assert rowptr.dtype == np.int32 and colind.dtype == np.int32 and val.dtype == np.float64
    n = len(rowptr) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    info = np.zeros(2, dtype=np.int32)
    hist = np.zeros(max_cycles + 1)
    st = lib().orc_rgmres(sketch.h, n, _p(rowptr), _p(colind), _p(val), _p(b), _p(x), restart, tol,
                          max_cycles, LS[ls], sweeps, STORAGE[storage], int(fixed_steps), inner_factor,
                          _p(info), _p(hist))
    out = CSolve()
    out.x, out.converged, out.cycles, out.steps = x, st == 0, int(info[0]), int(info[1])
    out.true_residuals = hist[: out.cycles + 1].copy()
    return out


def cgs2_gmres(csr, b, restart, tol=1e-8, max_cycles=50, x0=None, fixed_steps=False, inner_factor=0.5):
    rowptr, colind, val = (np.ascontiguousarray(a) for a in csr)
    n = len(rowptr) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    info = np.zeros(2, dtype=np.int32)
    hist = np.zeros(max_cycles + 1)
    st = lib().orc_cgs2_gmres(n, _p(rowptr), _p(colind), _p(val), _p(b), _p(x), restart, tol,
                              max_cycles, int(fixed_steps), inner_factor, _p(info), _p(hist))
    out = CSolve()
    out.x, out.converged, out.cycles, out.steps = x, st == 0, int(info[0]), int(info[1])
    out.true_residuals = hist[: out.cycles + 1].copy()
    return out
