"""Python binding of librgs: randomized Gram-Schmidt and RGS-GMRES on the GPU.

Argument marshalling only: every computation runs in the CUDA kernels of
``lib/librgs.so`` (built from ``csrc/`` by ``build.py``).  If the library is
missing, importing a function raises immediately; there is no fallback.

Matrices are torch tensors in column-major layout: an n x m matrix is a tensor
of shape (n, m) with stride (1, ld), e.g. ``torch.empty(m, n).T``.  Functions
keep the names of the C entry points in ``include/librgs.h``.
"""
from __future__ import annotations

import atexit
import ctypes
import os

import torch

_exiting = False


def _at_exit():
    # the CUDA runtime may already be torn down when finalizers run at interpreter exit:
    # leave the process's device memory to the driver instead of calling into the library
    global _exiting
    _exiting = True


atexit.register(_at_exit)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "librgs.so")

RGS_OK = 0
RGS_ERR_INVALID_ARG = 1
RGS_ERR_CUDA = 2
RGS_ERR_ALLOC = 3
RGS_ERR_BREAKDOWN = 4
RGS_ERR_NOT_CONVERGED = 5
RGS_ERR_TIMEOUT = 6
RGS_ERR_NONFINITE = 7
RGS_ERR_NOT_IMPLEMENTED = 8
RGS_ERR_CERT_FAILED = 9
RGS_ERR_CALLBACK = 10

RGS_F64, RGS_F32, RGS_BF16 = 0, 1, 2
RGS_SKETCH_GAUSSIAN, RGS_SKETCH_SRHT = 0, 1
RGS_QR_NO_CERTIFICATES = 1
RGS_QR_TIMINGS = 2
RGS_FP64_FINE = 4               # FP64 transform sums, products and least squares for every storage
RGS_FP64_LS = 8                 # FP64 least squares (and Givens); double-float transform sums
RGS_FP32_FINE = 16              # rgs_qr: unique precision, FP32 transform sums and least squares
RGS_LS_RICHARDSON = 32          # rgs_qr: step 2 by two Richardson sweeps on the normal equations
RGS_QR_FP64_FINE = RGS_FP64_FINE
RGS_QR_FP64_SKETCH = RGS_FP64_FINE
RGS_PRECOND_NONE, RGS_PRECOND_JACOBI, RGS_PRECOND_LEARNED_CONV, RGS_PRECOND_CALLBACK = 0, 1, 2, 3

_DTYPE = {torch.float64: RGS_F64, torch.float32: RGS_F32, torch.bfloat16: RGS_BF16}
_KIND = {"gaussian": RGS_SKETCH_GAUSSIAN, "srht": RGS_SKETCH_SRHT}

EXPORTED = ["rgs_create", "rgs_destroy", "rgs_set_stream", "rgs_set_wait_budget", "rgs_status_string",
            "rgs_last_error",
            "rgs_sketch_create", "rgs_sketch_destroy", "rgs_sketch_apply", "rgs_sketch_apply_noalloc", "rgs_qr",
            "rgs_arnoldi_create", "rgs_arnoldi_destroy", "rgs_arnoldi_start", "rgs_arnoldi_step",
            "rgs_arnoldi_get", "rgs_arnoldi_basis", "rgs_csr_matvec", "rgmres_solve", "cgs2_gmres_solve",
            "rgmres_set_preconditioner", "rgs_convnet_num_params", "rgs_convnet_create", "rgs_convnet_destroy",
            "rgs_convnet_get_params", "rgs_convnet_set_params", "rgs_convnet_forward", "rgs_convnet_loss_grad",
            "rgs_convnet_train_step", "rgmres_solve_batched", "rgs_get_tuning", "rgs_set_tuning",
            "rgs_autotune_update", "rgs_autotune_batched", "rgs_certify_embedding", "rgs_csr_residual",
            "rgs_convnet_input", "rgs_csr_to_stencil"]


class RgsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"librgs status {status}: {msg}")
        self.status = status


class QRInfo(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("delta_tilde", ctypes.c_double),
                ("breakdown_col", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("sketch_ms", ctypes.c_double), ("update_ms", ctypes.c_double), ("ls_ms", ctypes.c_double)]


class CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colind", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class GmresOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("max_cycles", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("inner_factor", ctypes.c_double), ("qtype", ctypes.c_int32), ("fixed_steps", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class GmresInfo(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int32), ("total_steps", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("status", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("fallback_cycle", ctypes.c_int32),
                ("sell", ctypes.c_int32), ("sketch_refreshes", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int32), ("k", ctypes.c_int32), ("max_cycles", ctypes.c_int32),
                ("qtype", ctypes.c_int32), ("rtol", ctypes.c_double), ("inner_factor", ctypes.c_double),
                ("fixed_steps", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("upd_blocks_per_sm", ctypes.c_int32), ("batch_blocks_per_sm", ctypes.c_int32),
                ("batch_min_team_work", ctypes.c_double), ("ls_blocks", ctypes.c_int32),
                ("batch_rows_per_thread", ctypes.c_int32)]


class LearnedPrecond(ctypes.Structure):
    _fields_ = [("net", ctypes.c_void_p), ("logkappa", ctypes.c_void_p)]


# int32_t apply(void* user, int64_t n, const void* v, int32_t vtype, void* z, int32_t ztype, void* stream)
PrecondApplyFn = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32,
                                  ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p)


class CallbackPrecond(ctypes.Structure):
    _fields_ = [("apply", PrecondApplyFn), ("user", ctypes.c_void_p), ("nonlinear", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None


def load():
    """Load librgs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2011_05090_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "rgs_create": [ctypes.POINTER(P), P],
        "rgs_destroy": [P],
        "rgs_set_stream": [P, P],
        "rgs_set_wait_budget": [P, I64],
        "rgs_certify_embedding": [P, P, P, I64, I32, P, ctypes.c_int, I64, P, P, I64, D, P],
        "rgs_csr_residual": [P, ctypes.POINTER(CSR), P, P, P, P],
        "rgs_convnet_input": [P, I64, P, P, P],
        "rgs_csr_to_stencil": [P, ctypes.POINTER(CSR), I32, I32, P],
        "rgs_status_string": [ctypes.c_int],
        "rgs_last_error": [P],
        "rgs_sketch_create": [P, ctypes.c_int, I64, I32, ctypes.c_uint64, ctypes.POINTER(P)],
        "rgs_sketch_destroy": [P],
        "rgs_sketch_apply": [P, P, I32, P, I64, P, I64],
        "rgs_sketch_apply_noalloc": [P, P, I32, P, I64, P, I64],
        "rgs_qr": [P, P, I64, I32, P, I64, P, ctypes.c_int, I64, P, P, I64, P, I64, I32, ctypes.POINTER(QRInfo)],
        "rgs_arnoldi_create": [P, P, I64, I32, ctypes.c_int, I32, ctypes.POINTER(P)],
        "rgs_arnoldi_destroy": [P],
        "rgs_arnoldi_start": [P, P, P],
        "rgs_arnoldi_step": [P, P, ctypes.POINTER(CSR), P],
        "rgs_arnoldi_get": [P, P, ctypes.POINTER(I32), P, I64, P],
        "rgs_arnoldi_basis": [P, ctypes.POINTER(P), ctypes.POINTER(I64)],
        "rgs_csr_matvec": [P, ctypes.POINTER(CSR), P, P],
        "rgmres_solve": [P, P, ctypes.POINTER(CSR), P, P, ctypes.POINTER(GmresOpts), ctypes.POINTER(GmresInfo)],
        "cgs2_gmres_solve": [P, ctypes.POINTER(CSR), P, P, ctypes.POINTER(GmresOpts), ctypes.POINTER(GmresInfo)],
        "rgmres_set_preconditioner": [P, ctypes.c_int, P, I32],
        "rgmres_solve_batched": [P, I32, ctypes.POINTER(CSR), ctypes.POINTER(P), ctypes.POINTER(P),
                                 ctypes.POINTER(BatchOpts), ctypes.c_uint64, ctypes.POINTER(GmresInfo)],
        "rgs_get_tuning": [P, ctypes.POINTER(Tuning)],
        "rgs_set_tuning": [P, ctypes.POINTER(Tuning)],
        "rgs_autotune_update": [P, P, I32, ctypes.c_int, ctypes.POINTER(Tuning), P],
        "rgs_autotune_batched": [P, I32, ctypes.POINTER(CSR), ctypes.POINTER(P), ctypes.POINTER(BatchOpts),
                                 ctypes.c_uint64, I32, ctypes.POINTER(Tuning), P],
        "rgs_convnet_num_params": [],
        "rgs_convnet_create": [P, I32, I32, I32, ctypes.c_uint64, ctypes.POINTER(P)],
        "rgs_convnet_destroy": [P],
        "rgs_convnet_get_params": [P, P, P, I64],
        "rgs_convnet_set_params": [P, P, P, I64],
        "rgs_convnet_forward": [P, P, I32, P, P],
        "rgs_convnet_loss_grad": [P, P, I32, P, P, P, ctypes.POINTER(D), P],
        "rgs_convnet_train_step": [P, P, I32, P, P, P, ctypes.c_float, ctypes.POINTER(D)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name in ("rgs_status_string", "rgs_last_error") else ctypes.c_int
    L.rgs_convnet_num_params.restype = I64
    _lib = L
    return L


def _check(status, handle=None):
    if status != RGS_OK:
        L = load()
        msg = L.rgs_status_string(status).decode()
        if handle is not None and handle.ptr:
            detail = L.rgs_last_error(handle.ptr).decode()
            if detail:
                msg += f" ({detail})"
        raise RgsError(status, msg)


def _colmajor(t, rows=None, cols=None):
    """(pointer, ld) of a column-major 2-D tensor of shape (rows, cols)."""
    if t.dim() == 1:
        t = t[:, None]
    if rows is not None and t.shape[0] != rows or cols is not None and t.shape[1] != cols:
        raise ValueError(f"shape {tuple(t.shape)} != ({rows}, {cols})")
    if t.stride(0) != 1 and t.shape[0] > 1:
        raise ValueError("matrix must be column-major (stride(0) == 1)")
    ld = t.stride(1) if t.shape[1] > 1 else max(t.shape[0], 1)
    return t.data_ptr(), ld


def colmajor_empty(rows, cols, dtype=torch.float64, device="cuda", pin=False):
    """An uninitialised column-major (rows x cols) tensor."""
    if pin:
        return torch.empty(cols, rows, dtype=dtype, pin_memory=True).T
    return torch.empty(cols, rows, dtype=dtype, device=device).T


class Handle:
    def __init__(self, ptr, device=0):
        self.ptr = ptr
        self.device = device

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None and not _exiting:
            _lib.rgs_destroy(self.ptr)
            self.ptr = None


class Sketch:
    def __init__(self, ptr, handle, kind, n, k, seed):
        self.ptr, self.handle, self.kind, self.n, self.k, self.seed = ptr, handle, kind, n, k, seed

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None and not _exiting:
            _lib.rgs_sketch_destroy(self.ptr)
            self.ptr = None


def rgs_create(stream=None):
    """Handle bound to ``stream`` (default: torch's current CUDA stream)."""
    L = load()
    if stream is None:
        stream = torch.cuda.current_stream()
    out = ctypes.c_void_p()
    _check(L.rgs_create(ctypes.byref(out), ctypes.c_void_p(stream.cuda_stream)))
    return Handle(out.value, torch.cuda.current_device())


def rgs_set_wait_budget(h, cycles):
    """Clock-cycle budget of every device-side wait (0: the default, about two seconds)."""
    _check(load().rgs_set_wait_budget(h.ptr, int(cycles)), h)


def rgs_set_stream(h, stream):
    _check(load().rgs_set_stream(h.ptr, ctypes.c_void_p(stream.cuda_stream)), h)


def rgs_sketch_create(h, kind, n, k, seed):
    out = ctypes.c_void_p()
    _check(load().rgs_sketch_create(h.ptr, _KIND[kind], int(n), int(k), int(seed), ctypes.byref(out)), h)
    return Sketch(out.value, h, kind, int(n), int(k), int(seed))


def _sketch_operands(h, X, Y):
    """X and Y of a sketch application: FP64 CUDA tensors on the handle's device."""
    for name, t in (("X", X), ("Y", Y)):
        if t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64, got {t.dtype}")
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != h.device:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the handle on cuda:{h.device}")


def rgs_sketch_apply(h, sk, X, Y=None):
    """Y (k x ncols) = Theta X for a column-major FP64 X (n x ncols) on the GPU."""
    if X.dim() == 1:
        X = X[:, None]
    ncols = X.shape[1]
    if Y is None:
        Y = colmajor_empty(sk.k, ncols, device=X.device)
    _sketch_operands(h, X, Y)
    px, ldx = _colmajor(X, sk.n, ncols)
    py, ldy = _colmajor(Y, sk.k, ncols)
    _check(load().rgs_sketch_apply(h.ptr, sk.ptr, ncols, px, ldx, py, ldy), h)
    return Y


def rgs_sketch_apply_noalloc(h, sk, X, Y):
    """Y (k x ncols) = Theta X like rgs_sketch_apply, with no device allocation during the call
    (the partial sketches use the library's fixed scratch array; see include/librgs.h)."""
    if X.dim() == 1:
        X = X[:, None]
    ncols = X.shape[1]
    _sketch_operands(h, X, Y)
    px, ldx = _colmajor(X, sk.n, ncols)
    py, ldy = _colmajor(Y, sk.k, ncols)
    _check(load().rgs_sketch_apply_noalloc(h.ptr, sk.ptr, ncols, px, ldx, py, ldy), h)
    return Y


RGS_NOALLOC_SCRATCH_BYTES = 8 << 20


def rgs_certify_embedding(h, theta, phi, V, eps_star=0.05, vscale=None, VTheta=None):
    """Sec. 3.2's certificate omega_bar for range(V diag(vscale)) (V: n x m CUDA tensor, FP64 / FP32 /
    BF16, column-major; VTheta: optional Theta V, k x m FP64).  Returns a dict with omega_bar,
    s_min, s_max and certified (omega_bar < 1)."""
    n, m = V.shape
    pv, ldv = _colmajor(V, n, m)
    for name, t in (("vscale", vscale), ("VTheta", VTheta)):
        if t is not None and (t.dtype != torch.float64 or not t.is_cuda):
            raise ValueError(f"{name} must be a float64 CUDA tensor")
    pt, ldt = (_colmajor(VTheta, theta.k, m) if VTheta is not None else (None, theta.k))
    out = (ctypes.c_double * 3)()
    st = load().rgs_certify_embedding(h.ptr, theta.ptr, phi.ptr, int(n), int(m), pv, _DTYPE[V.dtype], ldv,
                                      vscale.data_ptr() if vscale is not None else None, pt, ldt, float(eps_star),
                                      out)
    if st not in (RGS_OK, RGS_ERR_CERT_FAILED):
        _check(st, h)
    return {"omega_bar": out[0], "s_min": out[1], "s_max": out[2], "certified": st == RGS_OK}


def rgs_qr(h, sk, W, Q, R, qscale=None, S=None, flags=0):
    """Alg. 2 on W (n x m, FP64).  Fills Q (n x m, FP64/FP32/BF16), R (m x m) and optionally
    qscale (m) and S (k x m); returns the step-8 certificates as a dict."""
    n, m = W.shape
    pw, ldw = _colmajor(W, n, m)
    pq, ldq = _colmajor(Q, n, m)
    pr, ldr = _colmajor(R, m, m)
    ps, lds = (_colmajor(S, sk.k, m) if S is not None else (None, sk.k))
    info = QRInfo()
    st = load().rgs_qr(h.ptr, sk.ptr, n, m, pw, ldw, pq, _DTYPE[Q.dtype], ldq,
                       qscale.data_ptr() if qscale is not None else None, pr, ldr, ps, lds, flags,
                       ctypes.byref(info))
    res = {"delta": info.delta, "delta_tilde": info.delta_tilde, "breakdown_col": info.breakdown_col,
           "launches": info.launches, "sketch_ms": info.sketch_ms, "update_ms": info.update_ms,
           "ls_ms": info.ls_ms}
    if st != RGS_OK:
        try:
            _check(st, h)
        except RgsError as e:
            e.info = res
            raise
    return res


def csr_struct(rowptr, colind, val):
    n = rowptr.numel() - 1
    return CSR(n, colind.numel(), rowptr.data_ptr(), colind.data_ptr(), val.data_ptr())


class Arnoldi:
    def __init__(self, ptr, handle, sketch, n, mmax, qdtype):
        self.ptr, self.handle, self.sketch, self.n, self.mmax, self.qdtype = ptr, handle, sketch, n, mmax, qdtype

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None and not _exiting:
            _lib.rgs_arnoldi_destroy(self.ptr)
            self.ptr = None


class _DeviceArray:
    """__cuda_array_interface__ wrapper so torch can view library-owned device memory."""

    def __init__(self, ptr, shape, strides, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "strides": strides, "typestr": typestr,
                                         "data": (ptr, False), "version": 2}


def _fine_flags(fine64, ls64):
    return (RGS_FP64_FINE if fine64 else 0) | (RGS_FP64_LS if ls64 else 0)


def rgs_arnoldi_create(h, sk, n, mmax, qdtype=torch.float64, fine64=False, ls64=False):
    """RGS-Arnoldi object; for FP32 / BF16 bases ls64 selects FP64 least squares (RGS_FP64_LS) and
    fine64 all-FP64 fine arithmetic (RGS_FP64_FINE)."""
    out = ctypes.c_void_p()
    _check(load().rgs_arnoldi_create(h.ptr, sk.ptr, int(n), int(mmax), _DTYPE[qdtype], _fine_flags(fine64, ls64),
                                     ctypes.byref(out)), h)
    return Arnoldi(out.value, h, sk, int(n), int(mmax), qdtype)


def rgs_arnoldi_start(h, a, w1):
    _check(load().rgs_arnoldi_start(h.ptr, a.ptr, w1.data_ptr()), h)


def rgs_arnoldi_step(h, a, csr=None, w=None):
    A = ctypes.byref(csr) if csr is not None else None
    _check(load().rgs_arnoldi_step(h.ptr, a.ptr, A, w.data_ptr() if w is not None else None), h)


def rgs_arnoldi_get(h, a):
    """(ncols, R (ncols x ncols, numpy), qscale (ncols, numpy)) copied to the host."""
    import numpy as np
    nc = ctypes.c_int32()
    _check(load().rgs_arnoldi_get(h.ptr, a.ptr, ctypes.byref(nc), None, 0, None), h)
    m = nc.value
    R = np.zeros((m, m), order="F")
    qs = np.zeros(m)
    if m:
        _check(load().rgs_arnoldi_get(h.ptr, a.ptr, ctypes.byref(nc), R.ctypes.data_as(ctypes.c_void_p), m,
                                      qs.ctypes.data_as(ctypes.c_void_p)), h)
    return m, R, qs


def rgs_arnoldi_basis(a, ncols=None):
    """The stored basis Q' (n x ncols, column-major, in the object's dtype) as a torch view."""
    q = ctypes.c_void_p()
    ld = ctypes.c_int64()
    _check(load().rgs_arnoldi_basis(a.ptr, ctypes.byref(q), ctypes.byref(ld)))
    ncols = a.mmax if ncols is None else ncols
    esz = {torch.float64: 8, torch.float32: 4, torch.bfloat16: 2}[a.qdtype]
    typestr = {torch.float64: "<f8", torch.float32: "<f4", torch.bfloat16: "<V2"}[a.qdtype]
    arr = _DeviceArray(q.value, (ncols, a.n), (ld.value * esz, esz), typestr)
    if a.qdtype == torch.bfloat16:
        raw = torch.as_tensor(_DeviceArray(q.value, (ncols, a.n), (ld.value * 2, 2), "<i2"), device="cuda")
        return raw.view(torch.bfloat16).T
    return torch.as_tensor(arr, device="cuda").T


def _gmres_opts(restart, max_cycles, rtol, inner_factor, qdtype, fixed_steps, fine64=False, ls64=False):
    return GmresOpts(int(restart), int(max_cycles), float(rtol), float(inner_factor), _DTYPE[qdtype],
                     1 if fixed_steps else 0, _fine_flags(fine64, ls64))


def _gmres_result(st, info, hist, h):
    res = {"cycles": info.cycles, "total_steps": info.total_steps, "converged": bool(info.converged),
           "status": info.status, "rel_residual": info.rel_residual,
           "history": [hist[i] for i in range(info.cycles + 1)], "fallback_cycle": info.fallback_cycle,
           "sell": bool(info.sell), "sketch_refreshes": info.sketch_refreshes}
    if st not in (RGS_OK, RGS_ERR_NOT_CONVERGED):
        errors = getattr(h, "_precond_errors", None)
        cause = errors[0] if st == RGS_ERR_CALLBACK and errors else None
        if errors:
            errors.clear()
        try:
            _check(st, h)
        except RgsError as e:
            e.info = res
            raise e from cause
    return res


def rgmres_solve(h, sk, csr, b, x, restart, rtol=1e-8, max_cycles=100, inner_factor=0.5,
                 qdtype=torch.float32, fixed_steps=False, fine64=False, ls64=False):
    """Restarted randomized GMRES; x (FP64, CUDA) holds x0 and receives the solution.  For FP32 /
    BF16 bases, ls64: FP64 least squares and Givens; fine64: also FP64 sketch sums and products."""
    opts = _gmres_opts(restart, max_cycles, rtol, inner_factor, qdtype, fixed_steps, fine64, ls64)
    hist = (ctypes.c_double * (max_cycles + 2))()
    info = GmresInfo()
    info.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    st = load().rgmres_solve(h.ptr, sk.ptr, ctypes.byref(csr), b.data_ptr(), x.data_ptr(), ctypes.byref(opts),
                             ctypes.byref(info))
    return _gmres_result(st, info, hist, h)


def cgs2_gmres_solve(h, csr, b, x, restart, rtol=1e-8, max_cycles=100, inner_factor=0.5, fixed_steps=False):
    """Restarted FP64 GMRES with a CGS2 Arnoldi basis (the comparator)."""
    opts = _gmres_opts(restart, max_cycles, rtol, inner_factor, torch.float64, fixed_steps)
    hist = (ctypes.c_double * (max_cycles + 2))()
    info = GmresInfo()
    info.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    st = load().cgs2_gmres_solve(h.ptr, ctypes.byref(csr), b.data_ptr(), x.data_ptr(), ctypes.byref(opts),
                                 ctypes.byref(info))
    return _gmres_result(st, info, hist, h)


def rgs_csr_residual(h, csr, x, b, r=None):
    """r = b - A x (FP64 CUDA vectors); returns (r, ||r||)."""
    if r is None:
        r = torch.empty_like(b)
    nrm = ctypes.c_double()
    _check(load().rgs_csr_residual(h.ptr, ctypes.byref(csr), x.data_ptr(), b.data_ptr(), r.data_ptr(),
                                   ctypes.byref(nrm)), h)
    return r, nrm.value


def rgs_convnet_input(h, r, logkappa, out=None):
    """The network input (2, n) FP32 for one grid: r / rms(r) and log kappa (FP64 CUDA vectors)."""
    n = r.numel()
    if r.dtype != torch.float64 or logkappa.dtype != torch.float64 or not r.is_cuda or not logkappa.is_cuda:
        raise ValueError("r and logkappa must be float64 CUDA tensors")
    if logkappa.numel() != n:
        raise ValueError("r and logkappa differ in size")
    if out is None:
        out = torch.empty(2, n, dtype=torch.float32, device=r.device)
    if out.dtype != torch.float32 or not out.is_contiguous() or out.numel() != 2 * n:
        raise ValueError("out must be a contiguous float32 tensor of 2 n entries")
    _check(load().rgs_convnet_input(h.ptr, n, r.contiguous().data_ptr(), logkappa.contiguous().data_ptr(),
                                    out.data_ptr()), h)
    return out


def rgs_csr_to_stencil(h, csr, H, W):
    """(5, H, W) FP32 coefficients of a 5-point operator (centre, west, east, north, south)."""
    out = torch.empty(5, H, W, dtype=torch.float32, device="cuda")
    _check(load().rgs_csr_to_stencil(h.ptr, ctypes.byref(csr), int(H), int(W), out.data_ptr()), h)
    return out


def rgs_csr_matvec(h, csr, x, y=None):
    """y = A x (FP64 CUDA vectors)."""
    if y is None:
        y = torch.empty_like(x)
    _check(load().rgs_csr_matvec(h.ptr, ctypes.byref(csr), x.data_ptr(), y.data_ptr()), h)
    return y


def rgmres_solve_batched(h, csrs, bs, xs, restarts, ks, rtol=1e-8, max_cycles=100, inner_factor=0.5,
                         qdtype=torch.float32, fixed_steps=False, sketch_seed=0):
    """Independent restarted RGMRES solves in one persistent launch.  csrs: CSR structs,
    bs / xs: FP64 CUDA vectors (xs: initial guesses, overwritten), restarts / ks: per instance.
    Returns one result dict per instance (as rgmres_solve)."""
    nb = len(csrs)
    if not (len(bs) == len(xs) == len(restarts) == len(ks) == nb):
        raise ValueError("one b, x, restart and k per system")
    A = (CSR * nb)(*csrs)
    bp = (ctypes.c_void_p * nb)(*[v.data_ptr() for v in bs])
    xp = (ctypes.c_void_p * nb)(*[v.data_ptr() for v in xs])
    rt = [rtol] * nb if not hasattr(rtol, "__len__") else list(rtol)
    mc = [max_cycles] * nb if not hasattr(max_cycles, "__len__") else list(max_cycles)
    opts = (BatchOpts * nb)(*[BatchOpts(int(restarts[i]), int(ks[i]), int(mc[i]), _DTYPE[qdtype], float(rt[i]),
                                        float(inner_factor), 1 if fixed_steps else 0, 0) for i in range(nb)])
    hists = [(ctypes.c_double * (mc[i] + 1))() for i in range(nb)]
    info = (GmresInfo * nb)()
    for i in range(nb):
        info[i].history = ctypes.cast(hists[i], ctypes.POINTER(ctypes.c_double))
    _check(load().rgmres_solve_batched(h.ptr, nb, A, bp, xp, opts, int(sketch_seed), info), h)
    return [{"cycles": info[i].cycles, "total_steps": info[i].total_steps, "converged": bool(info[i].converged),
             "status": info[i].status, "rel_residual": info[i].rel_residual,
             "history": [hists[i][c] for c in range(info[i].cycles + 1)]} for i in range(nb)]


def _tuning_dict(t):
    return {"upd_blocks_per_sm": t.upd_blocks_per_sm, "batch_blocks_per_sm": t.batch_blocks_per_sm,
            "batch_min_team_work": t.batch_min_team_work, "ls_blocks": t.ls_blocks,
            "batch_rows_per_thread": t.batch_rows_per_thread}


def rgs_get_tuning(h):
    t = Tuning()
    _check(load().rgs_get_tuning(h.ptr, ctypes.byref(t)), h)
    return _tuning_dict(t)


def rgs_set_tuning(h, upd_blocks_per_sm, batch_blocks_per_sm, batch_min_team_work, ls_blocks=0,
                   batch_rows_per_thread=0):
    t = Tuning(int(upd_blocks_per_sm), int(batch_blocks_per_sm), float(batch_min_team_work), int(ls_blocks),
               int(batch_rows_per_thread))
    _check(load().rgs_set_tuning(h.ptr, ctypes.byref(t)), h)


def rgs_autotune_update(h, sk, ncols, qdtype=torch.float32):
    """Time the fused update pass for 2..4 CTAs per SM on this sketch's n; keep the fastest."""
    t = Tuning()
    ms = (ctypes.c_float * 3)()
    _check(load().rgs_autotune_update(h.ptr, sk.ptr, int(ncols), _DTYPE[qdtype], ctypes.byref(t), ms), h)
    return {**_tuning_dict(t), "ms": list(ms)}


def rgs_autotune_batched(h, csrs, bs, restarts, ks, cycles=1, qdtype=torch.float32, sketch_seed=0):
    """Time the batched solver's grid candidates on this batch (fixed cycles); keep the fastest."""
    nb = len(csrs)
    A = (CSR * nb)(*csrs)
    bp = (ctypes.c_void_p * nb)(*[v.data_ptr() for v in bs])
    opts = (BatchOpts * nb)(*[BatchOpts(int(restarts[i]), int(ks[i]), 1, _DTYPE[qdtype], 1e-8, 0.5, 1, 0)
                              for i in range(nb)])
    t = Tuning()
    ms = (ctypes.c_float * 12)()
    _check(load().rgs_autotune_batched(h.ptr, nb, A, bp, opts, int(sketch_seed), int(cycles), ctypes.byref(t), ms), h)
    return {**_tuning_dict(t), "ms": list(ms)}


def csr_to_device(rowptr, colind, val, device="cuda"):
    """Device copies of CSR arrays (int32, int32, FP64) and the C struct pointing at them."""
    t = (torch.as_tensor(rowptr, dtype=torch.int32).to(device), torch.as_tensor(colind, dtype=torch.int32).to(device),
         torch.as_tensor(val, dtype=torch.float64).to(device))
    return t, csr_struct(*t)


# ------------------------------------------------------------------ preconditioning
class _DeviceVector:
    """A device vector the library owns, seen as a torch tensor without a copy (torch takes no
    read-only flag: the callback's contract says v is not written)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 2,
                                         "strides": None}


def _device_tensor(ptr, n, dtype):
    if dtype == RGS_BF16:      # no BF16 type string in the array interface: view the 16-bit words
        return torch.as_tensor(_DeviceVector(ptr, n, "<i2"), device="cuda").view(torch.bfloat16)
    return torch.as_tensor(_DeviceVector(ptr, n, {RGS_F64: "<f8", RGS_F32: "<f4"}[dtype]), device="cuda")


def _precond_trampoline(fn, errors):
    """The C callback around ``fn(v, z)``: v (read only) and z are torch views of the library's
    device vectors, and fn runs with the handle's stream as torch's current stream.  An exception
    is kept in ``errors`` and returned as a nonzero status (the solve then fails with
    RGS_ERR_CALLBACK and the binding re-raises it)."""
    def apply(user, n, v, vtype, z, ztype, stream):
        try:
            vt = _device_tensor(v, n, vtype)
            zt = _device_tensor(z, n, ztype)
            ts = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(ts):
                fn(vt, zt)
            return 0
        except BaseException as e:          # noqa: BLE001 - carried back across the C frame
            errors.append(e)
            return 1
    return PrecondApplyFn(apply)


def rgmres_set_preconditioner(h, kind, net=None, logkappa=None, flexible=False, apply=None, nonlinear=False):
    """Select the right preconditioner of the following rgmres_solve calls on ``h``:
    "none", "jacobi", "learned" (a ConvNet and its log-kappa grid, FP64 on the device; flexible)
    or "callback": ``apply(v, z)`` writes z = M(v) with torch operations on the current stream
    (v of the basis type, or FP64 for the end-of-cycle vector Q y when not flexible; z FP64 for
    an FP64 basis, else FP32).  ``flexible`` keeps every z; a linear M may run without it.
    ``nonlinear`` puts M under the fallback rule of the learned preconditioner."""
    k = {"none": RGS_PRECOND_NONE, "jacobi": RGS_PRECOND_JACOBI, "learned": RGS_PRECOND_LEARNED_CONV,
         "callback": RGS_PRECOND_CALLBACK}[kind]
    params = None
    if k == RGS_PRECOND_CALLBACK:
        if apply is None:
            raise ValueError("the callback preconditioner needs apply(v, z)")
        errors = []
        fnp = _precond_trampoline(apply, errors)
        h._precond = CallbackPrecond(fnp, None, 1 if nonlinear else 0, 0)
        h._precond_refs = (fnp, apply)          # the C function pointer must outlive the solves
        h._precond_errors = errors
        params = ctypes.byref(h._precond)
    elif k == RGS_PRECOND_LEARNED_CONV:
        if logkappa.dtype != torch.float64 or not logkappa.is_cuda or not logkappa.is_contiguous():
            raise ValueError("logkappa must be a contiguous FP64 CUDA tensor")
        h._precond = LearnedPrecond(net.ptr, logkappa.data_ptr())
        h._precond_refs = (net, logkappa)          # the library keeps the pointers
        params = ctypes.byref(h._precond)
    else:
        h._precond_refs = None
    _check(load().rgmres_set_preconditioner(h.ptr, k, params, 1 if flexible else 0), h)


class ConvNet:
    def __init__(self, ptr, handle, height, width, max_batch):
        self.ptr, self.handle, self.height, self.width, self.max_batch = ptr, handle, height, width, max_batch

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None and not _exiting:
            _lib.rgs_convnet_destroy(self.ptr)
            self.ptr = None


def rgs_convnet_num_params():
    return int(load().rgs_convnet_num_params())


def rgs_convnet_create(h, height, width, max_batch=1, seed=0):
    out = ctypes.c_void_p()
    _check(load().rgs_convnet_create(h.ptr, int(height), int(width), int(max_batch), int(seed), ctypes.byref(out)), h)
    return ConvNet(out.value, h, int(height), int(width), int(max_batch))


def rgs_convnet_get_params(h, net):
    """The flat FP32 parameters as a NumPy array."""
    import numpy as np
    p = np.empty(rgs_convnet_num_params(), dtype=np.float32)
    _check(load().rgs_convnet_get_params(h.ptr, net.ptr, p.ctypes.data_as(ctypes.c_void_p), p.size), h)
    return p


def rgs_convnet_set_params(h, net, params):
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().rgs_convnet_set_params(h.ptr, net.ptr, p.ctypes.data_as(ctypes.c_void_p), p.size), h)


def _net_io(net, x, name, channels):
    shape = (x.shape[0], channels, net.height, net.width) if channels > 1 else (x.shape[0], net.height, net.width)
    if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous() or tuple(x.shape) != shape:
        raise ValueError(f"{name} must be a contiguous FP32 CUDA tensor of shape {shape}")


def rgs_convnet_forward(h, net, x, out=None):
    """out (B x H x W) = net(x) for x of shape (B, 2, H, W) FP32 on the device."""
    _net_io(net, x, "x", 2)
    if out is None:
        out = torch.empty(x.shape[0], net.height, net.width, dtype=torch.float32, device=x.device)
    _net_io(net, out, "out", 1)
    _check(load().rgs_convnet_forward(h.ptr, net.ptr, x.shape[0], x.data_ptr(), out.data_ptr()), h)
    return out


def _stencil_ptr(net, stencil, B):
    if stencil is None:
        return None
    shape = (B, 5, net.height, net.width)
    if stencil.dtype != torch.float32 or not stencil.is_cuda or not stencil.is_contiguous() or \
            tuple(stencil.shape) != shape:
        raise ValueError(f"stencil must be a contiguous FP32 CUDA tensor of shape {shape}")
    return stencil.data_ptr()


def rgs_convnet_loss_grad(h, net, x, target, stencil=None):
    """(loss, flat FP32 gradient as NumPy) of mean_b ||F_b - t_b||^2 / ||t_b||^2, F_b = net(x_b)
    or, with a 5-point ``stencil`` (B x 5 x H x W), F_b = A_b net(x_b)."""
    import numpy as np
    _net_io(net, x, "x", 2)
    _net_io(net, target, "target", 1)
    loss = ctypes.c_double()
    g = np.empty(rgs_convnet_num_params(), dtype=np.float32)
    _check(load().rgs_convnet_loss_grad(h.ptr, net.ptr, x.shape[0], x.data_ptr(), target.data_ptr(),
                                        _stencil_ptr(net, stencil, x.shape[0]), ctypes.byref(loss),
                                        g.ctypes.data_as(ctypes.c_void_p)), h)
    return loss.value, g


def rgs_convnet_train_step(h, net, x, target, lr=1e-3, stencil=None):
    """One Adam step on the batch; returns the loss before the step."""
    _net_io(net, x, "x", 2)
    _net_io(net, target, "target", 1)
    loss = ctypes.c_double()
    _check(load().rgs_convnet_train_step(h.ptr, net.ptr, x.shape[0], x.data_ptr(), target.data_ptr(),
                                         _stencil_ptr(net, stencil, x.shape[0]), float(lr), ctypes.byref(loss)), h)
    return loss.value
