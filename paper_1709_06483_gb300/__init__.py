"""GB300 (sm_103a) Magnus integrators with Leja interpolation (arXiv:1709.06483).

Thin Python binding over the C ABI of ``include/magnus.h`` (``libmagnus_gb300.so``,
built in-tree by :mod:`paper_1709_06483_gb300.build`).  It only marshals
arguments: every step of the method runs in the library's CUDA kernels.  PyTorch
provides device memory and streams.  There is no CPU fallback: if the library is
missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmagnus_gb300.so")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ENONFINITE, ETIMEOUT, EDRIFT = range(8)
M4, CF4, CF4_3, M2, M6 = 1, 2, 3, 4, 5
VARIANTS = {"M4": M4, "CF4": CF4, "CF4_3": CF4_3, "M2": M2, "M6": M6}
TERM_CSR, TERM_DENSE, TERM_XXZ, TERM_FIELD_X, TERM_CSR_REAL, TERM_DENSE_REAL = 0, 1, 2, 3, 4, 5
FP64, FP32_SPLIT, TENSOR_SLICED = 0, 1, 2
INTERVALS = {"gershgorin": 0, "lanczos": 1}
# options.row_layout (magnus_row_layout) of fixed-point CSR plans; stats report the number
ROW_LAYOUTS = {"auto": 0, "staged": 1, "csr": 2, "sliced": 3}

# Every symbol the header declares (checked by the CPU test suite).
EXPORTS = (
    "magnus_plan_create", "magnus_plan_destroy", "magnus_last_error", "magnus_status_string", "leja_expv",
    "magnus_propagate", "magnus_term_interval", "magnus_leja_points", "magnus_divided_differences",
    "magnus_xxz_nnz", "magnus_build_xxz_csr", "magnus_build_field_x_csr", "magnus_build_longrange_dense",
    "magnus_build_field_x_dense", "magnus_expv_xxz_static", "magnus_batch_create", "magnus_batch_propagate",
    "magnus_batch_destroy", "magnus_batch_last_error", "magnus_adjoint_grad", "magnus_real_parts", "magnus_apply",
    "magnus_set_coeff",
)


class MagnusError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_status_name(code)}: {msg}")
        self.code = code


class Term(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nspins", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p), ("J", C.POINTER(C.c_double)),
                ("hz", C.POINTER(C.c_double)), ("delta", C.c_double)]


class Coeff(C.Structure):
    _fields_ = [("a0", C.c_double), ("nmodes", C.c_int32), ("_pad", C.c_int32), ("ac", C.POINTER(C.c_double)),
                ("as_", C.POINTER(C.c_double)), ("om", C.POINTER(C.c_double))]


class Options(C.Structure):
    _fields_ = [("tol_rel", C.c_double), ("tol_abs", C.c_double), ("rho_max", C.c_double), ("m_max", C.c_int32),
                ("nvec", C.c_int32), ("ctas", C.c_int32), ("precision", C.c_int32), ("barrier_timeout_s", C.c_double),
                ("test_skip_arrival", C.c_int32), ("interval", C.c_int32), ("fixed_sums", C.c_int32),
                ("row_layout", C.c_int32), ("plain_values", C.c_int32), ("_reserved", C.c_int32),
                ("norm_check", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("n_exp", C.c_int64), ("n_substeps", C.c_int64), ("n_matvec", C.c_int64),
                ("n_termapply", C.c_int64), ("max_m", C.c_int32), ("status", C.c_int32),
                ("m_log", C.POINTER(C.c_int32)), ("m_log_cap", C.c_int64), ("kernel_ms", C.c_double),
                ("grid", C.c_int32), ("block", C.c_int32), ("fixed_sums", C.c_int32), ("row_layout", C.c_int32),
                ("norm_drift", C.c_double)]


class BatchItem(C.Structure):
    _fields_ = [("dim", C.c_int64), ("nterms", C.c_int32), ("_pad", C.c_int32), ("terms", C.POINTER(Term)),
                ("coeffs", C.POINTER(Coeff))]


class BatchStats(C.Structure):
    _fields_ = [("n_exp", C.c_int64), ("n_substeps", C.c_int64), ("n_matvec", C.c_int64),
                ("n_termapply", C.c_int64), ("max_m", C.c_int32), ("status", C.c_int32),
                ("m_log", C.POINTER(C.c_int32)), ("m_log_cap_per_item", C.c_int64), ("graph_ms", C.c_double),
                ("block", C.c_int32), ("cluster", C.c_int32), ("fixed_sums", C.c_int32), ("_pad", C.c_int32)]


_lib = None
_lock = threading.Lock()


def _declare(L):
    P, D, I32, I64 = C.c_void_p, C.c_double, C.c_int32, C.c_int64
    sig = {
        "magnus_plan_create": (I32, [C.POINTER(C.c_void_p), I64, I32, C.POINTER(Term), C.POINTER(Coeff),
                                     C.POINTER(Options), P]),
        "magnus_plan_destroy": (I32, [P]),
        "magnus_last_error": (C.c_char_p, [P]),
        "magnus_status_string": (C.c_char_p, [I32]),
        "leja_expv": (I32, [P, C.POINTER(D), P, P, C.POINTER(Stats)]),
        "magnus_propagate": (I32, [P, P, D, D, I64, I32, C.POINTER(Stats)]),
        "magnus_term_interval": (I32, [P, I32, C.POINTER(D), C.POINTER(D)]),
        "magnus_leja_points": (I32, [P, C.POINTER(D), I32]),
        "magnus_divided_differences": (I32, [P, D, P, I32]),
        "magnus_xxz_nnz": (I64, [I32]),
        "magnus_build_xxz_csr": (I32, [I32, C.POINTER(D), C.POINTER(D), D, P, P, P, P]),
        "magnus_build_field_x_csr": (I32, [I32, P, P, P, P]),
        "magnus_build_longrange_dense": (I32, [I32, D, C.POINTER(D), D, P, P]),
        "magnus_build_field_x_dense": (I32, [I32, P, P]),
        "magnus_expv_xxz_static": (I32, [I32, C.POINTER(D), C.POINTER(D), D, C.POINTER(D), P, P, D, P]),
        "magnus_batch_create": (I32, [C.POINTER(C.c_void_p), I32, C.POINTER(BatchItem), C.POINTER(Options), P]),
        "magnus_batch_propagate": (I32, [P, C.POINTER(C.c_void_p), D, D, I64, I32, C.POINTER(BatchStats)]),
        "magnus_batch_destroy": (I32, [P]),
        "magnus_batch_last_error": (C.c_char_p, [P]),
        "magnus_adjoint_grad": (I32, [P, P, P, D, D, I64, I32, I32, I32, C.POINTER(D), C.POINTER(D), C.POINTER(Stats)]),
        "magnus_real_parts": (I32, [P, I64, P, P]),
        "magnus_apply": (I32, [P, C.POINTER(D), P, P]),
        "magnus_set_coeff": (I32, [P, I32, C.POINTER(Coeff)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args


def load(path: str = LIB_PATH):
    """Load the in-tree CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with `python -m paper_1709_06483_gb300.build` "
                                   "(there is no CPU fallback)")
            L = C.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def _status_name(code: int) -> str:
    try:
        return load().magnus_status_string(code).decode()
    except Exception:  # noqa: BLE001 - naming only
        return f"status {code}"


def _check(code: int, plan=None):
    if code != OK:
        msg = load().magnus_last_error(plan).decode(errors="replace")
        raise MagnusError(code, msg)


def _dptr(t) -> int:
    """Device pointer of a contiguous CUDA tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ terms / coefficients
def real_parts(z, stream=None):
    """float64 copy of the real parts of a CUDA complex128 tensor; MagnusError(EINVAL) if some
    imaginary part is nonzero (the conversion to real storage must be exact)."""
    import torch
    z = z.contiguous()
    out = torch.empty(z.shape, dtype=torch.float64, device=z.device)
    _check(load().magnus_real_parts(_dptr(z), z.numel(), _dptr(out), _stream_ptr(stream)))
    return out


class CSRTerm:
    """CSR term on the device (int64 row pointers, int32 columns).  Complex values give
    MAGNUS_TERM_CSR (20 B per entry); float64 values give MAGNUS_TERM_CSR_REAL (12 B per entry) for a
    real symmetric matrix."""

    def __init__(self, rowptr, col, val):
        import torch
        self.rowptr = rowptr.to(torch.int64).contiguous()
        self.col = col.to(torch.int32).contiguous()
        self.real = not val.is_complex()
        self.val = val.to(torch.float64 if self.real else torch.complex128).contiguous()

    def as_real(self, stream=None) -> "CSRTerm":
        """The same matrix in real storage (exact; raises if it is not real)."""
        return self if self.real else CSRTerm(self.rowptr, self.col, real_parts(self.val, stream))

    def ctype(self):
        t = Term()
        t.kind, t.nnz = (TERM_CSR_REAL if self.real else TERM_CSR), self.col.numel()
        t.rowptr, t.col, t.val = _dptr(self.rowptr), _dptr(self.col), _dptr(self.val)
        return t


class DenseTerm:
    """Dense term on the device, row-major dim x dim: complex128 (MAGNUS_TERM_DENSE) or float64 for a
    real symmetric matrix (MAGNUS_TERM_DENSE_REAL, half the bytes)."""

    def __init__(self, H):
        import torch
        self.real = not H.is_complex()
        self.val = H.to(torch.float64 if self.real else torch.complex128).contiguous()

    def as_real(self, stream=None) -> "DenseTerm":
        """The same matrix in real storage (exact; raises if it is not real)."""
        return self if self.real else DenseTerm(real_parts(self.val, stream))

    def ctype(self):
        t = Term()
        t.kind, t.nnz = (TERM_DENSE_REAL if self.real else TERM_DENSE), self.val.numel()
        t.val = _dptr(self.val)
        return t


class XXZTerm:
    """Matrix-free open XXZ chain sum J_i (sx sx + sy sy + delta sz sz)_{i,i+1} + sum h_i sz_i."""

    def __init__(self, nspins, J, hz, delta=0.5):
        self.nspins, self.J, self.hz, self.delta = int(nspins), _f64(J), _f64(hz), float(delta)

    def ctype(self):
        t = Term()
        t.kind, t.nspins, t.delta = TERM_XXZ, self.nspins, self.delta
        t.J = self.J.ctypes.data_as(C.POINTER(C.c_double))
        t.hz = self.hz.ctypes.data_as(C.POINTER(C.c_double))
        return t


class FieldXTerm:
    """Matrix-free transverse field sum_i sigma^x_i."""

    def __init__(self, nspins):
        self.nspins = int(nspins)

    def ctype(self):
        t = Term()
        t.kind, t.nspins = TERM_FIELD_X, self.nspins
        return t


class Drive:
    """f(t) = a0 + sum_m (ac_m cos(om_m t) + as_m sin(om_m t))."""

    def __init__(self, a0=0.0, ac=(), as_=(), om=()):
        self.a0 = float(a0)
        self.om = _f64(om)
        n = self.om.size
        self.ac = _f64(ac) if len(ac) else np.zeros(n)
        self.as_ = _f64(as_) if len(as_) else np.zeros(n)

    @staticmethod
    def const(v=1.0):
        return Drive(a0=v)

    def ctype(self):
        c = Coeff()
        c.a0, c.nmodes = self.a0, self.om.size
        P = C.POINTER(C.c_double)
        c.ac, c.as_, c.om = (self.ac.ctypes.data_as(P), self.as_.ctypes.data_as(P), self.om.ctypes.data_as(P))
        return c


# ------------------------------------------------------------------ plan
class Plan:
    """A Magnus/Leja plan: dim, terms H_k with drives f_k, Leja tolerance, vectors per call."""

    def __init__(self, dim, terms, drives, tol=1e-10, tol_abs=None, rho_max=4.0, m_max=100, nvec=1, ctas=0,
                 precision=FP64, stream=None, barrier_timeout_s=0.0, test_skip_arrival=0, interval="gershgorin",
                 fixed_sums=True, rows="auto", plain_values=False, norm_check=0.0):
        import torch
        L = load()
        if len(terms) != len(drives):
            raise ValueError(f"{len(terms)} terms but {len(drives)} drives")
        self.dim, self.nvec, self.nterms = int(dim), int(nvec), len(terms)
        self._terms, self._drives = list(terms), list(drives)  # keep borrowed buffers alive
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        tarr = (Term * len(terms))(*[t.ctype() for t in terms])
        carr = (Coeff * len(drives))(*[d.ctype() for d in drives])
        opt = Options(float(tol), float(tol if tol_abs is None else tol_abs), float(rho_max), int(m_max), int(nvec),
                      int(ctas), int(precision), float(barrier_timeout_s), int(test_skip_arrival),
                      INTERVALS[interval], int(bool(fixed_sums)), ROW_LAYOUTS[rows], int(bool(plain_values)), 0,
                      float(norm_check))
        h = C.c_void_p()
        _check(L.magnus_plan_create(C.byref(h), self.dim, len(terms), tarr, carr, C.byref(opt),
                                    _stream_ptr(self.stream)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().magnus_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def _stats(self, log_cap):
        st = Stats()
        log = None
        if log_cap:
            log = np.zeros(log_cap, dtype=np.int32)
            st.m_log = log.ctypes.data_as(C.POINTER(C.c_int32))
            st.m_log_cap = log_cap
        return st, log

    def _check_state(self, t):
        import torch
        if t.dtype != torch.complex128 or t.numel() != self.dim * self.nvec:
            raise ValueError(f"expected complex128 with {self.nvec}x{self.dim} entries")

    def propagate(self, psi, t0, h, nsteps, variant="CF4", log_cap=0):
        """psi (CUDA complex128 [nvec][dim], in place) <- nsteps Magnus steps from t0."""
        self._check_state(psi)
        st, log = self._stats(log_cap)
        code = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        _check(load().magnus_propagate(self._h, C.c_void_p(_dptr(psi)), float(t0), float(h), int(nsteps), code,
                                       C.byref(st)), self._h)
        return _as_dict(st, log)

    def expv(self, beta, v, out=None, log_cap=0):
        """out = exp(-i sum_k beta_k H_k) v (CUDA complex128)."""
        import torch
        self._check_state(v)
        if out is None:
            out = torch.empty_like(v)
        b = _f64(beta)
        if b.size != self.nterms:
            raise ValueError(f"beta needs {self.nterms} values, got {b.size}")
        st, log = self._stats(log_cap)
        _check(load().leja_expv(self._h, b.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(_dptr(v)),
                                C.c_void_p(_dptr(out)), C.byref(st)), self._h)
        return out, _as_dict(st, log)

    def set_drive(self, k, drive):
        """Replace the drive f_k of term k (stream-ordered; enclosures unchanged)."""
        self._drives[k] = drive
        c = drive.ctype()
        _check(load().magnus_set_coeff(self._h, int(k), C.byref(c)), self._h)

    def apply(self, beta, x, y=None):
        """y = sum_k beta_k H_k x for every state (CUDA complex128 [nvec][dim]; asynchronous)."""
        import torch
        self._check_state(x)
        if y is None:
            y = torch.empty_like(x)
        b = _f64(beta)
        if b.size != self.nterms:
            raise ValueError(f"beta needs {self.nterms} values, got {b.size}")
        _check(load().magnus_apply(self._h, b.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(_dptr(x)),
                                   C.c_void_p(_dptr(y))), self._h)
        return y

    def adjoint_grad(self, psi0, phi, t0, h, nsteps, variant="CF4", kd=1, ckpt_every=16):
        """F = |<phi|psi(T)>|^2 and dF/d(a0, ac_m, as_m) of term kd's drive (adjoint, checkpointed)."""
        self._check_state(psi0)
        self._check_state(phi)
        nm = self._drives[kd].om.size
        grad = np.zeros(1 + 2 * nm)
        F = C.c_double()
        st = Stats()
        code = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        _check(load().magnus_adjoint_grad(self._h, C.c_void_p(_dptr(psi0)), C.c_void_p(_dptr(phi)), float(t0),
                                          float(h), int(nsteps), code, int(kd), int(ckpt_every), C.byref(F),
                                          grad.ctypes.data_as(C.POINTER(C.c_double)), C.byref(st)), self._h)
        return F.value, grad, _as_dict(st, None)

    def interval(self, k):
        a, b = C.c_double(), C.c_double()
        _check(load().magnus_term_interval(self._h, k, C.byref(a), C.byref(b)), self._h)
        return a.value, b.value

    def leja_points(self, count):
        xi = np.zeros(count)
        _check(load().magnus_leja_points(self._h, xi.ctypes.data_as(C.POINTER(C.c_double)), count), self._h)
        return xi

    def divided_differences(self, rho, count):
        d = np.zeros(count, dtype=np.complex128)
        _check(load().magnus_divided_differences(self._h, float(rho), C.c_void_p(d.ctypes.data), count), self._h)
        return d


def _as_dict(st: Stats, log):
    out = {k: getattr(st, k) for k in ("n_exp", "n_substeps", "n_matvec", "n_termapply", "max_m", "status",
                                       "kernel_ms", "grid", "block", "fixed_sums", "row_layout", "norm_drift")}
    if log is not None:
        out["m_log"] = log[: min(st.n_substeps, log.size)].copy()
    return out


# ------------------------------------------------------------------ batches
class Batch:
    """Many independent problems (dim_i, terms_i, drives_i) advanced together in one persistent launch
    under a replayed CUDA graph, with an autotuned CTA size."""

    def __init__(self, problems, tol=1e-10, tol_abs=None, rho_max=4.0, m_max=100, ctas=0, fixed_sums=True):
        L = load()
        self._keep = []
        arr = (BatchItem * len(problems))()
        for i, (dim, terms, drives) in enumerate(problems):
            t = (Term * len(terms))(*[x.ctype() for x in terms])
            c = (Coeff * len(drives))(*[x.ctype() for x in drives])
            self._keep += [terms, drives, t, c]
            arr[i].dim, arr[i].nterms = int(dim), len(terms)
            arr[i].terms, arr[i].coeffs = t, c
        self.count = len(problems)
        self.dims = [int(p[0]) for p in problems]
        opt = Options(float(tol), float(tol if tol_abs is None else tol_abs), float(rho_max), int(m_max), 1,
                      int(ctas), FP64, 0.0, 0, 0, int(bool(fixed_sums)), 0)
        h = C.c_void_p()
        code = L.magnus_batch_create(C.byref(h), self.count, arr, C.byref(opt), None)
        if code != OK:
            raise MagnusError(code, L.magnus_batch_last_error(None).decode(errors="replace"))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().magnus_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def propagate(self, psis, t0, h, nsteps, variant="CF4", log_cap=0):
        """psis: list of CUDA complex128 tensors (in place)."""
        if len(psis) != self.count:
            raise ValueError(f"expected {self.count} states, got {len(psis)}")
        ptrs = (C.c_void_p * self.count)(*[_dptr(p) for p in psis])
        st = BatchStats()
        log = None
        if log_cap:
            log = np.zeros((self.count, log_cap), dtype=np.int32)
            st.m_log = log.ctypes.data_as(C.POINTER(C.c_int32))
            st.m_log_cap_per_item = log_cap
        code = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        L = load()
        rc = L.magnus_batch_propagate(self._h, ptrs, float(t0), float(h), int(nsteps), code, C.byref(st))
        if rc != OK:
            raise MagnusError(rc, L.magnus_batch_last_error(self._h).decode(errors="replace"))
        out = {k: getattr(st, k) for k in ("n_exp", "n_substeps", "n_matvec", "n_termapply", "max_m", "status",
                                           "graph_ms", "block", "cluster", "fixed_sums")}
        if log is not None:
            out["m_log"] = log
        return out


# ------------------------------------------------------------------ builders
def xxz_nnz(nspins: int) -> int:
    return int(load().magnus_xxz_nnz(nspins))


def build_xxz_csr(nspins, J, hz, delta=0.5, device="cuda", stream=None) -> CSRTerm:
    import torch
    D = 1 << nspins
    nnz = xxz_nnz(nspins)
    rp = torch.empty(D + 1, dtype=torch.int64, device=device)
    col = torch.empty(nnz, dtype=torch.int32, device=device)
    val = torch.empty(nnz, dtype=torch.complex128, device=device)
    J, hz = _f64(J), _f64(hz)
    P = C.POINTER(C.c_double)
    _check(load().magnus_build_xxz_csr(nspins, J.ctypes.data_as(P), hz.ctypes.data_as(P), float(delta),
                                       C.c_void_p(_dptr(rp)), C.c_void_p(_dptr(col)), C.c_void_p(_dptr(val)),
                                       _stream_ptr(stream)))
    return CSRTerm(rp, col, val)


def build_field_x_csr(nspins, device="cuda", stream=None) -> CSRTerm:
    import torch
    D = 1 << nspins
    rp = torch.empty(D + 1, dtype=torch.int64, device=device)
    col = torch.empty(D * nspins, dtype=torch.int32, device=device)
    val = torch.empty(D * nspins, dtype=torch.complex128, device=device)
    _check(load().magnus_build_field_x_csr(nspins, C.c_void_p(_dptr(rp)), C.c_void_p(_dptr(col)),
                                           C.c_void_p(_dptr(val)), _stream_ptr(stream)))
    return CSRTerm(rp, col, val)


def build_longrange_dense(nspins, hz, alpha=1.5, delta=0.5, device="cuda", stream=None):
    import torch
    D = 1 << nspins
    H = torch.empty((D, D), dtype=torch.complex128, device=device)
    hz = _f64(hz)
    _check(load().magnus_build_longrange_dense(nspins, float(alpha), hz.ctypes.data_as(C.POINTER(C.c_double)),
                                               float(delta), C.c_void_p(_dptr(H)), _stream_ptr(stream)))
    return H


def build_field_x_dense(nspins, device="cuda", stream=None):
    import torch
    D = 1 << nspins
    H = torch.empty((D, D), dtype=torch.complex128, device=device)
    _check(load().magnus_build_field_x_dense(nspins, C.c_void_p(_dptr(H)), _stream_ptr(stream)))
    return H


# ------------------------------------------------------------------ allocation-free entry point
def expv_xxz_static(nspins, J, hz, delta, beta, v, out=None, tol=1e-10, stream=None):
    """out = exp(-i (beta_0 H_xxz + beta_1 sum_i sx_i)) v without a plan and without any device allocation
    inside the library (fixed ~3.2 MB scratch, nspins <= 16).  For callers that cannot call cudaMalloc.
    The first call on a device does a one-time set-up; calls that overlap on the GPU race.  With
    out=None this wrapper allocates the result tensor; pass out (it may be v itself) to allocate
    nothing at all."""
    import torch
    if out is None:
        out = torch.empty_like(v)
    J, hz, b = _f64(J), _f64(hz), _f64(beta)
    if b.size != 2:
        raise ValueError("beta holds the weights of the XXZ term and the field: 2 values")
    P = C.POINTER(C.c_double)
    _check(load().magnus_expv_xxz_static(int(nspins), J.ctypes.data_as(P), hz.ctypes.data_as(P), float(delta),
                                         b.ctypes.data_as(P), C.c_void_p(_dptr(v)), C.c_void_p(_dptr(out)),
                                         float(tol), _stream_ptr(stream)))
    return out


# ------------------------------------------------------------------ autograd
def _fidelity_function():
    import torch

    class FidelityFunction(torch.autograd.Function):
        """F(c) = |<phi|psi(T)>|^2 for the drive coefficients c = (a0, ac[0..m), as[0..m)) of term kd;
        backward returns dF/dc from the adjoint kernels (magnus_adjoint_grad)."""

        @staticmethod
        def forward(ctx, params, plan, kd, psi0, phi, t0, h, nsteps, variant, ckpt_every):
            om = plan._drives[kd].om
            nm = om.size
            p = params.detach().to("cpu", torch.float64).numpy()
            plan.set_drive(kd, Drive(p[0], p[1:1 + nm], p[1 + nm:1 + 2 * nm], om))
            F, grad, _ = plan.adjoint_grad(psi0, phi, t0, h, nsteps, variant, kd=kd, ckpt_every=ckpt_every)
            ctx.save_for_backward(torch.from_numpy(grad))
            return params.new_tensor(F)

        @staticmethod
        def backward(ctx, gF):
            (grad,) = ctx.saved_tensors
            return (gF * grad.to(gF.device, gF.dtype),) + (None,) * 9

    return FidelityFunction


_FIDELITY = None


def fidelity(plan, params, psi0, phi, t0, h, nsteps, variant="CF4", kd=1, ckpt_every=16):
    """Differentiable F = |<phi|psi(T)>|^2 with respect to params = (a0, ac, as) of term kd's drive
    (a float64 tensor of 1 + 2 nmodes entries, the drive's frequencies fixed); the plan's drive for
    term kd is set to params."""
    global _FIDELITY
    if _FIDELITY is None:
        _FIDELITY = _fidelity_function()
    return _FIDELITY.apply(params, plan, kd, psi0, phi, t0, h, nsteps, variant, ckpt_every)
