"""FP64 CPU oracle for the Magnus + Leja method -- TEST INFRASTRUCTURE, not the product.

Auer, Einkemmer, Kandolf, Ostermann, "Magnus integrators on multicore CPUs and
GPUs" (arXiv:1709.06483): Magnus integrators of Sec. 2 (Methods M2, M4, Cf4,
Cf4:3) with the exponentials applied by Newton-form Leja interpolation (Sec. 3).

The arithmetic lives in plain C (``magnus_oracle.c``); this module only
compiles it with gcc and marshals numpy arrays through ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA library and never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "magnus_oracle.c")
_HDR = os.path.join(_HERE, "magnus_oracle.h")
_LIB = os.path.join(_HERE, "libmagnus_oracle.so")
_LIB_OMP = os.path.join(_HERE, "libmagnus_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

OK, EINVAL, ENOMEM, ENOCONV, ENONFINITE = 0, 1, 2, 4, 5
M4, CF4, CF4_3, M2, M6 = 1, 2, 3, 4, 5
VARIANTS = {"M4": M4, "CF4": CF4, "CF4_3": CF4_3, "M2": M2, "M6": M6}


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no BLAS).  The checker is the build without OpenMP;
    openmp=True gives libmagnus_oracle_omp.so, the same source with its element-wise loops spread
    over threads (identical bits), used only to time the CPU baseline on all host cores."""
    lib_path = _LIB_OMP if openmp else _LIB
    stale = (not os.path.exists(lib_path)) or max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(lib_path)
    if force or stale:
        tmp = lib_path + f".{os.getpid()}.tmp"
        flags = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *flags, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib_path)
    return lib_path


class _Stats(C.Structure):
    _fields_ = [("n_exp", C.c_int64), ("n_substeps", C.c_int64), ("n_matvec", C.c_int64),
                ("n_termapply", C.c_int64), ("max_m", C.c_int32), ("_pad", C.c_int32),
                ("m_log", C.POINTER(C.c_int32)), ("m_log_cap", C.c_int64)]


def _signatures():
    P, D, I64, I32 = C.c_void_p, C.c_double, C.c_int64, C.c_int
    return {
        "orc_leja_points": (I32, [I32, P]),
        "orc_divided_differences": (I32, [I32, P, D, P]),
        "orc_xxz_nnz": (I64, [I32, P, D]),
        "orc_build_xxz_csr": (I32, [I32, P, P, D, P, P, P]),
        "orc_build_field_x_csr": (I32, [I32, P, P, P]),
        "orc_build_longrange_dense": (I32, [I32, D, P, D, P]),
        "orc_build_field_x_dense": (I32, [I32, P]),
        "orc_problem_new": (P, [I64, I32]),
        "orc_problem_free": (None, [P]),
        "orc_set_csr": (I32, [P, I32, P, P, P]),
        "orc_set_dense": (I32, [P, I32, P]),
        "orc_set_coeff": (I32, [P, I32, D, I32, P, P, P]),
        "orc_set_leja": (I32, [P, D, D, I32, D]),
        "orc_term_interval": (I32, [P, I32, C.POINTER(D), C.POINTER(D)]),
        "orc_set_interval_lanczos": (I32, [P, I32, I32]),
        "orc_coeff_eval": (D, [P, I32, D]),
        "orc_apply_term": (I32, [P, I32, P, P]),
        "orc_expv": (I32, [P, P, P, C.POINTER(_Stats)]),
        "orc_propagate": (I32, [P, P, D, D, I64, I32, C.POINTER(_Stats)]),
        "orc_generator_interval": (I32, [P, I32, D, D, C.POINTER(D), C.POINTER(D)]),
        "orc_frechet_expv": (I32, [P, P, I32, P, P, P, C.POINTER(_Stats)]),
        "orc_adjoint_grad": (I32, [P, P, P, D, D, I64, I32, I32, C.POINTER(D), P]),
    }


def load(path: str):
    """Open a build of ``magnus_oracle.c`` at ``path`` and declare its entry points' signatures."""
    L = C.CDLL(path)
    for name, (res, args) in _signatures().items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib(threaded: bool = False):
    """The checker (single-threaded build), or with threaded=True the OpenMP build."""
    global _lib, _lib_omp
    with _lock:
        if threaded:
            if _lib_omp is None:
                _lib_omp = load(build(openmp=True))
            return _lib_omp
        if _lib is None:
            _lib = load(build())
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def _check(code, what):
    if code != OK:
        raise OracleError(code, what)


def leja_points(m: int) -> np.ndarray:
    xi = np.zeros(m + 1, dtype=np.float64)
    _check(lib().orc_leja_points(m, _ptr(xi)), "leja_points")
    return xi


def divided_differences(xi: np.ndarray, rho: float) -> np.ndarray:
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    d = np.zeros(xi.size, dtype=np.complex128)
    _check(lib().orc_divided_differences(xi.size - 1, _ptr(xi), float(rho), _ptr(d)), "divided_differences")
    return d


class CSR:
    """Row-major CSR, int64 row pointers, int32 columns, complex128 values."""

    def __init__(self, rowptr, col, val):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.complex128)
        self.dim = self.rowptr.size - 1

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def todense(self):
        H = np.zeros((self.dim, self.dim), dtype=np.complex128)
        rows = np.repeat(np.arange(self.dim), np.diff(self.rowptr))
        np.add.at(H, (rows, self.col), self.val)
        return H


def xxz_csr(nspins: int, J, hz, delta: float = 0.5) -> CSR:
    J = np.ascontiguousarray(J, dtype=np.float64)
    hz = np.ascontiguousarray(hz, dtype=np.float64)
    assert J.size == nspins - 1 and hz.size == nspins
    D = 1 << nspins
    nnz = lib().orc_xxz_nnz(nspins, _ptr(J), delta)
    rp = np.zeros(D + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz, dtype=np.complex128)
    _check(lib().orc_build_xxz_csr(nspins, _ptr(J), _ptr(hz), float(delta), _ptr(rp), _ptr(col), _ptr(val)),
           "build_xxz_csr")
    return CSR(rp, col, val)


def field_x_csr(nspins: int) -> CSR:
    D = 1 << nspins
    rp = np.zeros(D + 1, dtype=np.int64)
    col = np.zeros(D * nspins, dtype=np.int32)
    val = np.zeros(D * nspins, dtype=np.complex128)
    _check(lib().orc_build_field_x_csr(nspins, _ptr(rp), _ptr(col), _ptr(val)), "build_field_x_csr")
    return CSR(rp, col, val)


def longrange_dense(nspins: int, hz, alpha: float = 1.5, delta: float = 0.5) -> np.ndarray:
    hz = np.ascontiguousarray(hz, dtype=np.float64)
    D = 1 << nspins
    H = np.zeros((D, D), dtype=np.complex128)
    _check(lib().orc_build_longrange_dense(nspins, float(alpha), _ptr(hz), float(delta), _ptr(H)),
           "build_longrange_dense")
    return H


def field_x_dense(nspins: int) -> np.ndarray:
    D = 1 << nspins
    H = np.zeros((D, D), dtype=np.complex128)
    _check(lib().orc_build_field_x_dense(nspins, _ptr(H)), "build_field_x_dense")
    return H


class Coeff:
    """f(t) = a0 + sum_m (ac_m cos(om_m t) + as_m sin(om_m t))."""

    def __init__(self, a0=0.0, ac=(), as_=(), om=()):
        self.a0 = float(a0)
        self.om = np.ascontiguousarray(om, dtype=np.float64)
        n = self.om.size
        self.ac = np.ascontiguousarray(ac if len(ac) else np.zeros(n), dtype=np.float64)
        self.as_ = np.ascontiguousarray(as_ if len(as_) else np.zeros(n), dtype=np.float64)
        assert self.ac.size == n and self.as_.size == n

    @staticmethod
    def const(v=1.0):
        return Coeff(a0=v)

    def __call__(self, t):
        return self.a0 + np.sum(self.ac * np.cos(self.om * t) + self.as_ * np.sin(self.om * t))


class Stats:
    def __init__(self, cap=0):
        self._s = _Stats()
        self._log = np.zeros(max(cap, 1), dtype=np.int32)
        if cap:
            self._s.m_log = self._log.ctypes.data_as(C.POINTER(C.c_int32))
            self._s.m_log_cap = cap

    def __getattr__(self, k):
        if k in ("n_exp", "n_substeps", "n_matvec", "n_termapply", "max_m"):
            return getattr(self._s, k)
        raise AttributeError(k)

    @property
    def m_log(self):
        return self._log[: min(self._s.n_substeps, self._s.m_log_cap)].copy()


class Problem:
    """H(t) = sum_k f_k(t) H_k with H_k CSR or dense (Sec. 4, H = H_1 + h(t) H_2)."""

    def __init__(self, terms, coeffs, tol=1e-10, tol_abs=None, m_max=100, rho_max=4.0, interval="gershgorin",
                 lanczos_steps=48, threaded=False):
        assert len(terms) == len(coeffs) and len(terms) >= 1
        self.terms, self.coeffs = list(terms), list(coeffs)
        self.dim = terms[0].dim if isinstance(terms[0], CSR) else terms[0].shape[0]
        self._keep = []
        L = self._L = lib(threaded)
        self._h = L.orc_problem_new(self.dim, len(terms))
        if not self._h:
            raise OracleError(EINVAL, "problem_new")
        for k, (t, c) in enumerate(zip(terms, coeffs)):
            if isinstance(t, CSR):
                assert t.dim == self.dim
                _check(L.orc_set_csr(self._h, k, _ptr(t.rowptr), _ptr(t.col), _ptr(t.val)), "set_csr")
                self._keep.append(t)
            else:
                H = np.ascontiguousarray(t, dtype=np.complex128)
                assert H.shape == (self.dim, self.dim)
                _check(L.orc_set_dense(self._h, k, _ptr(H)), "set_dense")
                self._keep.append(H)
            self._keep.append(c)
            _check(L.orc_set_coeff(self._h, k, c.a0, c.om.size, _ptr(c.ac), _ptr(c.as_), _ptr(c.om)), "set_coeff")
        _check(L.orc_set_leja(self._h, tol, tol if tol_abs is None else tol_abs, m_max, rho_max), "set_leja")
        if interval == "lanczos":
            for k in range(len(terms)):
                _check(L.orc_set_interval_lanczos(self._h, k, lanczos_steps), "set_interval_lanczos")
        elif interval != "gershgorin":
            raise ValueError(interval)

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.orc_problem_free(self._h)
            self._h = None

    def interval(self, k):
        a, b = C.c_double(), C.c_double()
        _check(self._L.orc_term_interval(self._h, k, C.byref(a), C.byref(b)), "term_interval")
        return a.value, b.value

    def coeff(self, k, t):
        return self._L.orc_coeff_eval(self._h, k, float(t))

    def apply_term(self, k, x):
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y = np.zeros_like(x)
        _check(self._L.orc_apply_term(self._h, k, _ptr(x), _ptr(y)), "apply_term")
        return y

    def expv(self, beta, v, stats: Stats | None = None):
        beta = np.ascontiguousarray(beta, dtype=np.float64)
        out = np.array(v, dtype=np.complex128, copy=True, order="C")
        st = stats._s if stats else None
        _check(self._L.orc_expv(self._h, _ptr(beta), _ptr(out), C.byref(st) if st else None), "expv")
        return out

    def propagate(self, psi, t0, h, nsteps, variant="CF4", stats: Stats | None = None):
        out = np.array(psi, dtype=np.complex128, copy=True, order="C")
        st = stats._s if stats else None
        code = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        _check(self._L.orc_propagate(self._h, _ptr(out), float(t0), float(h), int(nsteps), code,
                                   C.byref(st) if st else None), "propagate")
        return out

    def generator_interval(self, variant, tn, h):
        """Spectral enclosure of the generator K of one M4 or M6 step of size h from tn."""
        a, b = C.c_double(), C.c_double()
        _check(self._L.orc_generator_interval(self._h, VARIANTS[variant], float(tn), float(h), C.byref(a), C.byref(b)),
               "generator_interval")
        return a.value, b.value

    def frechet_expv(self, beta, kd, v):
        """(L(Omega, -i H_kd) v, exp(Omega) v) for Omega = -i sum_k beta_k H_k (augmented block matrix)."""
        beta = np.ascontiguousarray(beta, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.complex128)
        a, b = np.zeros_like(v), np.zeros_like(v)
        _check(self._L.orc_frechet_expv(self._h, _ptr(beta), int(kd), _ptr(v), _ptr(a), _ptr(b), None), "frechet_expv")
        return a, b

    def adjoint_grad(self, psi0, phi, t0, h, nsteps, variant="CF4", kd=1):
        """F = |<phi|psi(T)>|^2 and dF/d(a0, ac_m, as_m) of term kd's drive."""
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
        phi = np.ascontiguousarray(phi, dtype=np.complex128)
        ng = 1 + 2 * self.coeffs[kd].om.size
        grad = np.zeros(ng)
        F = C.c_double()
        code = VARIANTS[variant] if isinstance(variant, str) else int(variant)
        _check(self._L.orc_adjoint_grad(self._h, _ptr(psi0), _ptr(phi), float(t0), float(h), int(nsteps), code, int(kd),
                                      C.byref(F), _ptr(grad)), "adjoint_grad")
        return F.value, grad
