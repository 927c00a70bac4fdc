"""Error behaviour of the C ABI on invalid arguments (CPU only).

Every call below is rejected by the library's host-side checks before it makes any CUDA call, so
the test needs no GPU and never hands a kernel a bad pointer: the pointers are either null or never
dereferenced because an earlier check fails.  Each rejection must return MAGNUS_EINVAL, leave the
output handle NULL, and describe the problem in the last-error text.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1709_06483_gb300 as mg

FAKE = 0x10000        # a 16-byte aligned address that no check below lets a kernel see
FAKE_ODD = 0x10008    # 8-byte aligned, not 16-byte aligned


@pytest.fixture(scope="module")
def L():
    from paper_1709_06483_gb300 import build
    build.build()
    return mg.load()


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _plan_create(L, dim, terms, coeffs, opt=None, nterms=None):
    out = C.c_void_p(FAKE)
    T = (mg.Term * max(1, len(terms)))(*terms) if terms else None
    Cf = (mg.Coeff * max(1, len(coeffs)))(*coeffs) if coeffs else None
    n = len(terms) if nterms is None else nterms
    rc = L.magnus_plan_create(C.byref(out), dim, n, T, Cf, C.byref(opt) if opt is not None else None, None)
    return rc, out.value


def _options(**kw):
    o = mg.Options(tol_rel=1e-10, tol_abs=1e-10, rho_max=4.0, m_max=100, nvec=1, ctas=0, precision=mg.FP64,
                   barrier_timeout_s=4.0, test_skip_arrival=0, interval=0, fixed_sums=1)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


J = np.array([1.0, 0.8, 1.2])
HZ = np.array([0.1, -0.3, 0.2, 0.5])


def _xxz(nspins=4):
    return mg.Term(kind=mg.TERM_XXZ, nspins=nspins, J=_dp(J), hz=_dp(HZ), delta=0.5)


def _field(nspins=4):
    return mg.Term(kind=mg.TERM_FIELD_X, nspins=nspins)


def _const():
    return mg.Coeff(a0=1.0, nmodes=0)


def _last(L):
    return L.magnus_last_error(None).decode()


def test_status_names(L):
    names = ["MAGNUS_OK", "MAGNUS_EINVAL", "MAGNUS_ENOMEM", "MAGNUS_ECUDA", "MAGNUS_ENOCONV",
             "MAGNUS_ENONFINITE", "MAGNUS_ETIMEOUT"]
    for code, name in enumerate(names):
        assert L.magnus_status_string(code).decode() == name


@pytest.mark.parametrize("case, expect", [
    ("dim0", "dim 0 out of range"),
    ("nterms0", "nterms must be"),
    ("nterms5", "nterms must be"),
    ("tol", "tolerances"),
    ("fixed_sums", "fixed_sums must be 0 or 1"),
    ("rho_max", "rho_max must be > 0"),
    ("barrier", "barrier_timeout_s"),
    ("m_max", "m_max must be"),
    ("nvec", "nvec must be"),
    ("interval", "interval must be"),
    ("precision", "precision must be"),
    ("nmodes", "nmodes must be"),
    ("csr_missing", "CSR arrays missing"),
    ("csr_misaligned", "16-byte aligned"),
    ("dense_big", "dense terms need dim <= 65536"),
    ("xxz_dim", "XXZ needs dim = 2^nspins"),
    ("xxz_no_J", "XXZ needs dim = 2^nspins"),
    ("field_dim", "FIELD_X needs dim = 2^nspins"),
    ("kind", "unknown kind"),
])
def test_plan_create_rejects(L, case, expect):
    terms, coeffs, dim, opt, nterms = [_xxz(), _field()], [_const(), _const()], 16, None, None
    if case == "dim0":
        dim = 0
    elif case == "nterms0":
        nterms = 0
    elif case == "nterms5":
        terms, coeffs = [_xxz()] * 5, [_const()] * 5
    elif case == "tol":
        opt = _options(tol_rel=0.0, tol_abs=0.0)
    elif case == "fixed_sums":
        opt = _options(fixed_sums=2)
    elif case == "rho_max":
        opt = _options(rho_max=0.0)
    elif case == "barrier":
        opt = _options(barrier_timeout_s=601.0)
    elif case == "m_max":
        opt = _options(m_max=1)
    elif case == "nvec":
        opt = _options(nvec=65)
    elif case == "interval":
        opt = _options(interval=7)
    elif case == "precision":
        opt = _options(precision=9)
    elif case == "nmodes":
        coeffs = [_const(), mg.Coeff(a0=0.0, nmodes=2)]  # modes without frequencies
    elif case == "csr_missing":
        terms = [mg.Term(kind=mg.TERM_CSR, nnz=4, rowptr=FAKE, col=None, val=FAKE), _field()]
    elif case == "csr_misaligned":
        terms = [mg.Term(kind=mg.TERM_CSR, nnz=4, rowptr=FAKE, col=FAKE, val=FAKE_ODD), _field()]
    elif case == "dense_big":
        dim = 1 << 17
        terms, coeffs = [mg.Term(kind=mg.TERM_DENSE, val=FAKE)], [_const()]
    elif case == "xxz_dim":
        dim = 32
    elif case == "xxz_no_J":
        terms = [mg.Term(kind=mg.TERM_XXZ, nspins=4, J=None, hz=_dp(HZ), delta=0.5), _field()]
    elif case == "field_dim":
        terms = [_field(3)]
        coeffs = [_const()]
    elif case == "kind":
        terms = [mg.Term(kind=42), _field()]
    rc, handle = _plan_create(L, dim, terms, coeffs, opt, nterms)
    assert rc == mg.EINVAL
    assert handle is None  # *plan is NULL on error
    assert expect in _last(L), _last(L)


def test_plan_create_null_arguments(L):
    assert L.magnus_plan_create(None, 16, 1, None, None, None, None) == mg.EINVAL
    assert "plan pointer is null" in _last(L)
    out = C.c_void_p(FAKE)
    assert L.magnus_plan_create(C.byref(out), 16, 1, None, None, None, None) == mg.EINVAL
    assert out.value is None and "terms/coeffs are null" in _last(L)


def test_calls_on_a_null_plan(L):
    beta = np.zeros(2)
    a, b = C.c_double(), C.c_double()
    xi = np.zeros(4)
    assert L.magnus_plan_destroy(None) == mg.OK
    assert L.leja_expv(None, _dp(beta), FAKE, FAKE, None) == mg.EINVAL
    assert L.magnus_propagate(None, FAKE, 0.0, 0.01, 1, mg.CF4, None) == mg.EINVAL
    assert L.magnus_apply(None, _dp(beta), FAKE, FAKE + 16) == mg.EINVAL
    assert L.magnus_set_coeff(None, 0, None) == mg.EINVAL
    assert L.magnus_term_interval(None, 0, C.byref(a), C.byref(b)) == mg.EINVAL
    assert L.magnus_leja_points(None, _dp(xi), 4) == mg.EINVAL
    F, g = C.c_double(), np.zeros(3)
    assert L.magnus_adjoint_grad(None, FAKE, FAKE, 0.0, 0.01, 1, mg.CF4, 1, 16, C.byref(F), _dp(g), None) == mg.EINVAL
    assert "plan is null" in _last(L)


def test_real_parts_rejects_bad_sizes(L):
    assert L.magnus_real_parts(FAKE, -1, FAKE, None) == mg.EINVAL
    assert L.magnus_real_parts(None, 4, FAKE, None) == mg.EINVAL
    assert "real_parts: bad arguments" in _last(L)


@pytest.mark.parametrize("case, expect", [
    ("nspins17", "nspins must be 2..16"),
    ("nspins1", "nspins must be 2..16"),
    ("null", "null argument"),
    ("misaligned", "16-byte aligned"),
    ("tol", "tol must be > 0"),
    ("beta_inf", "beta not finite"),
    ("beta_nan", "beta not finite"),
])
def test_static_expv_rejects(L, case, expect):
    """The allocation-free entry point refuses chains beyond its fixed scratch and bad arguments
    before touching the device."""
    nspins, j, hz, v, out, tol = 4, _dp(J), _dp(HZ), FAKE, FAKE + 4096, 1e-10
    beta = np.array([0.1, 0.05])
    if case == "nspins17":
        nspins = 17
    elif case == "nspins1":
        nspins = 1
    elif case == "null":
        j = None
    elif case == "misaligned":
        v = FAKE_ODD
    elif case == "tol":
        tol = 0.0
    elif case == "beta_inf":
        beta[1] = np.inf
    elif case == "beta_nan":
        beta[0] = np.nan
    rc = L.magnus_expv_xxz_static(nspins, j, hz, 0.5, _dp(beta), v, out, tol, None)
    assert rc == mg.EINVAL
    assert expect in _last(L), _last(L)


@pytest.mark.parametrize("case, expect", [
    ("null_out", "batch pointer is null"),
    ("count0", "count must be >= 1"),
    ("nvec", "nvec = 1"),
    ("fixed_sums", "fixed_sums must be 0 or 1"),
    ("precision", "MAGNUS_FP64"),
    ("interval", "MAGNUS_INTERVAL_GERSHGORIN"),
])
def test_batch_create_rejects(L, case, expect):
    terms = (mg.Term * 2)(_xxz(), _field())
    coeffs = (mg.Coeff * 2)(_const(), _const())
    items = (mg.BatchItem * 1)(mg.BatchItem(dim=16, nterms=2, terms=terms, coeffs=coeffs))
    out = C.c_void_p(FAKE)
    opt, count, outp = None, 1, C.byref(out)
    if case == "null_out":
        outp = None
    elif case == "count0":
        count = 0
    elif case == "nvec":
        opt = _options(nvec=2)
    elif case == "fixed_sums":
        opt = _options(fixed_sums=3)
    elif case == "precision":
        opt = _options(precision=mg.FP32_SPLIT)
    elif case == "interval":
        opt = _options(interval=1)
    rc = L.magnus_batch_create(outp, count, items, C.byref(opt) if opt is not None else None, None)
    assert rc == mg.EINVAL
    assert expect in L.magnus_batch_last_error(None).decode(), L.magnus_batch_last_error(None)


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: without the compiled library the binding raises instead of computing."""
    monkeypatch.setattr(mg, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mg.load(str(tmp_path / "libmissing.so"))


def test_binding_refuses_host_tensors(L):
    """Host (CPU) or strided tensors never reach the C ABI: the binding raises before the call."""
    torch = pytest.importorskip("torch")
    v = torch.zeros(16, dtype=torch.complex128)
    with pytest.raises(TypeError, match="CUDA tensor"):
        mg.expv_xxz_static(4, J, HZ, 0.5, np.array([0.1, 0.05]), v)
    with pytest.raises(TypeError, match="CUDA tensor"):
        mg._dptr(v)
    with pytest.raises(TypeError, match="CUDA tensor"):
        mg._dptr(np.zeros(4))


def test_binding_argument_checks(L):
    """Mismatched argument counts are refused by the binding before any CUDA call."""
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError, match="2 terms but 1 drives"):
        mg.Plan(16, [mg.XXZTerm(4, J, HZ), mg.FieldXTerm(4)], [mg.Drive.const()])
    with pytest.raises(ValueError, match="2 values"):
        mg.expv_xxz_static(4, J, HZ, 0.5, np.array([0.1, 0.2, 0.3]), torch.zeros(16, dtype=torch.complex128))


def test_builders_reject_bad_sizes(L):
    """The spin-chain builders refuse out-of-range chains and null buffers before any launch."""
    assert L.magnus_xxz_nnz(1) == -1 and L.magnus_xxz_nnz(31) == -1 and L.magnus_xxz_nnz(2) == 4 + 2
    assert L.magnus_build_xxz_csr(31, _dp(J), _dp(HZ), 0.5, FAKE, FAKE, FAKE, None) == mg.EINVAL
    assert L.magnus_build_xxz_csr(4, _dp(J), _dp(HZ), 0.5, FAKE, None, FAKE, None) == mg.EINVAL
    assert "build_xxz_csr: bad argument" in _last(L)
    assert L.magnus_build_field_x_csr(0, FAKE, FAKE, FAKE, None) == mg.EINVAL
    assert L.magnus_build_longrange_dense(16, 1.5, _dp(HZ), 0.5, FAKE, None) == mg.EINVAL  # dense: <= 15 spins
    assert L.magnus_build_field_x_dense(4, None, None) == mg.EINVAL
    assert "build_field_x_dense: bad argument" in _last(L)
    assert L.magnus_batch_destroy(None) == mg.OK
