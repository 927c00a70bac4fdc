"""Exact fixed-point sums of pattern terms (options.fixed_sums) against the FP64 CPU oracle.

A pattern term stores one value on every entry (the transverse field sum_i sx_i, adjacency
patterns); with fixed_sums its row sums run in 64-bit integers on a fixed-point copy of each Leja
vector, scaled from a bound on the vector's largest component.  The method's result is unchanged:
the same tolerance as every other parity test (relative 2-norm error <= 1e-10, identical Leja
degrees), with the FP64 sums (fixed_sums=False) checked the same way beside it.
"""
import numpy as np
import pytest

import magnus_inputs as mi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-10


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_06483_gb300 as m
    m.load()
    return m


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def chain_terms(mg, c, kind):
    n = c.nspins
    if kind == "csr":
        return [mg.build_xxz_csr(n, c.J, c.hz, c.delta), mg.build_field_x_csr(n)]
    if kind == "csr_real":
        return [mg.build_xxz_csr(n, c.J, c.hz, c.delta).as_real(), mg.build_field_x_csr(n).as_real()]
    return [mg.XXZTerm(n, c.J, c.hz, c.delta), mg.FieldXTerm(n)]


def drives(mg, c):
    return [mg.Drive.const(), mg.Drive(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)]


def chain_problem(c, **kw):
    return oracle.Problem([oracle.xxz_csr(c.nspins, c.J, c.hz, c.delta), oracle.field_x_csr(c.nspins)],
                          [oracle.Coeff.const(), oracle.Coeff(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)], **kw)


@pytest.mark.parametrize("kind", ["csr", "csr_real", "mfree"])
@pytest.mark.parametrize("variant", ["CF4", "CF4_3", "M2", "M4"])
def test_fixed_and_fp64_sums_match_oracle(mg, kind, variant):
    c = mi.xxz_chain(41, 11, 0.01, 30)
    ost = oracle.Stats(512)
    ref = chain_problem(c).propagate(c.psi0, 0.0, c.h, c.nsteps, variant, ost)
    out = {}
    for fixed in (True, False):
        plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives(mg, c), fixed_sums=fixed)
        psi = cuda(c.psi0)
        st = plan.propagate(psi, 0.0, c.h, c.nsteps, variant, log_cap=512)
        assert st["fixed_sums"] == int(fixed)
        assert np.array_equal(st["m_log"], ost.m_log)
        out[fixed] = psi.cpu().numpy()
        assert rel(out[fixed], ref) < REL_TOL, (fixed, rel(out[fixed], ref))
    # both summations are FP64-accurate: they differ by rounding only
    assert rel(out[True], out[False]) < 1e-12


@pytest.mark.parametrize("kind", ["csr", "mfree"])
def test_methods_in_turn_on_one_plan(mg, kind):
    """M6 (FP64 sums), then M4 and Cf4 (fixed point) on one plan: each call scales its fixed-point
    copies from the maxima the previous call left."""
    c = mi.xxz_chain(42, 10, 0.01, 12)
    plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives(mg, c))
    P = chain_problem(c)
    psi = cuda(c.psi0)
    assert plan.propagate(psi, 0.0, c.h, 4, "M6")["fixed_sums"] == 0
    assert plan.propagate(psi, 4 * c.h, c.h, 4, "M4")["fixed_sums"] == 1
    assert plan.propagate(psi, 8 * c.h, c.h, 4, "CF4")["fixed_sums"] == 1
    ref = P.propagate(c.psi0, 0.0, c.h, 4, "M6")
    ref = P.propagate(ref, 4 * c.h, c.h, 4, "M4")
    ref = P.propagate(ref, 8 * c.h, c.h, 4, "CF4")
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


@pytest.mark.parametrize("kind", ["csr", "mfree"])
def test_wide_dynamic_range_state(mg, kind):
    """Components spread over 250 decades: the fixed-point copy resolves the large ones to 2^-55 of
    the largest and the tiny ones to zero, which leaves the norm-wise error at the FP64 level."""
    c = mi.xxz_chain(43, 10, 0.01, 10)
    rng = np.random.default_rng(431)
    psi0 = c.psi0 * 10.0 ** (-rng.integers(0, 250, c.dim))
    psi0 /= np.linalg.norm(psi0)
    ref = chain_problem(c).propagate(psi0, 0.0, c.h, c.nsteps, "CF4")
    plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives(mg, c))
    psi = cuda(psi0)
    plan.propagate(psi, 0.0, c.h, c.nsteps, "CF4")
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


@pytest.mark.parametrize("kind", ["csr", "mfree"])
def test_zero_state_stays_zero(mg, kind):
    c = mi.xxz_chain(44, 8, 0.01, 4)
    plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives(mg, c))
    psi = torch.zeros(c.dim, dtype=torch.complex128, device="cuda")
    st = plan.propagate(psi, 0.0, c.h, c.nsteps, "CF4")
    assert st["fixed_sums"] == 1
    assert not torch.any(psi != 0)


def _pattern_csr(rng, D, value, max_degree):
    """Symmetric pattern with ragged rows (empty ones included, the longest max_degree entries),
    every stored value `value`."""
    deg = rng.integers(0, max_degree // 4 + 1, D)
    A = np.zeros((D, D), dtype=bool)
    for r in range(D):
        A[r, rng.choice(D, deg[r], replace=False)] = True
    A = A | A.T
    np.fill_diagonal(A, False)
    empty = rng.choice(D, D // 20, replace=False)
    rest = np.setdiff1d(np.arange(D), empty)
    heavy = int(rng.choice(rest))
    A[empty, :] = A[:, empty] = False
    A[heavy, :] = A[:, heavy] = False
    others = rng.choice(np.setdiff1d(rest, [heavy]), max_degree, replace=False)
    A[heavy, others] = A[others, heavy] = True
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(D + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cols.astype(np.int32), np.full(rows.size, value)


def _hermitian_csr(rng, D, density):
    A = np.zeros((D, D), dtype=np.complex128)
    mask = rng.random((D, D)) < density
    A[mask] = rng.standard_normal(mask.sum()) + 1j * rng.standard_normal(mask.sum())
    A = (A + A.conj().T) / 2
    A[np.diag_indices(D)] = rng.uniform(-2, 2, D)
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(D + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32), A[rows, cols]


@pytest.mark.parametrize("storage", ["complex", "real"])
def test_ragged_pattern_with_complex_term_odd_dimension(mg, storage):
    """A pattern term of value 0.7 (rows of 0 to 70 entries) beside a complex Hermitian term, dim
    1003, 2 states: the pattern is detected, its sums run in fixed point with the complex-term bound."""
    rng = np.random.default_rng(45)
    D = 1003
    prow, pcol, pval = _pattern_csr(rng, D, 0.7, 70)
    assert np.diff(prow).max() == 70 and np.diff(prow).min() == 0
    hrow, hcol, hval = _hermitian_csr(rng, D, 0.004)
    psi0 = np.stack([mi.random_state(rng, D), mi.random_state(rng, D)])
    f = oracle.Coeff(0.2, [1.0], [0.3], [4.0])
    P = oracle.Problem([oracle.CSR(hrow, hcol, hval), oracle.CSR(prow, pcol, pval.astype(np.complex128))],
                       [oracle.Coeff.const(), f])
    pv = cuda(pval) if storage == "real" else cuda(pval.astype(np.complex128))
    terms = [mg.CSRTerm(cuda(hrow), cuda(hcol), cuda(hval)), mg.CSRTerm(cuda(prow), cuda(pcol), pv)]
    plan = mg.Plan(D, terms, [mg.Drive.const(), mg.Drive(0.2, [1.0], [0.3], [4.0])], nvec=2)
    for variant in ("CF4", "M4"):
        psi = cuda(psi0)
        st = plan.propagate(psi, 0.0, 0.05, 10, variant)
        assert st["fixed_sums"] == 1
        out = psi.cpu().numpy()
        for v in range(2):
            ref = P.propagate(psi0[v], 0.0, 0.05, 10, variant)
            assert rel(out[v], ref) < REL_TOL, (variant, v, rel(out[v], ref))


def test_no_pattern_term_means_fp64_sums(mg):
    """A plan whose CSR terms all carry varying values has nothing to sum in fixed point."""
    rng = np.random.default_rng(46)
    D = 300
    h1 = _hermitian_csr(rng, D, 0.01)
    h2 = _hermitian_csr(rng, D, 0.01)
    terms = [mg.CSRTerm(cuda(r), cuda(c), cuda(v)) for r, c, v in (h1, h2)]
    plan = mg.Plan(D, terms, [mg.Drive.const(), mg.Drive(0.0, [1.0], [], [2.0])])
    psi = cuda(mi.random_state(rng, D))
    st = plan.propagate(psi, 0.0, 0.05, 2, "CF4")
    assert st["fixed_sums"] == 0


def _banded_csr(rng, D, wmin, wmax, value=None):
    """Real symmetric banded matrix, half-bandwidth w_r ~ U{wmin..wmax} per row (ragged rows of
    moderate spread), all values `value` if given."""
    A = np.zeros((D, D))
    for r in range(D):
        w = int(rng.integers(wmin, wmax + 1))
        for c in range(max(0, r - w), min(D, r + w + 1)):
            A[r, c] = A[c, r] = rng.uniform(-1, 1) if value is None else value
    if value is None:
        A[np.diag_indices(D)] = rng.uniform(-2, 2, D)
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(D + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32), A[rows, cols]


@pytest.mark.parametrize("D", [1003, 4096])
def test_ragged_banded_rows_odd_and_even_dimension(mg, D):
    """A real banded term (rows of 5 to 13 entries: the warp-uniform trip count pads every lane to
    its warp's longest row) and a ragged banded pattern term of value 0.5 (row pointers loaded), with
    a partial last warp for dim 1003."""
    rng = np.random.default_rng(47 + D)
    h1 = _banded_csr(rng, D, 2, 6)
    h2 = _banded_csr(rng, D, 1, 3, value=0.5)
    psi0 = mi.random_state(rng, D)
    f = oracle.Coeff(0.3, [1.0], [], [2.5])
    P = oracle.Problem([oracle.CSR(r, c, v.astype(np.complex128)) for r, c, v in (h1, h2)], [oracle.Coeff.const(), f])
    terms = [mg.CSRTerm(cuda(r), cuda(c), cuda(v)) for r, c, v in (h1, h2)]
    plan = mg.Plan(D, terms, [mg.Drive.const(), mg.Drive(0.3, [1.0], [], [2.5])])
    ost = oracle.Stats(256)
    ref = P.propagate(psi0, 0.0, 0.05, 12, "CF4", ost)
    psi = cuda(psi0)
    st = plan.propagate(psi, 0.0, 0.05, 12, "CF4", log_cap=256)
    assert st["fixed_sums"] == 1
    assert np.array_equal(st["m_log"], ost.m_log)
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


def _random_real_csr(rng, D, density, decades):
    """Real symmetric CSR with values of random sign spread over 2 x decades decades around 1, some
    rows empty (the diagonal too)."""
    A = np.zeros((D, D))
    mask = rng.random((D, D)) < density
    A[mask] = rng.choice([-1.0, 1.0], mask.sum()) * 10.0 ** rng.uniform(-decades, decades, mask.sum())
    A = (A + A.T) / 2
    empty = rng.choice(D, D // 25, replace=False)
    A[empty, :] = 0.0
    A[:, empty] = 0.0
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(D + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32), A[rows, cols]


@pytest.mark.parametrize("decades", [0.5, 8.0])
def test_fixed_point_products_wide_value_range(mg, decades):
    """Real CSR values spread over up to 16 decades inside a row (row-scaled 62-bit mantissas times
    the fixed-point vector), beside a pattern term of value -0.3, dim 777, 2 states, against the
    oracle; with FP64 products checked the same way."""
    rng = np.random.default_rng(48 + int(decades))
    D = 777
    h1 = _random_real_csr(rng, D, 0.01, decades)
    h2 = _pattern_csr(rng, D, -0.3, 24)
    scale = 1.0 / np.max(np.abs(h1[2]))  # |H_1| <= 1 so that h = 0.05 stays a moderate step
    h1 = (h1[0], h1[1], h1[2] * scale)
    psi0 = np.stack([mi.random_state(rng, D), mi.random_state(rng, D)])
    f = oracle.Coeff(0.1, [1.0], [], [3.0])
    P = oracle.Problem([oracle.CSR(r, c, v.astype(np.complex128)) for r, c, v in (h1, h2)], [oracle.Coeff.const(), f])
    refs = [P.propagate(psi0[v], 0.0, 0.05, 10, "CF4") for v in range(2)]
    for fixed in (True, False):
        terms = [mg.CSRTerm(cuda(r), cuda(c), cuda(v)) for r, c, v in (h1, h2)]
        plan = mg.Plan(D, terms, [mg.Drive.const(), mg.Drive(0.1, [1.0], [], [3.0])], nvec=2, fixed_sums=fixed)
        psi = cuda(psi0)
        st = plan.propagate(psi, 0.0, 0.05, 10, "CF4")
        assert st["fixed_sums"] == int(fixed)
        out = psi.cpu().numpy()
        for v in range(2):
            assert rel(out[v], refs[v]) < REL_TOL, (fixed, v, rel(out[v], refs[v]))


def test_values_beyond_the_fixed_point_range_keep_fp64_products(mg):
    """Values near 1e121 (row exponents beyond the range the scales cover) keep FP64 products; the
    step h = 1e-121 keeps the exponentials moderate.  The pattern term still sums in fixed point."""
    rng = np.random.default_rng(49)
    D = 300
    h1 = _banded_csr(rng, D, 1, 3)
    h1 = (h1[0], h1[1], h1[2] * 1e121)
    h2 = _pattern_csr(rng, D, 1.0, 12)
    psi0 = mi.random_state(rng, D)
    f = oracle.Coeff(0.0, [1e121], [], [1e120])
    P = oracle.Problem([oracle.CSR(r, c, v.astype(np.complex128)) for r, c, v in (h1, h2)], [oracle.Coeff.const(), f])
    ref = P.propagate(psi0, 0.0, 1e-121, 6, "CF4")
    terms = [mg.CSRTerm(cuda(r), cuda(c), cuda(v)) for r, c, v in (h1, h2)]
    plan = mg.Plan(D, terms, [mg.Drive.const(), mg.Drive(0.0, [1e121], [], [1e120])])
    psi = cuda(psi0)
    st = plan.propagate(psi, 0.0, 1e-121, 6, "CF4")
    assert st["fixed_sums"] == 1
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


@pytest.mark.parametrize("kind", ["csr", "mfree"])
@pytest.mark.parametrize("variant", ["CF4", "M4"])
def test_many_vectors_each_with_its_own_scales(mg, kind, variant):
    """5 states of very different size (1e-6 to 1e6) in one plan: every state has its own
    fixed-point scales and maxima; each against the oracle with its own Leja degrees."""
    c = mi.xxz_chain(50, 9, 0.01, 12, nvec=5)
    psi0 = c.psi0 * (10.0 ** np.arange(-6, 7, 3))[:, None]
    plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives(mg, c), nvec=5)
    psi = cuda(psi0)
    st = plan.propagate(psi, 0.0, c.h, c.nsteps, variant, log_cap=4096)
    assert st["fixed_sums"] == 1
    out = psi.cpu().numpy()
    P = chain_problem(c)
    for v in range(5):
        ost = oracle.Stats(4096)
        ref = P.propagate(psi0[v], 0.0, c.h, c.nsteps, variant, ost)
        assert rel(out[v], ref) < REL_TOL, (v, rel(out[v], ref))
        assert np.array_equal(st["m_log"].reshape(-1, 5)[:, v], ost.m_log)


@pytest.mark.parametrize("ctas", [1, 3, 7])
def test_ragged_block_partitions_fixed_point(mg, ctas):
    """2^11 rows over a few blocks (partial warps at the block ends): Cf4 and M4 in fixed point."""
    c = mi.xxz_chain(51, 11, 0.01, 8)
    for kind in ("csr", "mfree"):
        plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives(mg, c), ctas=ctas)
        for variant in ("CF4", "M4"):
            psi = cuda(c.psi0)
            assert plan.propagate(psi, 0.0, c.h, c.nsteps, variant)["fixed_sums"] == 1
            ref = chain_problem(c).propagate(c.psi0, 0.0, c.h, c.nsteps, variant)
            assert rel(psi.cpu().numpy(), ref) < REL_TOL, (kind, variant)


# ----------------------------------------------------------------- the generator matvec alone
def rel_scaled(a, b):
    """rel() after dividing both by max |b|, so that vectors near the ends of the double range do
    not overflow or underflow inside the norms."""
    s = np.max(np.abs(b))
    return rel(a / s, b / s)


@pytest.mark.parametrize("kind", ["csr", "csr_real", "mfree"])
def test_apply_fixed_point_any_magnitude(mg, kind):
    """magnus_apply in fixed point: states of size 1e-290, 1e-3, 1e5 and 1e290 (each with its own
    scale; the copy keeps its full width at both ends of the double range) and a zero state, against
    the oracle's term products and beside the FP64 matvec."""
    c = mi.xxz_chain(52, 10, 0.01, 1, nvec=5)
    x0 = c.psi0 * np.array([1e-290, 1e-3, 1e5, 1e290, 0.0])[:, None]
    beta = np.array([0.7, -1.3])
    ys = {}
    for fixed in (True, False):
        plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives(mg, c), nvec=5, fixed_sums=fixed)
        ys[fixed] = plan.apply(beta, cuda(x0)).cpu().numpy()
        plan.close()
    P = chain_problem(c)
    for v in range(4):
        ref = beta[0] * P.apply_term(0, x0[v]) + beta[1] * P.apply_term(1, x0[v])
        for fixed in (True, False):
            assert rel_scaled(ys[fixed][v], ref) < 1e-13, (fixed, v, rel_scaled(ys[fixed][v], ref))
    assert not np.any(ys[True][4] != 0)


@pytest.mark.parametrize("kind", ["csr", "mfree"])
def test_apply_fixed_point_nonfinite_state_takes_fp64_rows(mg, kind):
    """A state holding an Inf and a NaN: its rows run in FP64 and give the FP64 matvec's non-finite
    entries; the finite state beside it keeps the fixed-point rows."""
    c = mi.xxz_chain(53, 9, 0.01, 1, nvec=2)
    x0 = c.psi0.copy()
    x0[0, 17] = np.inf
    x0[0, 300] = complex(0.0, np.nan)
    beta = np.array([0.9, 0.4])
    ys = {}
    for fixed in (True, False):
        plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives(mg, c), nvec=2, fixed_sums=fixed)
        ys[fixed] = plan.apply(beta, cuda(x0)).cpu().numpy()
        plan.close()
    for part in (np.real, np.imag):
        a, b = part(ys[True][0]), part(ys[False][0])
        assert np.array_equal(np.isnan(a), np.isnan(b))
        assert np.array_equal(np.isinf(a), np.isinf(b))
        fin = np.isfinite(b)
        assert not np.all(fin)
        assert np.allclose(a[fin], b[fin], rtol=1e-12, atol=0.0)
    P = chain_problem(c)
    ref = beta[0] * P.apply_term(0, x0[1]) + beta[1] * P.apply_term(1, x0[1])
    assert rel(ys[True][1], ref) < 1e-13


def test_apply_fixed_point_general_terms(mg):
    """magnus_apply on a ragged pattern term beside a real term whose values span 8 decades (value
    mantissas at per-row exponents) and a complex term (FP64 rows), dim 1003, 3 states."""
    rng = np.random.default_rng(531)
    D = 1003
    mats = (_pattern_csr(rng, D, -0.75, 24), _random_real_csr(rng, D, 0.01, 8), _hermitian_csr(rng, D, 0.005))
    terms = [mg.CSRTerm(cuda(r), cuda(c), cuda(v)) for r, c, v in mats]
    const = [mg.Drive.const()] * 3
    x0 = ((rng.standard_normal((3, D)) + 1j * rng.standard_normal((3, D))) *
          np.array([1e-200, 1.0, 1e200])[:, None])
    beta = np.array([1.1, -0.3, 0.6])
    ys = {}
    for fixed in (True, False):
        plan = mg.Plan(D, terms, const, nvec=3, fixed_sums=fixed)
        ys[fixed] = plan.apply(beta, cuda(x0)).cpu().numpy()
        plan.close()
    P = oracle.Problem([oracle.CSR(r, c, v.astype(np.complex128)) for r, c, v in mats], [oracle.Coeff.const()] * 3)
    for v in range(3):
        ref = sum(beta[k] * P.apply_term(k, x0[v]) for k in range(3))
        for fixed in (True, False):
            assert rel_scaled(ys[fixed][v], ref) < 1e-13, (fixed, v, rel_scaled(ys[fixed][v], ref))


# ----------------------------------------------------------------- row layouts of the fixed-point CSR rows
LAYOUTS = {"csr": 2, "staged": 1, "sliced": 3}


@pytest.mark.parametrize("nvec", [1, 3])
def test_row_layouts_bit_identical(mg, nvec):
    """The three layouts of the fixed-point CSR rows -- the CSR arrays as given, each warp's 32-row
    tiles staged in shared memory by the TMA bulk engine, and the sliced rows (column-major heads of
    32-row slices, entries reordered so that shared column offsets line up) -- read the same entries
    and sum them exactly in int64, so the three plans agree bit for bit, and match the oracle.
    12-spin chain (dim 4096, 128 slices), CF4 and CF4:3."""
    c = mi.xxz_chain(49, 12, 0.01, 12, nvec=nvec)
    P = chain_problem(c)
    for variant in ("CF4", "CF4_3"):
        out = {}
        for rows, code in LAYOUTS.items():
            plan = mg.Plan(c.dim, chain_terms(mg, c, "csr"), drives(mg, c), nvec=nvec, rows=rows)
            psi = cuda(c.psi0)
            st = plan.propagate(psi, 0.0, c.h, c.nsteps, variant, log_cap=1024)
            assert st["row_layout"] == code and st["fixed_sums"] == 1
            out[rows] = (psi.cpu().numpy(), st["m_log"])
            plan.close()
        for rows in ("staged", "sliced"):
            assert np.array_equal(out[rows][0], out["csr"][0]), rows
            assert np.array_equal(out[rows][1], out["csr"][1]), rows
        psi0 = c.psi0.reshape(nvec, -1)
        got = out["sliced"][0].reshape(nvec, -1)
        for v in range(nvec):
            ref = P.propagate(psi0[v], 0.0, c.h, c.nsteps, variant)
            assert rel(got[v], ref) < REL_TOL, (variant, v, rel(got[v], ref))


def test_sliced_rows_m4_and_apply(mg):
    """M4 (both phases on the sliced rows) and the generator matvec alone (magnus_apply) give the
    bits of the CSR layout; 11 spins, odd number of slices per block."""
    c = mi.xxz_chain(52, 11, 0.01, 10)
    res = {}
    for rows in ("csr", "sliced"):
        plan = mg.Plan(c.dim, chain_terms(mg, c, "csr"), drives(mg, c), rows=rows)
        psi = cuda(c.psi0)
        plan.propagate(psi, 0.0, c.h, c.nsteps, "M4")
        y = plan.apply(np.array([0.7, -1.3]), cuda(c.psi0))
        res[rows] = (psi.cpu().numpy(), y.cpu().numpy())
        plan.close()
    assert np.array_equal(res["csr"][0], res["sliced"][0])
    assert np.array_equal(res["csr"][1], res["sliced"][1])
    ref = chain_problem(c).propagate(c.psi0, 0.0, c.h, c.nsteps, "M4")
    assert rel(res["sliced"][0], ref) < REL_TOL


def _banded_with_heavy_band(rng, D, band, w_heavy):
    """Real symmetric banded matrix: half-bandwidth 2-6 per row, except rows [band, band + 32) with
    half-bandwidth w_heavy (their tile and its neighbours' tiles hold hundreds of entries)."""
    import scipy.sparse as sp
    rr, cc = [], []
    for r in range(D):
        w = w_heavy if band <= r < band + 32 else int(rng.integers(2, 7))
        c = np.arange(max(0, r - w), min(D, r + w + 1))
        rr.append(np.full(c.size, r))
        cc.append(c)
    rr, cc = np.concatenate(rr), np.concatenate(cc)
    A = sp.coo_matrix((rng.uniform(-1, 1, rr.size), (rr, cc)), shape=(D, D)).tocsr()
    A = ((A + A.T) / 2).tocsr()
    A.sort_indices()
    return A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64)


def _tiles_too_large(rowptrs, slot=9472):
    """32-row tiles whose runs (4 B per column, 8 B per mantissa of the first term, 16-byte blocks)
    exceed one staging slot."""
    D = rowptrs[0].size - 1
    bad = 0
    for t in range(0, D, 32):
        tot = 0
        for k, rp in enumerate(rowptrs):
            e0, e1 = int(rp[t]), int(rp[min(D, t + 32)])
            for es in ((4, 8) if k == 0 else (4,)):
                tot += ((e1 * es + 15) // 16 * 16) - (e0 * es // 16 * 16)
        bad += tot > slot
    return bad


def test_row_layouts_with_long_rows(mg):
    """A real banded term with one band of 32 rows of 81 entries beside a pattern term; dim 16384
    (512 tiles).  Staged: a few tiles do not fit a slot and are read from global memory inside the
    staged kernel.  Sliced: the rows of those slices are longer than the reordering handles (CSR
    order kept) and most of their entries sit in the tails.  Bit-identical to the CSR layout and
    within 1e-10 of the oracle, with identical Leja degrees."""
    rng = np.random.default_rng(50)
    D = 16384
    h1 = _banded_with_heavy_band(rng, D, 8000, 40)
    # pattern term: the same banded structure at half-bandwidth 1-3, value 0.5, built sparsely
    import scipy.sparse as sp
    rr, cc = [], []
    for r in range(D):
        w = int(rng.integers(1, 4))
        c = np.arange(max(0, r - w), min(D, r + w + 1))
        rr.append(np.full(c.size, r))
        cc.append(c)
    rr, cc = np.concatenate(rr), np.concatenate(cc)
    B = sp.coo_matrix((np.ones(rr.size), (rr, cc)), shape=(D, D)).tocsr()
    B = (B + B.T).tocsr()
    B.data[:] = 0.5
    B.sort_indices()
    h2 = (B.indptr.astype(np.int64), B.indices.astype(np.int32), B.data.astype(np.float64))
    bad = _tiles_too_large([h1[0], h2[0]])
    assert 1 <= bad <= D // 32 // 64, bad
    psi0 = mi.random_state(rng, D)
    f = oracle.Coeff(0.3, [1.0], [], [2.5])
    Pr = oracle.Problem([oracle.CSR(r, c, v.astype(np.complex128)) for r, c, v in (h1, h2)], [oracle.Coeff.const(), f])
    ost = oracle.Stats(256)
    ref = Pr.propagate(psi0, 0.0, 0.02, 6, "CF4", ost)
    out = {}
    for rows, code in LAYOUTS.items():
        terms = [mg.CSRTerm(cuda(r), cuda(c), cuda(v)) for r, c, v in (h1, h2)]
        plan = mg.Plan(D, terms, [mg.Drive.const(), mg.Drive(0.3, [1.0], [], [2.5])], rows=rows)
        psi = cuda(psi0)
        st = plan.propagate(psi, 0.0, 0.02, 6, "CF4", log_cap=256)
        assert st["row_layout"] == code, rows
        assert np.array_equal(st["m_log"], ost.m_log)
        out[rows] = psi.cpu().numpy()
        plan.close()
    assert np.array_equal(out["staged"], out["csr"])
    assert np.array_equal(out["sliced"], out["csr"])
    assert rel(out["sliced"], ref) < REL_TOL
