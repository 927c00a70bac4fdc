"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle on identical seeded inputs.

Tolerance: relative 2-norm error <= 1e-10 on the state, the Leja-degree sequence equal
(both sides take the same stop decisions in FP64).  Builders and index work are bit-exact.
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
    if kind == "csr_real":  # float64 value arrays (MAGNUS_TERM_CSR_REAL)
        return [mg.build_xxz_csr(n, c.J, c.hz, c.delta).as_real(), mg.build_field_x_csr(n).as_real()]
    if kind == "mfree":
        return [mg.XXZTerm(n, c.J, c.hz, c.delta), mg.FieldXTerm(n)]
    raise ValueError(kind)


def drives_gpu(mg, c):
    return [mg.Drive.const(), mg.Drive(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)]


def oracle_problem(c, tol=1e-10, **kw):
    Hs = oracle.xxz_csr(c.nspins, c.J, c.hz, c.delta)
    Hd = oracle.field_x_csr(c.nspins)
    f = oracle.Coeff(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)
    return oracle.Problem([Hs, Hd], [oracle.Coeff.const(), f], tol=tol, **kw)


# ----------------------------------------------------------------- tables
def test_leja_points_match_oracle(mg):
    c = mi.xxz_chain(1, 6, 0.01, 1)
    plan = mg.Plan(c.dim, chain_terms(mg, c, "mfree"), drives_gpu(mg, c), m_max=100)
    xi = plan.leja_points(101)
    ref = oracle.leja_points(100)
    assert np.max(np.abs(xi - ref)) < 1e-14
    assert xi[0] == 2.0 and xi[1] == -2.0 and xi[2] == 0.0


@pytest.mark.parametrize("m_max", [100, 200])
@pytest.mark.parametrize("rho", [0.0, 0.05, 0.9, 2.5, 4.0])
def test_divided_differences_match_oracle(mg, rho, m_max):
    """Both lane layouts of the device computation (4 entries per lane up to m_max 127, else 8)."""
    c = mi.xxz_chain(1, 6, 0.01, 1)
    plan = mg.Plan(c.dim, chain_terms(mg, c, "mfree"), drives_gpu(mg, c), m_max=m_max)
    d = plan.divided_differences(rho, m_max + 1)
    ref = oracle.divided_differences(oracle.leja_points(m_max), rho)
    assert np.max(np.abs(d - ref)) < 2e-15


# ----------------------------------------------------------------- builders, intervals
@pytest.mark.parametrize("n", [3, 8, 11])
def test_csr_builders_bit_exact(mg, n):
    c = mi.xxz_chain(30 + n, n, 0.01, 1)
    g = mg.build_xxz_csr(n, c.J, c.hz, c.delta)
    o = oracle.xxz_csr(n, c.J, c.hz, c.delta)
    assert np.array_equal(g.rowptr.cpu().numpy(), o.rowptr)
    assert np.array_equal(g.col.cpu().numpy(), o.col)
    assert np.max(np.abs(g.val.cpu().numpy() - o.val)) < 1e-14
    gf, of = mg.build_field_x_csr(n), oracle.field_x_csr(n)
    assert np.array_equal(gf.rowptr.cpu().numpy(), of.rowptr)
    assert np.array_equal(gf.col.cpu().numpy(), of.col)
    assert np.array_equal(gf.val.cpu().numpy(), of.val)


@pytest.mark.parametrize("n", [4, 7])
def test_dense_builders(mg, n):
    hz = np.linspace(-0.7, 0.9, n)
    g = mg.build_longrange_dense(n, hz, 1.5, 0.5).cpu().numpy()
    assert np.max(np.abs(g - oracle.longrange_dense(n, hz, 1.5, 0.5))) < 1e-13
    assert np.array_equal(mg.build_field_x_dense(n).cpu().numpy(), oracle.field_x_dense(n))


@pytest.mark.parametrize("kind", ["csr", "mfree"])
def test_gershgorin_intervals(mg, kind):
    c = mi.xxz_chain(1, 10, 0.01, 1)
    plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives_gpu(mg, c))
    P = oracle_problem(c)
    for k in range(2):
        a, b = plan.interval(k)
        ra, rb = P.interval(k)
        assert abs(a - ra) <= 1e-13 * abs(ra) and abs(b - rb) <= 1e-13 * abs(rb)


# ----------------------------------------------------------------- expv
@pytest.mark.parametrize("kind", ["csr", "mfree"])
@pytest.mark.parametrize("beta", [(0.005, 0.003), (0.05, -0.02), (3.0, -1.5), (0.0, 0.0)])
def test_expv_parity(mg, kind, beta):
    c = mi.xxz_chain(1, 10, 0.01, 1)
    plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives_gpu(mg, c))
    out, st = plan.expv(np.array(beta), cuda(c.psi0), log_cap=64)
    P = oracle_problem(c)
    ost = oracle.Stats(64)
    ref = P.expv(np.array(beta), c.psi0, ost)
    if beta == (0.0, 0.0):
        assert np.array_equal(out.cpu().numpy(), c.psi0)
        return
    assert rel(out.cpu().numpy(), ref) < REL_TOL
    assert np.array_equal(st["m_log"], ost.m_log)


# ----------------------------------------------------------------- real-valued storage
def test_real_storage_same_arithmetic_as_complex_storage(mg):
    """Real storage multiplies the same real parts in the same order as complex storage with zero
    imaginary parts, so the two propagations agree bit for bit (and with the oracle to 1e-10)."""
    c = mi.xxz_chain(23, 10, 0.01, 20)
    out = {}
    for kind in ("csr", "csr_real"):
        plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives_gpu(mg, c))
        psi = cuda(c.psi0)
        plan.propagate(psi, 0.0, c.h, c.nsteps, "CF4")
        out[kind] = psi.cpu().numpy()
    assert np.array_equal(out["csr"], out["csr_real"])
    assert rel(out["csr_real"], oracle_problem(c).propagate(c.psi0, 0.0, c.h, c.nsteps, "CF4")) < REL_TOL


def test_real_parts_rejects_complex_values(mg):
    z = torch.tensor([1.0 + 0j, 2.0 + 1e-300j], dtype=torch.complex128, device="cuda")
    with pytest.raises(mg.MagnusError) as e:
        mg.real_parts(z)
    assert e.value.code == mg.EINVAL
    r = mg.real_parts(torch.tensor([1.5 + 0j, -2.0 + 0j], dtype=torch.complex128, device="cuda"))
    assert r.dtype == torch.float64 and r.cpu().tolist() == [1.5, -2.0]


# ----------------------------------------------------------------- Lanczos enclosures
@pytest.mark.parametrize("kind", ["csr", "csr_real", "mfree"])
def test_lanczos_intervals_match_oracle(mg, kind):
    """The device Lanczos enclosure (same start vector, same recurrence, fixed-order reductions)
    against the oracle's, and against the true spectrum."""
    c = mi.xxz_chain(26, 10, 0.01, 1)
    plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives_gpu(mg, c), interval="lanczos")
    P = oracle_problem(c, interval="lanczos")
    Hs = oracle.xxz_csr(c.nspins, c.J, c.hz, c.delta)
    ev = np.linalg.eigvalsh(Hs.todense())
    for k in range(2):
        a, b = plan.interval(k)
        ra, rb = P.interval(k)
        assert abs(a - ra) < 1e-8 * (rb - ra) and abs(b - rb) < 1e-8 * (rb - ra), (k, a, b, ra, rb)
    a, b = plan.interval(0)
    assert a <= ev[0] + 1e-11 and ev[-1] - 1e-11 <= b


def test_lanczos_intervals_dense(mg):
    c = mi.workload3(nvec=1, nspins=8, h=0.02, nsteps=2)
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    plan = mg.Plan(c.dim, [mg.DenseTerm(Hs), mg.FieldXTerm(c.nspins)], drives_gpu(mg, c), interval="lanczos")
    Ho = oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    P = oracle.Problem([Ho, oracle.field_x_csr(c.nspins)], [oracle.Coeff.const()] * 2, interval="lanczos")
    a, b = plan.interval(0)
    ra, rb = P.interval(0)
    assert abs(a - ra) < 1e-8 * (rb - ra) and abs(b - rb) < 1e-8 * (rb - ra)
    ev = np.linalg.eigvalsh(Ho)
    assert a <= ev[0] + 1e-11 and ev[-1] - 1e-11 <= b


@pytest.mark.parametrize("variant", ["CF4", "M4"])
def test_lanczos_propagation_matches_oracle(mg, variant):
    """Propagation on Lanczos enclosures: same state (1e-10) and Leja degrees as the oracle on its
    own Lanczos enclosures, and fewer matvecs than on Gershgorin enclosures."""
    c = mi.workload1()
    plan = mg.Plan(c.dim, chain_terms(mg, c, "csr"), drives_gpu(mg, c), interval="lanczos")
    psi = cuda(c.psi0)
    st = plan.propagate(psi, c.t0, c.h, c.nsteps, variant, log_cap=512)
    ost = oracle.Stats(512)
    ref = oracle_problem(c, interval="lanczos").propagate(c.psi0, c.t0, c.h, c.nsteps, variant, ost)
    assert np.array_equal(st["m_log"], ost.m_log)
    assert rel(psi.cpu().numpy(), ref) < REL_TOL
    g = mg.Plan(c.dim, chain_terms(mg, c, "csr"), drives_gpu(mg, c)).propagate(cuda(c.psi0), c.t0, c.h, c.nsteps, variant)
    assert st["n_matvec"] < g["n_matvec"]


# ----------------------------------------------------------------- propagation, workload 1
@pytest.mark.parametrize("kind", ["csr", "csr_real", "mfree"])
@pytest.mark.parametrize("variant", ["CF4", "M4"])
def test_propagate_workload1(mg, kind, variant):
    c = mi.workload1()
    plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives_gpu(mg, c))
    psi = cuda(c.psi0)
    st = plan.propagate(psi, c.t0, c.h, c.nsteps, variant, log_cap=512)
    ost = oracle.Stats(512)
    ref = oracle_problem(c).propagate(c.psi0, c.t0, c.h, c.nsteps, variant, ost)
    assert st["n_exp"] == ost.n_exp and st["n_substeps"] == ost.n_substeps
    assert np.array_equal(st["m_log"], ost.m_log)
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


@pytest.mark.parametrize("kind", ["csr", "csr_real"])
@pytest.mark.parametrize("variant", ["CF4_3", "M2"])
def test_propagate_other_methods(mg, variant, kind):
    c = mi.xxz_chain(21, 9, 0.02, 30)
    plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives_gpu(mg, c))
    psi = cuda(c.psi0)
    plan.propagate(psi, 0.1, c.h, c.nsteps, variant)
    ref = oracle_problem(c).propagate(c.psi0, 0.1, c.h, c.nsteps, variant)
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


@pytest.mark.parametrize("kind", ["csr", "csr_real", "mfree"])
def test_propagate_m6(mg, kind):
    """Method M6 (nested commutators applied matrix-free in five passes) against the oracle."""
    c = mi.workload1()
    plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives_gpu(mg, c))
    psi = cuda(c.psi0)
    st = plan.propagate(psi, c.t0, c.h, 40, "M6", log_cap=512)
    ost = oracle.Stats(512)
    ref = oracle_problem(c).propagate(c.psi0, c.t0, c.h, 40, "M6", ost)
    assert st["n_exp"] == ost.n_exp and st["n_substeps"] == ost.n_substeps
    assert np.array_equal(st["m_log"], ost.m_log)
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


def _sum_sz_csr(n):
    """sum_i sigma^z_i as a diagonal CSR term (spin 1 the most significant bit: z_i = 1 - 2 b_i)."""
    D = 1 << n
    r = np.arange(D)
    z = sum(1 - 2 * ((r >> (n - i)) & 1) for i in range(1, n + 1)).astype(np.float64)
    return np.arange(D + 1, dtype=np.int64), r.astype(np.int32), z


@pytest.mark.parametrize("kind", ["csr", "mixed"])
def test_propagate_m6_two_independent_drives(mg, kind):
    """Method M6 with three terms, H(t) = H_s + f(t) sum_i sx_i + g(t) sum_i sz_i, f != g: with two
    independently driven terms [B_2, B_3] no longer vanishes, so the sign and weight of every nested
    commutator in U and V reach the result (Sec. 2, Method M6).  CSR terms (FAM_CSR) and the
    matrix-free chain and field beside a CSR sum_i sz_i (generic family), 10 spins, 30 steps of
    h = 0.02, against the oracle at 1e-10 with identical Leja degrees."""
    c = mi.xxz_chain(26, 10, 0.02, 30)
    n = c.nspins
    zr, zc, zv = _sum_sz_csr(n)
    f = (c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)
    g = (0.3, np.array([0.0]), np.array([0.8]), np.array([3.0]))  # 0.3 + 0.8 sin(3t)
    if kind == "csr":
        terms = [mg.build_xxz_csr(n, c.J, c.hz, c.delta), mg.build_field_x_csr(n)]
    else:
        terms = [mg.XXZTerm(n, c.J, c.hz, c.delta), mg.FieldXTerm(n)]
    terms.append(mg.CSRTerm(cuda(zr), cuda(zc), cuda(zv.astype(np.complex128))))
    plan = mg.Plan(c.dim, terms, [mg.Drive.const(), mg.Drive(*f), mg.Drive(*g)])
    psi = cuda(c.psi0)
    st = plan.propagate(psi, 0.0, c.h, c.nsteps, "M6", log_cap=512)
    P = oracle.Problem([oracle.xxz_csr(n, c.J, c.hz, c.delta), oracle.field_x_csr(n),
                        oracle.CSR(zr, zc, zv.astype(np.complex128))],
                       [oracle.Coeff.const(), oracle.Coeff(*f), oracle.Coeff(*g)])
    ost = oracle.Stats(512)
    ref = P.propagate(c.psi0, 0.0, c.h, c.nsteps, "M6", ost)
    assert np.array_equal(st["m_log"], ost.m_log)
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


def test_m6_many_vectors_ragged_blocks(mg):
    """M6 with 3 state vectors over 7 blocks of 256 rows (2^11 rows: several tiles, ragged tail),
    large steps so that substepping (s > 1) occurs."""
    c = mi.xxz_chain(24, 11, 0.3, 4, nvec=3)
    for kind in ("csr", "mfree"):
        plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives_gpu(mg, c), nvec=3, ctas=7)
        psi = cuda(c.psi0)
        st = plan.propagate(psi, 0.0, c.h, c.nsteps, "M6")
        out = psi.cpu().numpy().reshape(3, -1)
        P = oracle_problem(c)
        for v in range(3):
            ref = P.propagate(c.psi0.reshape(3, -1)[v], 0.0, c.h, c.nsteps, "M6")
            assert rel(out[v], ref) < REL_TOL, (kind, v)
        assert st["n_substeps"] > 3 * st["n_exp"]  # some exponential took more than one substep


def test_m6_rejected_where_not_supported(mg):
    c = mi.xxz_chain(25, 7, 0.01, 2)
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    plan = mg.Plan(c.dim, [mg.DenseTerm(Hs), mg.FieldXTerm(c.nspins)], drives_gpu(mg, c))
    with pytest.raises(mg.MagnusError) as e:
        plan.propagate(cuda(c.psi0), 0.0, 0.01, 1, "M6")
    assert e.value.code == mg.EINVAL
    B = mg.Batch([(c.dim, chain_terms(mg, c, "csr"), drives_gpu(mg, c))])
    with pytest.raises(mg.MagnusError) as e:
        B.propagate([cuda(c.psi0)], 0.0, 0.01, 1, "M6")
    assert e.value.code == mg.EINVAL


@pytest.mark.parametrize("ctas", [1, 3, 7, 64])
def test_ragged_block_partitions(mg, ctas):
    """Many tiles and a ragged tail: 2^11 rows over ctas blocks of 256 threads."""
    c = mi.xxz_chain(22, 11, 0.01, 10)
    for kind in ("csr", "csr_real", "mfree"):
        plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives_gpu(mg, c), ctas=ctas)
        psi = cuda(c.psi0)
        plan.propagate(psi, 0.0, c.h, c.nsteps, "M4")
        ref = oracle_problem(c).propagate(c.psi0, 0.0, c.h, c.nsteps, "M4")
        assert rel(psi.cpu().numpy(), ref) < REL_TOL


def test_multiple_vectors(mg):
    c = mi.xxz_chain(23, 8, 0.01, 20, nvec=5)
    plan = mg.Plan(c.dim, chain_terms(mg, c, "csr"), drives_gpu(mg, c), nvec=5)
    psi = cuda(c.psi0)
    st = plan.propagate(psi, 0.0, c.h, c.nsteps, "CF4", log_cap=4096)
    P = oracle_problem(c)
    out = psi.cpu().numpy()
    for v in range(5):
        ost = oracle.Stats(4096)
        ref = P.propagate(c.psi0[v], 0.0, c.h, c.nsteps, "CF4", ost)
        assert rel(out[v], ref) < REL_TOL
        assert np.array_equal(st["m_log"].reshape(-1, 5)[:, v], ost.m_log)


def test_smallest_chain_and_zero_steps(mg):
    c = mi.xxz_chain(24, 2, 0.05, 10)
    plan = mg.Plan(c.dim, chain_terms(mg, c, "csr"), drives_gpu(mg, c))
    psi = cuda(c.psi0)
    st = plan.propagate(psi, 0.0, c.h, 0, "CF4")
    assert st["n_exp"] == 0 and np.array_equal(psi.cpu().numpy(), c.psi0)
    plan.propagate(psi, 0.0, c.h, c.nsteps, "CF4")
    ref = oracle_problem(c).propagate(c.psi0, 0.0, c.h, c.nsteps, "CF4")
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


def test_norm_conservation_tight_tolerance(mg):
    c = mi.xxz_chain(25, 12, 0.01, 100)
    plan = mg.Plan(c.dim, chain_terms(mg, c, "mfree"), drives_gpu(mg, c), tol=1e-13)
    psi = cuda(c.psi0)
    plan.propagate(psi, 0.0, c.h, c.nsteps, "CF4")
    assert abs(np.linalg.norm(psi.cpu().numpy()) - 1.0) < 1e-12


def test_errors_are_reported(mg):
    c = mi.xxz_chain(26, 8, 0.01, 1)
    plan = mg.Plan(c.dim, chain_terms(mg, c, "csr"), drives_gpu(mg, c), m_max=3)
    with pytest.raises(mg.MagnusError) as e:
        plan.expv(np.array([2.0, 1.0]), cuda(c.psi0))
    assert e.value.code == mg.ENOCONV
    with pytest.raises(mg.MagnusError) as e:
        plan.propagate(cuda(c.psi0), 0.0, 0.01, 1, 99)
    assert e.value.code == mg.EINVAL
    with pytest.raises(mg.MagnusError) as e:
        mg.Plan(1000, [mg.FieldXTerm(10)], [mg.Drive.const()])  # dim is not 2^nspins
    assert e.value.code == mg.EINVAL
    # the plan is still usable after an error
    plan2 = mg.Plan(c.dim, chain_terms(mg, c, "csr"), drives_gpu(mg, c))
    psi = cuda(c.psi0)
    plan2.propagate(psi, 0.0, 0.01, 2, "CF4")
    ref = oracle_problem(c).propagate(c.psi0, 0.0, 0.01, 2, "CF4")
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


# ----------------------------------------------------------------- workload 2 at full size
@pytest.fixture(scope="module")
def wl2():
    c = mi.workload2()
    return c, {}, {}


@pytest.mark.parametrize("interval", ["gershgorin", "lanczos"])
@pytest.mark.parametrize("kind", ["csr", "mfree"])
@pytest.mark.parametrize("variant", ["CF4", "M4"])
def test_workload2_full_size_first_steps(mg, wl2, kind, variant, interval):
    """20 spins (dim 2^20) in the bench's launch configuration: the first 2 steps against the oracle,
    every entry compared, on either enclosure."""
    c, problems, cache = wl2
    if interval not in problems:
        problems[interval] = oracle_problem(c, interval=interval)
    plan = mg.Plan(c.dim, chain_terms(mg, c, kind), drives_gpu(mg, c), interval=interval)
    psi = cuda(c.psi0)
    st = plan.propagate(psi, 0.0, c.h, 2, variant, log_cap=16)
    if (variant, interval) not in cache:
        ost = oracle.Stats(16)
        cache[(variant, interval)] = (problems[interval].propagate(c.psi0, 0.0, c.h, 2, variant, ost), ost.m_log)
    ref, mlog = cache[(variant, interval)]
    assert np.array_equal(st["m_log"], mlog)
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


def test_barrier_timeout_is_reported_and_context_survives(mg):
    """A grid-barrier wait that nothing satisfies (CTA 0 leaves before arriving) runs out after the
    plan's short limit; the call returns MAGNUS_ETIMEOUT and the next plan runs normally."""
    c = mi.xxz_chain(27, 12, 0.01, 4)
    plan = mg.Plan(c.dim, chain_terms(mg, c, "csr"), drives_gpu(mg, c), ctas=8, barrier_timeout_s=0.05,
                   test_skip_arrival=1)
    with pytest.raises(mg.MagnusError) as e:
        plan.propagate(cuda(c.psi0), 0.0, c.h, c.nsteps, "CF4")
    assert e.value.code == mg.ETIMEOUT
    plan.close()
    ok = mg.Plan(c.dim, chain_terms(mg, c, "csr"), drives_gpu(mg, c), ctas=8)
    psi = cuda(c.psi0)
    ok.propagate(psi, 0.0, c.h, c.nsteps, "CF4")
    ref = oracle_problem(c).propagate(c.psi0, 0.0, c.h, c.nsteps, "CF4")
    assert rel(psi.cpu().numpy(), ref) < REL_TOL


# ----------------------------------------------------------------- the generator matvec alone
@pytest.mark.parametrize("kind", ["csr", "csr_real", "mfree", "dense"])
def test_apply_matches_oracle_terms(mg, kind):
    """magnus_apply: y = sum_k beta_k H_k x for 3 states against the oracle's term products."""
    c = mi.xxz_chain(28, 9, 0.01, 1, nvec=3)
    if kind == "dense":
        Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
        terms = [mg.DenseTerm(Hs), mg.FieldXTerm(c.nspins)]
        P = oracle.Problem([oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta), oracle.field_x_csr(c.nspins)],
                           [oracle.Coeff.const()] * 2)
    else:
        terms = chain_terms(mg, c, kind)
        P = oracle_problem(c)
    plan = mg.Plan(c.dim, terms, drives_gpu(mg, c), nvec=3)
    beta = np.array([0.7, -1.3])
    x = cuda(c.psi0)
    y = plan.apply(beta, x).cpu().numpy().reshape(3, -1)
    for v in range(3):
        xv = c.psi0.reshape(3, -1)[v]
        ref = beta[0] * P.apply_term(0, xv) + beta[1] * P.apply_term(1, xv)
        assert rel(y[v], ref) < 1e-13, (kind, v, rel(y[v], ref))


# ----------------------------------------------------------------- general matrices
def _random_hermitian_csr(rng, D, density, complex_values=True):
    """Random sparse Hermitian matrix with a ragged row-length mix (some rows hold only the diagonal)."""
    A = np.zeros((D, D), dtype=np.complex128)
    mask = rng.random((D, D)) < density
    vals = rng.standard_normal((D, D)) + (1j * rng.standard_normal((D, D)) if complex_values else 0.0)
    A[mask] = vals[mask]
    A = (A + A.conj().T) / 2
    A[np.diag_indices(D)] = rng.uniform(-2, 2, D)
    rows, cols = np.nonzero(A)
    rowptr = np.zeros(D + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return oracle.CSR(rowptr, cols.astype(np.int32), A[rows, cols]), A


@pytest.mark.parametrize("interval", ["gershgorin", "lanczos"])
def test_general_complex_csr_odd_dimension(mg, interval):
    """A complex Hermitian CSR term (complex products, no real-value path) plus a real one, dim 1003
    (not a multiple of the warp or block), 2 states, Cf4 and M4, against the oracle."""
    rng = np.random.default_rng(29)
    D = 1003
    H1, _ = _random_hermitian_csr(rng, D, 0.004, complex_values=True)
    H2, _ = _random_hermitian_csr(rng, D, 0.002, complex_values=False)
    psi0 = np.stack([mi.random_state(rng, D), mi.random_state(rng, D)])
    f = oracle.Coeff(0.2, [1.0], [0.3], [4.0])
    P = oracle.Problem([H1, H2], [oracle.Coeff.const(), f], interval=interval)
    terms = [mg.CSRTerm(cuda(H.rowptr), cuda(H.col), cuda(H.val)) for H in (H1, H2)]
    plan = mg.Plan(D, terms, [mg.Drive.const(), mg.Drive(0.2, [1.0], [0.3], [4.0])], nvec=2, interval=interval)
    for k in range(2):
        a, b = plan.interval(k)
        ra, rb = P.interval(k)
        assert abs(a - ra) < 1e-8 * (rb - ra) and abs(b - rb) < 1e-8 * (rb - ra)
    for variant in ("CF4", "M4"):
        psi = cuda(psi0)
        plan.propagate(psi, 0.0, 0.05, 10, variant)
        out = psi.cpu().numpy()
        for v in range(2):
            ref = P.propagate(psi0[v], 0.0, 0.05, 10, variant)
            assert rel(out[v], ref) < REL_TOL, (variant, v, rel(out[v], ref))


def test_general_complex_dense_odd_dimension(mg):
    """A complex Hermitian dense term (complex FP64 tile path), dim 200, 3 states, against the oracle."""
    rng = np.random.default_rng(30)
    D = 200
    A = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    A = (A + A.conj().T) / 4
    B = rng.standard_normal((D, D))
    B = ((B + B.T) / 4).astype(np.complex128)
    psi0 = np.stack([mi.random_state(rng, D) for _ in range(3)])
    f = oracle.Coeff(0.0, [1.0], [], [3.0])
    P = oracle.Problem([A, B], [oracle.Coeff.const(), f])
    plan = mg.Plan(D, [mg.DenseTerm(cuda(A)), mg.DenseTerm(cuda(B))], [mg.Drive.const(), mg.Drive(0.0, [1.0], [], [3.0])],
                   nvec=3)
    psi = cuda(psi0)
    plan.propagate(psi, 0.0, 0.02, 8, "CF4")
    out = psi.cpu().numpy()
    for v in range(3):
        assert rel(out[v], P.propagate(psi0[v], 0.0, 0.02, 8, "CF4")) < REL_TOL
