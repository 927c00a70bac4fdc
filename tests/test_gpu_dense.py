"""Dense terms on the GPU (long-range chain stored as a dense complex128 matrix) against the oracle.

Tolerance: relative 2-norm error <= 1e-10 per state vector and identical Leja degrees.
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


def drive_pair(mg, c):
    return [mg.Drive.const(), mg.Drive(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)]


def oracle_dense(c, Hs, Hd, tol=1e-10):
    f = oracle.Coeff(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)
    return oracle.Problem([Hs, Hd], [oracle.Coeff.const(), f], tol=tol)


@pytest.mark.parametrize("nvec", [1, 5])
@pytest.mark.parametrize("variant", ["CF4", "M4"])
@pytest.mark.parametrize("field", ["dense", "mfree"])
def test_longrange_dense_parity(mg, nvec, variant, field):
    c = mi.workload3(nvec=nvec, nspins=7, h=0.02, nsteps=15)
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    Hd = mg.build_field_x_dense(c.nspins) if field == "dense" else mg.FieldXTerm(c.nspins)
    terms = [mg.DenseTerm(Hs), mg.DenseTerm(Hd) if field == "dense" else Hd]
    plan = mg.Plan(c.dim, terms, drive_pair(mg, c), nvec=nvec)
    psi = cuda(c.psi0)
    st = plan.propagate(psi, 0.0, c.h, c.nsteps, variant, log_cap=4096)
    P = oracle_dense(c, oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta), oracle.field_x_dense(c.nspins))
    out = psi.cpu().numpy().reshape(nvec, -1)
    for v in range(nvec):
        ost = oracle.Stats(4096)
        ref = P.propagate(c.psi0.reshape(nvec, -1)[v], 0.0, c.h, c.nsteps, variant, ost)
        assert rel(out[v], ref) < REL_TOL, (v, rel(out[v], ref))
        assert np.array_equal(st["m_log"].reshape(-1, nvec)[:, v], ost.m_log)


@pytest.mark.parametrize("dim,nvec", [(100, 1), (100, 3), (37, 2), (16, 1)])
def test_complex_hermitian_ragged(mg, dim, nvec):
    """General complex Hermitian H (imaginary parts present), dims that leave ragged tiles."""
    rng = np.random.default_rng(dim + nvec)
    A = rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))
    H1 = (A + A.conj().T) / 4
    B = rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))
    H2 = (B + B.conj().T) / 8
    psi0 = mi.random_state(rng, dim, nvec)
    plan = mg.Plan(dim, [mg.DenseTerm(cuda(H1)), mg.DenseTerm(cuda(H2))],
                   [mg.Drive.const(), mg.Drive(0.0, [1.0], [], [3.0])], nvec=nvec)
    for variant in ("CF4", "M4"):
        psi = cuda(psi0)
        plan.propagate(psi, 0.0, 0.05, 8, variant)
        P = oracle.Problem([H1, H2], [oracle.Coeff.const(), oracle.Coeff(0.0, [1.0], [], [3.0])])
        out = psi.cpu().numpy().reshape(nvec, -1)
        for v in range(nvec):
            ref = P.propagate(psi0.reshape(nvec, -1)[v], 0.0, 0.05, 8, variant)
            assert rel(out[v], ref) < REL_TOL


def test_dense_expv_matches_eigh(mg):
    c = mi.workload3(nvec=2, nspins=8)
    Hs = mg.build_longrange_dense(c.nspins, c.hz)
    Hd = mg.build_field_x_dense(c.nspins)
    plan = mg.Plan(c.dim, [mg.DenseTerm(Hs), mg.DenseTerm(Hd)], drive_pair(mg, c), nvec=2, tol=1e-12)
    beta = np.array([0.05, 0.02])
    out, _ = plan.expv(beta, cuda(c.psi0))
    K = beta[0] * oracle.longrange_dense(c.nspins, c.hz) + beta[1] * oracle.field_x_dense(c.nspins)
    lam, U = np.linalg.eigh(K)
    for v in range(2):
        ref = U @ (np.exp(-1j * lam) * (U.conj().T @ c.psi0[v]))
        assert rel(out.cpu().numpy()[v], ref) < 1e-11


def test_workload3_full_size_sampled(mg):
    """13 spins (dim 8192), 64 states, dense H_s and dense sum sx: one Cf4 step of all 64 states in
    the bench's configuration; states 0 and 63 compared with the oracle entry by entry."""
    c = mi.workload3()
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    Hd = mg.build_field_x_dense(c.nspins)
    plan = mg.Plan(c.dim, [mg.DenseTerm(Hs), mg.DenseTerm(Hd)], drive_pair(mg, c), nvec=64)
    psi = cuda(c.psi0)
    st = plan.propagate(psi, 0.0, c.h, 1, "CF4", log_cap=1024)
    out = psi.cpu().numpy()
    P = oracle_dense(c, oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta), oracle.field_x_dense(c.nspins))
    for v in (0, 63):
        ost = oracle.Stats(64)
        ref = P.propagate(c.psi0[v], 0.0, c.h, 1, "CF4", ost)
        assert rel(out[v], ref) < REL_TOL
        assert np.array_equal(st["m_log"].reshape(-1, 64)[:, v], ost.m_log)


@pytest.mark.parametrize("variant", ["CF4", "M4"])
def test_fp32_split_precision(mg, variant):
    """MAGNUS_FP32_SPLIT: dense matvecs on the FP32 pipe with error-free products and sums.
    Stated accuracy: state error <= 1e-9 relative to the FP64 oracle (target of the mode: 1e-8)."""
    c = mi.workload3(nvec=6, nspins=8, h=0.02, nsteps=10)
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    Hd = mg.build_field_x_dense(c.nspins)
    plan = mg.Plan(c.dim, [mg.DenseTerm(Hs), mg.DenseTerm(Hd)], drive_pair(mg, c), nvec=6, precision=mg.FP32_SPLIT)
    psi = cuda(c.psi0)
    plan.propagate(psi, 0.0, c.h, c.nsteps, variant)
    P = oracle_dense(c, oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta), oracle.field_x_dense(c.nspins))
    out = psi.cpu().numpy()
    errs = [rel(out[v], P.propagate(c.psi0[v], 0.0, c.h, c.nsteps, variant)) for v in range(6)]
    assert max(errs) < 1e-9, errs


def test_fp32_split_rejects_complex_terms(mg):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    with pytest.raises(mg.MagnusError) as e:
        mg.Plan(32, [mg.DenseTerm(cuda(A + A.conj().T))], [mg.Drive.const()], nvec=2, precision=mg.FP32_SPLIT)
    assert e.value.code == mg.EINVAL


@pytest.mark.parametrize("variant", ["CF4", "M4"])
@pytest.mark.parametrize("field", ["dense", "mfree"])
@pytest.mark.parametrize("nspins,nvec", [(8, 6), (7, 1), (9, 64)])
def test_tensor_sliced_precision(mg, variant, field, nspins, nvec):
    """MAGNUS_TENSOR_SLICED: dense matvecs as exact bf16 digit products on the tcgen05 tensor cores
    (Cf4: one product phase per Leja iteration; M4: u_k = H_k w, then the commutator phase).
    Stated accuracy: state error <= 1e-9 relative to the FP64 oracle; the Leja degrees may differ
    by rounding, so they are not compared."""
    c = mi.workload3(nvec=nvec, nspins=nspins, h=0.02, nsteps=6)
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    Hd = mg.build_field_x_dense(c.nspins) if field == "dense" else mg.FieldXTerm(c.nspins)
    terms = [mg.DenseTerm(Hs), mg.DenseTerm(Hd) if field == "dense" else Hd]
    plan = mg.Plan(c.dim, terms, drive_pair(mg, c), nvec=nvec, precision=mg.TENSOR_SLICED)
    psi = cuda(c.psi0)
    plan.propagate(psi, 0.0, c.h, c.nsteps, variant)
    P = oracle_dense(c, oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta), oracle.field_x_dense(c.nspins))
    out = psi.cpu().numpy().reshape(nvec, -1)
    psi0 = c.psi0.reshape(nvec, -1)
    check = range(nvec) if nvec <= 8 else [0, 1, 31, 62, 63]
    errs = [rel(out[v], P.propagate(psi0[v], 0.0, c.h, c.nsteps, variant)) for v in check]
    assert max(errs) < 1e-9, errs


@pytest.mark.parametrize("nterms", [1, 3])
def test_tensor_sliced_m4_commutator_pairs(mg, nterms):
    """M4 on the tensor cores with one term (no commutator: the commutator sum stays zero) and with
    three terms (two dense terms and a matrix-free field: three commutator pairs, each its own
    product phase, summed in pair order), against the FP64 oracle with the same terms."""
    c = mi.workload3(nvec=5, nspins=8, h=0.02, nsteps=6)
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    Hd = mg.build_field_x_dense(c.nspins)
    f = (c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)
    g = (0.2, [-0.15], [0.1], [1.3])  # the third term's drive
    terms = [mg.DenseTerm(Hs), mg.DenseTerm(Hd), mg.FieldXTerm(c.nspins)][:nterms]
    drives = [mg.Drive.const(), mg.Drive(*f), mg.Drive(*g)][:nterms]
    plan = mg.Plan(c.dim, terms, drives, nvec=5, precision=mg.TENSOR_SLICED)
    psi = cuda(c.psi0)
    plan.propagate(psi, 0.0, c.h, c.nsteps, "M4")
    H_or = [oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta), oracle.field_x_dense(c.nspins),
            oracle.field_x_dense(c.nspins)][:nterms]
    C_or = [oracle.Coeff.const(), oracle.Coeff(*f), oracle.Coeff(*g)][:nterms]
    P = oracle.Problem(H_or, C_or, tol=1e-10)
    out = psi.cpu().numpy().reshape(5, -1)
    psi0 = c.psi0.reshape(5, -1)
    errs = [rel(out[v], P.propagate(psi0[v], 0.0, c.h, c.nsteps, "M4")) for v in range(5)]
    assert max(errs) < 1e-9, errs


def test_tensor_sliced_wide_spread_states(mg):
    """Columns whose entries span many binades (one large entry, the rest tiny) and a zero state:
    the per-column exponent keeps the large entry exact and the zero column stays zero."""
    c = mi.workload3(nvec=3, nspins=8, h=0.02, nsteps=4)
    psi0 = c.psi0.reshape(3, -1).copy()
    psi0[1] *= 1e-6
    psi0[1][7] = 1.0
    psi0[2] = 0.0
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    plan = mg.Plan(c.dim, [mg.DenseTerm(Hs), mg.FieldXTerm(c.nspins)], drive_pair(mg, c), nvec=3,
                   precision=mg.TENSOR_SLICED)
    psi = cuda(psi0)
    plan.propagate(psi, 0.0, c.h, c.nsteps, "CF4")
    P = oracle_dense(c, oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta), oracle.field_x_dense(c.nspins))
    out = psi.cpu().numpy()
    for v in range(2):
        assert rel(out[v], P.propagate(psi0[v], 0.0, c.h, c.nsteps, "CF4")) < 1e-9
    assert not np.any(out[2])


def test_tensor_sliced_rejects_unsupported(mg):
    rng = np.random.default_rng(6)
    A = rng.standard_normal((128, 128)) + 1j * rng.standard_normal((128, 128))
    with pytest.raises(mg.MagnusError) as e:
        mg.Plan(128, [mg.DenseTerm(cuda(A + A.conj().T))], [mg.Drive.const()], nvec=2, precision=mg.TENSOR_SLICED)
    assert e.value.code == mg.EINVAL
    B = rng.standard_normal((64, 64))
    with pytest.raises(mg.MagnusError) as e:
        mg.Plan(64, [mg.DenseTerm(cuda((B + B.T).astype(np.complex128)))], [mg.Drive.const()], nvec=2,
                precision=mg.TENSOR_SLICED)
    assert e.value.code == mg.EINVAL


@pytest.mark.parametrize("precision", ["FP64", "FP32_SPLIT", "TENSOR_SLICED"])
@pytest.mark.parametrize("nvec", [1, 4])
def test_dense_real_storage(mg, precision, nvec):
    """MAGNUS_TERM_DENSE_REAL (float64, 8 B per element) in every precision against the oracle."""
    c = mi.workload3(nvec=nvec, nspins=8, h=0.02, nsteps=6)
    Hs = mg.DenseTerm(mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)).as_real()
    Hd = mg.DenseTerm(mg.build_field_x_dense(c.nspins)).as_real()
    assert Hs.real and Hs.val.dtype == torch.float64
    plan = mg.Plan(c.dim, [Hs, Hd], drive_pair(mg, c), nvec=nvec, precision=getattr(mg, precision))
    psi = cuda(c.psi0)
    plan.propagate(psi, 0.0, c.h, c.nsteps, "CF4")
    P = oracle_dense(c, oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta), oracle.field_x_dense(c.nspins))
    out = psi.cpu().numpy().reshape(nvec, -1)
    tol = REL_TOL if precision == "FP64" else 1e-9
    for v in range(nvec):
        ref = P.propagate(c.psi0.reshape(nvec, -1)[v], 0.0, c.h, c.nsteps, "CF4")
        assert rel(out[v], ref) < tol, (v, rel(out[v], ref))


@pytest.fixture(scope="module")
def dense13():
    """The 13-spin long-range chain (dim 8192, 2 x 1.07 GB complex128 dense terms) and the oracle
    built from the oracle's own dense matrices."""
    c = mi.workload3()
    Ho = oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    Hd = oracle.field_x_dense(c.nspins)
    return c, oracle_dense(c, Ho, Hd)


def test_dense13_full_size_tensor_sampled(mg, dense13):
    """Full size, in the bench's launch configuration (64 states, tcgen05 digit products, Cf4): one
    step; states 0 and 63 against the oracle (one by one), every state's norm conserved."""
    c, P = dense13
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    Hd = mg.build_field_x_dense(c.nspins)
    plan = mg.Plan(c.dim, [mg.DenseTerm(Hs), mg.DenseTerm(Hd)], drive_pair(mg, c), nvec=64,
                   precision=mg.TENSOR_SLICED)
    psi = cuda(c.psi0)
    plan.propagate(psi, 0.0, c.h, 1, "CF4")
    out = psi.cpu().numpy()
    norms = np.linalg.norm(out, axis=1) / np.linalg.norm(c.psi0, axis=1)
    assert np.max(np.abs(norms - 1.0)) < 1e-9
    for v in (0, 63):
        ref = P.propagate(c.psi0[v], 0.0, c.h, 1, "CF4")
        assert rel(out[v], ref) < 1e-9, (v, rel(out[v], ref))


@pytest.mark.parametrize("precision,tol,variant", [("tensor_sliced", 1e-8, "CF4"), ("fp32_split", 1e-10, "CF4"),
                                                   ("tensor_sliced", 1e-8, "M4")])
def test_reduced_precision_over_a_whole_propagation(mg, precision, tol, variant):
    """The reduced-precision dense paths over the whole propagation t in [0, 1] (100 steps of 0.01,
    Cf4, and M4 on the tensor cores), 12 spins (dim 4096), 64 states in the bench's launch
    configuration: states 0 and 63 against the FP64 oracle.  Bound: the 1e-8 state error the
    tensor-core path is held to (its neglected digit products accumulate over the steps), 1e-10 for
    the FP32 split (error-free products).  The oracle runs its OpenMP build (the checker's bits on
    all host cores)."""
    c = mi.workload3(nvec=64, nspins=12, h=0.01, nsteps=100)
    Hs = mg.build_longrange_dense(c.nspins, c.hz, 1.5, c.delta)
    Hd = mg.build_field_x_dense(c.nspins)
    prec = {"tensor_sliced": mg.TENSOR_SLICED, "fp32_split": mg.FP32_SPLIT}[precision]
    plan = mg.Plan(c.dim, [mg.DenseTerm(Hs), mg.DenseTerm(Hd)], drive_pair(mg, c), nvec=64, precision=prec)
    psi = cuda(c.psi0)
    plan.propagate(psi, 0.0, c.h, c.nsteps, variant)
    out = psi.cpu().numpy()
    f = oracle.Coeff(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)
    P = oracle.Problem([oracle.longrange_dense(c.nspins, c.hz, 1.5, c.delta), oracle.field_x_dense(c.nspins)],
                       [oracle.Coeff.const(), f], threaded=True)
    for v in (0, 63):
        ref = P.propagate(c.psi0[v], 0.0, c.h, c.nsteps, variant)
        assert rel(out[v], ref) < tol, (precision, variant, v, rel(out[v], ref))
