"""Batches of independent chains in one persistent launch, against the oracle chain by chain.

Tolerance: relative 2-norm error <= 1e-10 per chain and identical Leja degree sequences.
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


def problems(mg, chains, kind):
    out = []
    for c in chains:
        if kind == "csr":
            terms = [mg.build_xxz_csr(c.nspins, c.J, c.hz, c.delta), mg.build_field_x_csr(c.nspins)]
        elif kind == "csr_real":
            terms = [mg.build_xxz_csr(c.nspins, c.J, c.hz, c.delta).as_real(), mg.build_field_x_csr(c.nspins).as_real()]
        else:
            terms = [mg.XXZTerm(c.nspins, c.J, c.hz, c.delta), mg.FieldXTerm(c.nspins)]
        out.append((c.dim, terms, [mg.Drive.const(), mg.Drive(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)]))
    return out


def oracle_run(c, t0, h, nsteps, variant, cap=4096):
    Hs = oracle.xxz_csr(c.nspins, c.J, c.hz, c.delta)
    Hd = oracle.field_x_csr(c.nspins)
    P = oracle.Problem([Hs, Hd], [oracle.Coeff.const(), oracle.Coeff(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)])
    st = oracle.Stats(cap)
    return P.propagate(c.psi0, t0, h, nsteps, variant, st), st.m_log


@pytest.fixture(scope="module")
def small_chains():
    return mi.workload4(count=14, nmin=3, nmax=9, nsteps=12)


@pytest.mark.parametrize("kind", ["csr", "csr_real", "mfree"])
@pytest.mark.parametrize("variant", ["CF4", "M4"])
def test_batch_matches_oracle(mg, small_chains, kind, variant):
    chains = small_chains
    B = mg.Batch(problems(mg, chains, kind))
    psis = [torch.from_numpy(c.psi0.copy()).cuda() for c in chains]
    st = B.propagate(psis, 0.0, chains[0].h, chains[0].nsteps, variant, log_cap=256)
    for i, c in enumerate(chains):
        ref, mlog = oracle_run(c, 0.0, c.h, c.nsteps, variant)
        assert rel(psis[i].cpu().numpy(), ref) < REL_TOL, i
        assert np.array_equal(st["m_log"][i, :mlog.size], mlog), i
    assert st["block"] in (128, 256, 512, 1024) and st["cluster"] in (1, 2, 4)


@pytest.mark.parametrize("cs", [1, 2, 4])
@pytest.mark.parametrize("bs", [128, 256, 512, 1024])
def test_every_cta_and_cluster_size(mg, small_chains, bs, cs):
    """Each problem on a cluster of cs CTAs of bs threads (rows split across the cluster)."""
    chains = small_chains[:6]
    B = mg.Batch(problems(mg, chains, "csr" if bs != 512 else "mfree"), ctas=-(bs + 65536 * cs))
    psis = [torch.from_numpy(c.psi0.copy()).cuda() for c in chains]
    st = B.propagate(psis, 0.0, chains[0].h, 5, "CF4" if cs != 2 else "M4")
    assert st["block"] == bs and st["cluster"] == cs
    for i, c in enumerate(chains):
        ref, _ = oracle_run(c, 0.0, c.h, 5, "CF4" if cs != 2 else "M4")
        assert rel(psis[i].cpu().numpy(), ref) < REL_TOL


@pytest.mark.parametrize("cs", [2, 4])
def test_shared_large_item_then_small_items_alone(mg, cs):
    """One chain far above a CTA's fair share of the rows (shared by the CTAs of a cluster) and ten
    small ones (taken by single CTAs from the second queue once the shared items are handed out),
    Cf4 with fixed-point sums and M4 in FP64, against the oracle."""
    big = mi.xxz_chain(60, 12, 0.01, 6)
    small = [mi.xxz_chain(61 + i, 5, 0.01, 6) for i in range(10)]
    chains = [small[0], big] + small[1:]  # the large one is not first in the list
    for variant in ("CF4", "M4"):
        B = mg.Batch(problems(mg, chains, "csr"), ctas=-(256 + 65536 * cs))
        psis = [torch.from_numpy(c.psi0.copy()).cuda() for c in chains]
        st = B.propagate(psis, 0.0, 0.01, 6, variant)
        assert st["cluster"] == cs
        for i, c in enumerate(chains):
            ref, _ = oracle_run(c, 0.0, 0.01, 6, variant)
            assert rel(psis[i].cpu().numpy(), ref) < REL_TOL, (variant, i)
        B.close()


def test_graph_replay_and_continuation(mg, small_chains):
    """Two calls of 6 steps (the second replays a new graph from t0 = 6h) equal one run of 12 steps;
    a third identical call replays the cached graph."""
    chains = small_chains[:5]
    B = mg.Batch(problems(mg, chains, "mfree"))
    h = chains[0].h
    psis = [torch.from_numpy(c.psi0.copy()).cuda() for c in chains]
    B.propagate(psis, 0.0, h, 6, "CF4")
    B.propagate(psis, 6 * h, h, 6, "CF4")
    for i, c in enumerate(chains):
        ref, _ = oracle_run(c, 0.0, h, 12, "CF4")
        assert rel(psis[i].cpu().numpy(), ref) < REL_TOL
    again = [torch.from_numpy(c.psi0.copy()).cuda() for c in chains]
    B.propagate(again, 6 * h, h, 6, "CF4")  # same parameters as the last call: cached graph
    for i, c in enumerate(chains):
        ref, _ = oracle_run(c, 6 * h, h, 6, "CF4")
        assert rel(again[i].cpu().numpy(), ref) < REL_TOL


def test_workload4_full_size_sampled(mg):
    """512 chains of 8-14 spins, 100 Cf4 steps in one launch; the smallest, the largest and two
    others compared with the oracle entry by entry."""
    chains = mi.workload4()
    B = mg.Batch(problems(mg, chains, "csr"))
    psis = [torch.from_numpy(c.psi0.copy()).cuda() for c in chains]
    st = B.propagate(psis, 0.0, 0.01, 100, "CF4")
    assert st["n_exp"] == 512 * 200
    dims = np.array([c.dim for c in chains])
    for i in (int(np.argmin(dims)), int(np.argmax(dims)), 7, 300):
        ref, _ = oracle_run(chains[i], 0.0, 0.01, 100, "CF4")
        assert rel(psis[i].cpu().numpy(), ref) < REL_TOL, i


@pytest.mark.parametrize("kind", ["csr", "csr_real", "mfree"])
@pytest.mark.parametrize("variant", ["CF4", "CF4_3", "M2"])
def test_batch_fixed_and_fp64_sums(mg, small_chains, kind, variant):
    """Linear generators sum the transverse field in fixed point (options.fixed_sums), on every
    CTA and cluster size the autotuner may pick; FP64 sums beside them; both against the oracle."""
    chains = small_chains[:8]
    for fixed in (True, False):
        B = mg.Batch(problems(mg, chains, kind), fixed_sums=fixed)
        psis = [torch.from_numpy(c.psi0.copy()).cuda() for c in chains]
        st = B.propagate(psis, 0.0, chains[0].h, 8, variant, log_cap=128)
        assert st["fixed_sums"] == int(fixed)
        for i, c in enumerate(chains):
            ref, mlog = oracle_run(c, 0.0, c.h, 8, variant)
            assert rel(psis[i].cpu().numpy(), ref) < REL_TOL, (fixed, i)
            assert np.array_equal(st["m_log"][i, :mlog.size], mlog), (fixed, i)


@pytest.mark.parametrize("cs", [1, 4])
def test_batch_fixed_sums_m4_then_cf4(mg, small_chains, cs):
    """M4 keeps FP64 sums in a batch that sums in fixed point; a Cf4 call after it scales its copies
    from the maxima the M4 launch left (clusters of cs CTAs)."""
    chains = small_chains[:6]
    B = mg.Batch(problems(mg, chains, "mfree"), ctas=-(256 + 65536 * cs))
    psis = [torch.from_numpy(c.psi0.copy()).cuda() for c in chains]
    h = chains[0].h
    assert B.propagate(psis, 0.0, h, 4, "M4")["fixed_sums"] == 0
    assert B.propagate(psis, 4 * h, h, 4, "CF4")["fixed_sums"] == 1
    for i, c in enumerate(chains):
        mid, _ = oracle_run(c, 0.0, h, 4, "M4")
        d = type(c)(**{**c.__dict__, "psi0": mid})
        ref, _ = oracle_run(d, 4 * h, h, 4, "CF4")
        assert rel(psis[i].cpu().numpy(), ref) < REL_TOL, i


def test_workload4_full_size_sampled_matrix_free(mg):
    """The 512 chains with matrix-free terms and fixed-point field sums, 100 Cf4 steps; four chains
    compared with the oracle entry by entry."""
    chains = mi.workload4()
    B = mg.Batch(problems(mg, chains, "mfree"))
    psis = [torch.from_numpy(c.psi0.copy()).cuda() for c in chains]
    st = B.propagate(psis, 0.0, 0.01, 100, "CF4")
    assert st["fixed_sums"] == 1 and st["n_exp"] == 512 * 200
    dims = np.array([c.dim for c in chains])
    for i in (int(np.argmin(dims)), int(np.argmax(dims)), 11, 400):
        ref, _ = oracle_run(chains[i], 0.0, 0.01, 100, "CF4")
        assert rel(psis[i].cpu().numpy(), ref) < REL_TOL, i
