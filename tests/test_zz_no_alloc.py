"""The allocation-free entry point magnus_expv_xxz_static against the plan-based leja_expv and the
FP64 CPU oracle.

magnus_expv_xxz_static serves callers that cannot call cudaMalloc (memory owned by another
allocator or pool, or loops that must not pay cudaMalloc's synchronisation).  It keeps its scratch
in one fixed device array inside the library, so this test checks through the C ABI:
- that its results agree with leja_expv of a plan holding the same matrix-free terms, on two calls
  in a row (the second call must not be disturbed by what the first left in the shared array);
- the same at both ends of the supported range: 2 spins and 16 spins (dim 65,536, the array's
  maximum, where the grid reaches its occupancy cap);
- at 16 spins, directly against the oracle's expv with the same terms;
- that chains above the fixed maximum are rejected.
It sits in a file of its own, collected last.
"""
import numpy as np
import pytest

import magnus_inputs as mi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10  # same tolerance as the other parity tests


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_06483_gb300 as m
    m.load()
    return m


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


CASES = [  # (seed, spins, beta)
    (41, 12, (0.004, 0.0021)),
    (42, 9, (0.35, -0.8)),
    (43, 16, (0.01, 0.006)),
    (44, 2, (0.7, 0.3)),
]


def test_static_expv_matches_plan_expv_on_two_calls(mg):
    for seed, n, beta in CASES:
        c = mi.xxz_chain(seed, n, 0.01, 1)
        beta = np.array(beta)
        terms = [mg.XXZTerm(c.nspins, c.J, c.hz, c.delta), mg.FieldXTerm(c.nspins)]
        plan = mg.Plan(c.dim, terms, [mg.Drive.const(), mg.Drive.const()], tol=1e-10)
        v = torch.from_numpy(c.psi0).cuda()
        ref, _ = plan.expv(beta, v)
        out = mg.expv_xxz_static(c.nspins, c.J, c.hz, c.delta, beta, v, tol=1e-10)
        assert rel(out, ref) < TOL, (n, rel(out, ref))
        # in place (v and out alias), right after the first call
        w = v.clone()
        mg.expv_xxz_static(c.nspins, c.J, c.hz, c.delta, beta, w, out=w, tol=1e-10)
        assert rel(w, ref) < TOL, (n, rel(w, ref))
        plan.close()


def test_static_expv_matches_oracle_at_the_maximum_size(mg):
    c = mi.xxz_chain(45, 16, 0.01, 1)
    beta = np.array([0.02, -0.013])
    P = oracle.Problem([oracle.xxz_csr(c.nspins, c.J, c.hz, c.delta), oracle.field_x_csr(c.nspins)],
                       [oracle.Coeff.const(), oracle.Coeff.const()], tol=1e-10)
    ref = P.expv(beta, c.psi0)
    v = torch.from_numpy(c.psi0).cuda()
    for _ in range(2):  # two calls in a row on the shared array
        out = mg.expv_xxz_static(c.nspins, c.J, c.hz, c.delta, beta, v, tol=1e-10).cpu().numpy()
        assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < TOL


def test_static_expv_rejects_chains_above_the_fixed_maximum(mg):
    n = 17
    v = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    with pytest.raises(mg.MagnusError) as e:
        mg.expv_xxz_static(n, np.ones(n - 1), np.zeros(n), 0.5, np.array([0.1, 0.1]), v)
    assert e.value.code == mg.EINVAL
    assert "2..16" in str(e.value)
