"""The a posteriori norm check (options.norm_check, stats.norm_drift) on the GPU.

Every exponential of a Hermitian generator keeps the norm, so | ||p|| - ||v|| | / ||v|| of a substep
(p its result, v its input) is 0 up to rounding and the Leja tolerance.  These tests check:
- that the drift is reported at that level on the 10-spin chain (CSR, fixed point) with both the
  Gershgorin and the Lanczos interval, and that a norm check of 100 x the tolerance passes there;
- the GPU side of the hidden-eigenvalue case (tests/hidden_eigen.py): the Lanczos interval misses
  the top eigenvalue, the propagation still matches exp(-i T H) psi and the check passes;
- that a generator which does not keep the norm (a term i eps Identity: exp(-i tau (H + i eps)) =
  e^{eps tau} exp(-i tau H)) is caught: MAGNUS_EDRIFT with the check on; with it off the call runs,
  reports the drift, and the state's norm grows by e^{eps T} as it should.
"""
import numpy as np
import pytest

import magnus_inputs as mi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_06483_gb300 as m
    m.load()
    return m


def _chain(mg, c):
    Hs = mg.build_xxz_csr(c.nspins, c.J, c.hz, c.delta)
    Hd = mg.build_field_x_csr(c.nspins)
    drives = [mg.Drive.const(), mg.Drive(c.drive_a0, c.drive_ac, c.drive_as, c.drive_om)]
    return [Hs, Hd], drives


@pytest.mark.parametrize("interval", ["gershgorin", "lanczos"])
def test_norm_drift_is_at_the_tolerance_level(mg, interval):
    c = mi.workload1()
    terms, drives = _chain(mg, c)
    plan = mg.Plan(c.dim, terms, drives, interval=interval, norm_check=100.0)
    psi = torch.from_numpy(c.psi0).cuda()
    st = plan.propagate(psi, c.t0, c.h, 20, "CF4")
    assert 0.0 <= st["norm_drift"] < 1e-9, st["norm_drift"]
    plan.close()


def test_hidden_eigenvalue_is_propagated_and_passes_the_check(mg):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    import hidden_eigen
    H, Q = hidden_eigen.hidden_top(256, 1.2)
    psi0 = Q[:, 0] + 0.1 * Q[:, 5]
    psi0 /= np.linalg.norm(psi0)
    plan = mg.Plan(256, [mg.DenseTerm(torch.from_numpy(np.ascontiguousarray(H)).cuda())], [mg.Drive.const()],
                   interval="lanczos", norm_check=100.0)
    for h, ns in ((0.2, 5), (4.0, 1)):
        psi = torch.from_numpy(psi0.copy()).cuda()
        st = plan.propagate(psi, 0.0, h, ns, "CF4")
        ref = scipy_linalg.expm(-1j * (h * ns) * H) @ psi0
        assert np.linalg.norm(psi.cpu().numpy() - ref) < 1e-9
        assert st["norm_drift"] < 1e-9
    plan.close()


def test_norm_check_catches_a_generator_that_does_not_keep_the_norm(mg):
    c = mi.workload1()
    terms, drives = _chain(mg, c)
    eps = 1e-3
    D = c.dim
    shift = mg.CSRTerm(torch.arange(D + 1, device="cuda"), torch.arange(D, device="cuda"),
                       torch.full((D,), 1j * eps, dtype=torch.complex128, device="cuda"))
    terms, drives = terms + [shift], drives + [mg.Drive.const()]
    psi0 = torch.from_numpy(c.psi0).cuda()
    nsteps = 10
    plan = mg.Plan(D, terms, drives, norm_check=100.0)
    with pytest.raises(mg.MagnusError) as e:
        plan.propagate(psi0.clone(), c.t0, c.h, nsteps, "CF4")
    assert e.value.code == mg.EDRIFT
    plan.close()
    plan = mg.Plan(D, terms, drives)  # check off: runs, reports the drift
    psi = psi0.clone()
    st = plan.propagate(psi, c.t0, c.h, nsteps, "CF4")
    assert st["norm_drift"] > 1e-7
    grow = float(torch.linalg.norm(psi) / torch.linalg.norm(psi0))
    assert abs(grow - np.exp(eps * c.h * nsteps)) < 1e-9, grow
    plan.close()
