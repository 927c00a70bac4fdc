"""Adjoint gradient on the GPU against the FP64 CPU adjoint and against central differences.

Tolerance: F within 1e-12 and every gradient component within 1e-9 (absolute, gradients are O(1e-2)).
"""
import numpy as np
import pytest

import magnus_inputs as mi
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1709_06483_gb300 as m
    m.load()
    return m


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def control_chain(n, nmodes, T, seed):
    c = mi.xxz_chain(seed, n, 0.01, 1)
    rng = np.random.default_rng(seed + 1)
    ck = rng.normal(0, 0.3, nmodes)
    om = np.pi * np.arange(1, nmodes + 1) / T
    phi = mi.random_state(rng, 1 << n)
    return c, ck, om, phi


@pytest.mark.parametrize("kind", ["csr", "csr_real", "mfree"])
@pytest.mark.parametrize("variant,ckpt", [("CF4", 3), ("CF4_3", 4), ("M2", 7)])
def test_adjoint_matches_oracle(mg, kind, variant, ckpt):
    n, nmodes, T, h, N = 8, 6, 1.0, 0.04, 25
    c, ck, om, phi = control_chain(n, nmodes, T, 51)
    ac = 0.1 * np.ones(nmodes)
    if kind == "csr":
        terms = [mg.build_xxz_csr(n, c.J, c.hz, c.delta), mg.build_field_x_csr(n)]
    elif kind == "csr_real":
        terms = [mg.build_xxz_csr(n, c.J, c.hz, c.delta).as_real(), mg.build_field_x_csr(n).as_real()]
    else:
        terms = [mg.XXZTerm(n, c.J, c.hz, c.delta), mg.FieldXTerm(n)]
    plan = mg.Plan(c.dim, terms, [mg.Drive.const(), mg.Drive(0.2, ac, ck, om)], tol=1e-12)
    F, grad, st = plan.adjoint_grad(cuda(c.psi0), cuda(phi), 0.0, h, N, variant, kd=1, ckpt_every=ckpt)
    P = oracle.Problem([oracle.xxz_csr(n, c.J, c.hz, c.delta), oracle.field_x_csr(n)],
                       [oracle.Coeff.const(), oracle.Coeff(0.2, ac, ck, om)], tol=1e-12)
    Fr, gr = P.adjoint_grad(c.psi0, phi, 0.0, h, N, variant, kd=1)
    assert abs(F - Fr) < 1e-12
    assert np.max(np.abs(grad - gr)) < 1e-9, np.max(np.abs(grad - gr))


def test_workload5_full_size_vs_central_differences(mg):
    """16 spins, 32 sine modes, T = 10, 1000 Cf4 steps, checkpoints every 16 steps: the adjoint
    gradient against central differences of F (GPU forward propagations) for 4 coefficients."""
    c = mi.workload5()
    om, ck = c.drive_om, c.drive_as
    n = c.nspins

    def plan_for(coefs, tol):
        terms = [mg.XXZTerm(n, c.J, c.hz, c.delta), mg.FieldXTerm(n)]
        return mg.Plan(c.dim, terms, [mg.Drive.const(), mg.Drive(0.0, np.zeros(om.size), coefs, om)], tol=tol)

    plan = plan_for(ck, 1e-12)
    F, grad, st = plan.adjoint_grad(cuda(c.psi0), cuda(c.phi), 0.0, c.h, c.nsteps, "CF4", kd=1, ckpt_every=16)
    assert 0.0 <= F <= 1.0

    def fid(coefs):
        p = plan_for(coefs, 1e-13)
        psi = cuda(c.psi0)
        p.propagate(psi, 0.0, c.h, c.nsteps, "CF4")
        return abs(torch.vdot(cuda(c.phi), psi).item()) ** 2

    dl = 1e-5
    for k in (0, 7, 15, 31):
        up, dn = ck.copy(), ck.copy()
        up[k] += dl
        dn[k] -= dl
        fd = (fid(up) - fid(dn)) / (2 * dl)
        g = grad[1 + om.size + k]  # dF/das_k
        assert abs(g - fd) < 1e-8 + 1e-5 * abs(fd), (k, g, fd)


def test_fidelity_autograd_function(mg):
    """torch.autograd: F(c) through mg.fidelity, F.backward() gives the oracle's adjoint gradient,
    and a gradient-ascent step on c increases F."""
    n, nmodes, T, h, N = 8, 6, 1.0, 0.04, 25
    c, ck, om, phi = control_chain(n, nmodes, T, 52)
    ac = 0.1 * np.ones(nmodes)
    terms = [mg.XXZTerm(n, c.J, c.hz, c.delta), mg.FieldXTerm(n)]
    plan = mg.Plan(c.dim, terms, [mg.Drive.const(), mg.Drive(0.0, np.zeros(nmodes), np.zeros(nmodes), om)], tol=1e-12)
    params = torch.tensor(np.concatenate([[0.2], ac, ck]), dtype=torch.float64, requires_grad=True)
    psi0, phit = cuda(c.psi0), cuda(phi)
    F = mg.fidelity(plan, params, psi0, phit, 0.0, h, N, "CF4", kd=1, ckpt_every=5)
    F.backward()
    P = oracle.Problem([oracle.xxz_csr(n, c.J, c.hz, c.delta), oracle.field_x_csr(n)],
                       [oracle.Coeff.const(), oracle.Coeff(0.2, ac, ck, om)], tol=1e-12)
    Fr, gr = P.adjoint_grad(c.psi0, phi, 0.0, h, N, "CF4", kd=1)
    assert abs(F.item() - Fr) < 1e-12
    assert np.max(np.abs(params.grad.numpy() - gr)) < 1e-9
    with torch.no_grad():
        stepped = params + 0.05 * params.grad / params.grad.norm()
    F2 = mg.fidelity(plan, stepped, psi0, phit, 0.0, h, N, "CF4", kd=1, ckpt_every=5)
    assert F2.item() > F.item()


def test_workload5_size_against_the_cpu_adjoint_every_entry(mg):
    """16 spins (dim 65,536), the 32-mode sine drive of the control workload (T = 10), checkpoints
    every 16 steps, but 48 Cf4 steps of 0.01 instead of 1000 so that the CPU adjoint finishes in
    seconds: all 65 gradient entries (a0, 32 cosine, 32 sine amplitudes) and F against the FP64 CPU
    adjoint, to 1e-8 relative to the largest entry.  GPU terms matrix-free (the control workload's),
    the oracle's CSR."""
    c = mi.workload5()
    om, ck = c.drive_om, c.drive_as
    n, N = c.nspins, 48
    plan = mg.Plan(c.dim, [mg.XXZTerm(n, c.J, c.hz, c.delta), mg.FieldXTerm(n)],
                   [mg.Drive.const(), mg.Drive(0.0, np.zeros(om.size), ck, om)], tol=1e-12)
    F, grad, st = plan.adjoint_grad(cuda(c.psi0), cuda(c.phi), 0.0, c.h, N, "CF4", kd=1, ckpt_every=16)
    P = oracle.Problem([oracle.xxz_csr(n, c.J, c.hz, c.delta), oracle.field_x_csr(n)],
                       [oracle.Coeff.const(), oracle.Coeff(0.0, np.zeros(om.size), ck, om)], tol=1e-12)
    Fr, gr = P.adjoint_grad(c.psi0, c.phi, 0.0, c.h, N, "CF4", kd=1)
    assert grad.size == gr.size == 65
    assert abs(F - Fr) <= 1e-10 * abs(Fr)
    assert np.max(np.abs(grad - gr)) <= 1e-8 * np.max(np.abs(gr)), np.max(np.abs(grad - gr)) / np.max(np.abs(gr))
