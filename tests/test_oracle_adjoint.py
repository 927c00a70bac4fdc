"""Pins of the oracle's Frechet derivative and adjoint gradient.

* The augmented-block Frechet derivative against the Daleckii-Krein closed form
  L(Omega, E) = U [(U^H E U) o Phi] U^H, Phi_ij = (e^{l_i} - e^{l_j}) / (l_i - l_j) (Phi_ii = e^{l_i}),
  for Omega = U diag(l) U^H normal.
* Its second block equals exp(Omega) v.
* The adjoint gradient of F = |<phi|psi(T)>|^2 against central finite differences of F.
"""
import numpy as np
import pytest

import magnus_inputs as mi
import oracle


def chain_problem(n, workload, drive, tol=1e-13):
    c = mi.xxz_chain(workload, n, 0.01, 1)
    Hs = oracle.xxz_csr(n, c.J, c.hz, 0.5)
    Hd = oracle.field_x_csr(n)
    return c, Hs, Hd, oracle.Problem([Hs, Hd], [oracle.Coeff.const(), drive], tol=tol, tol_abs=tol)


def daleckii_krein(Omega, E):
    lam, U = np.linalg.eig(Omega)
    Ui = np.linalg.inv(U)
    el = np.exp(lam)
    dl = lam[:, None] - lam[None, :]
    same = np.abs(dl) < 1e-12
    Phi = np.where(same, el[:, None], (el[:, None] - el[None, :]) / np.where(same, 1.0, dl))
    return U @ ((Ui @ E @ U) * Phi) @ Ui


@pytest.mark.parametrize("beta", [(0.03, 0.02), (0.4, -0.7), (3.0, 1.0)])
def test_frechet_matches_daleckii_krein(beta):
    n = 7
    c, Hs, Hd, P = chain_problem(n, 31, oracle.Coeff.const())
    K = beta[0] * Hs.todense() + beta[1] * Hd.todense()
    Omega, E = -1j * K, -1j * Hd.todense()
    a, b = P.frechet_expv(np.array(beta), 1, c.psi0)
    ref = daleckii_krein(Omega, E) @ c.psi0
    assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < 1e-10
    assert np.linalg.norm(b - P.expv(np.array(beta), c.psi0)) < 1e-12


def test_frechet_of_a_scalar_generator():
    """Omega = -i c I (a multiple of the identity): the block matrix [[Omega, E], [0, Omega]] has
    exponential e^{-ic} [[I, E], [0, I]], so L(Omega, E) v = e^{-ic} E v and the second block is
    e^{-ic} v (the Daleckii-Krein form with all eigenvalues equal).  Covers K = 0 and K = 0.7 I."""
    n = 5
    D = 1 << n
    c = oracle.CSR(np.arange(D + 1), np.arange(D), np.ones(D))  # the identity
    Hd = oracle.field_x_csr(n)
    P = oracle.Problem([c, Hd], [oracle.Coeff.const(), oracle.Coeff.const()], tol=1e-13, tol_abs=1e-13)
    v = mi.random_state(np.random.default_rng(35), D)
    for shift in (0.0, 0.7):
        a, b = P.frechet_expv(np.array([shift, 0.0]), 1, v)
        ph = np.exp(-1j * shift)
        assert np.max(np.abs(a - ph * (-1j) * (Hd.todense() @ v))) < 1e-14
        assert np.max(np.abs(b - ph * v)) < 1e-15


def test_frechet_matches_finite_difference():
    n = 6
    c, Hs, Hd, P = chain_problem(n, 32, oracle.Coeff.const())
    beta, dlt = np.array([0.2, 0.1]), 1e-5
    a, _ = P.frechet_expv(beta, 1, c.psi0)
    fd = (P.expv(beta + [0, dlt], c.psi0) - P.expv(beta - [0, dlt], c.psi0)) / (2 * dlt)
    assert np.linalg.norm(a - fd) / np.linalg.norm(fd) < 1e-8


@pytest.mark.parametrize("variant", ["CF4", "CF4_3", "M2"])
def test_adjoint_gradient_matches_central_differences(variant):
    n, T, nmodes = 6, 1.0, 4
    rng = np.random.default_rng(33)
    ck = rng.normal(0, 0.3, nmodes)
    om = np.pi * np.arange(1, nmodes + 1) / T
    ac = rng.normal(0, 0.2, nmodes)
    drive = oracle.Coeff(0.3, ac, ck, om)
    c, Hs, Hd, P = chain_problem(n, 34, drive)
    phi = mi.random_state(rng, 1 << n)
    h, N = 0.05, 20
    F, grad = P.adjoint_grad(c.psi0, phi, 0.0, h, N, variant, kd=1)

    def fid(a0, acv, asv):
        Q = oracle.Problem([Hs, Hd], [oracle.Coeff.const(), oracle.Coeff(a0, acv, asv, om)], tol=1e-13, tol_abs=1e-13)
        psi = Q.propagate(c.psi0, 0.0, h, N, variant)
        return abs(np.vdot(phi, psi)) ** 2

    assert abs(F - fid(0.3, ac, ck)) < 1e-12
    dl = 1e-5
    params = np.concatenate([[0.3], ac, ck])
    for q in range(params.size):
        up, dn = params.copy(), params.copy()
        up[q] += dl
        dn[q] -= dl
        fd = (fid(up[0], up[1:1 + nmodes], up[1 + nmodes:]) - fid(dn[0], dn[1:1 + nmodes], dn[1 + nmodes:])) / (2 * dl)
        assert abs(grad[q] - fd) < 1e-8 + 1e-6 * abs(fd), (q, grad[q], fd)
