"""The seeded synthetic inputs follow their stated recipe (CPU only).

Sizes, value ranges, normalisation and determinism of each workload's draws: 10- and 20-spin XXZ
chains with J ~ U[0.5, 1.5], h ~ U[-1, 1] and the drive cos(5t); the 13-spin long-range chain with
64 states; 512 chains of 8-14 spins with A ~ U[0.5, 2], w ~ U[1, 10]; the 16-spin control problem
with 32 sine modes of k pi / T, T = 10.
"""
import numpy as np

import magnus_inputs as mi


def _unit(states):
    return np.allclose(np.linalg.norm(np.atleast_2d(states), axis=1), 1.0, atol=1e-14)


def test_xxz_workloads():
    for c, n, h, steps in ((mi.workload1(), 10, 0.01, 100), (mi.workload2(), 20, 0.005, 200)):
        assert c.nspins == n and c.dim == 1 << n and c.h == h and c.nsteps == steps and c.t0 == 0.0
        assert c.J.shape == (n - 1,) and np.all((0.5 <= c.J) & (c.J <= 1.5))
        assert c.hz.shape == (n,) and np.all(np.abs(c.hz) <= 1.0)
        assert c.delta == 0.5 and c.drive_a0 == 0.0
        assert list(c.drive_ac) == [1.0] and list(c.drive_as) == [0.0] and list(c.drive_om) == [5.0]
        assert c.psi0.dtype == np.complex128 and c.psi0.shape == (c.dim,) and _unit(c.psi0)
    a, b = mi.workload1(), mi.workload1()
    assert np.array_equal(a.J, b.J) and np.array_equal(a.psi0, b.psi0)  # seeded: reproducible
    assert not np.array_equal(mi.xxz_chain(1, 10, 0.01, 1).J, mi.xxz_chain(2, 10, 0.01, 1).J)


def test_longrange_workload():
    c = mi.workload3()
    assert c.nspins == 13 and c.alpha == 1.5 and c.psi0.shape == (64, 8192) and _unit(c.psi0)
    assert np.all(np.abs(c.hz) <= 1.0) and list(c.drive_om) == [5.0]


def test_batch_workload():
    chains = mi.workload4()
    assert len(chains) == 512
    sizes = np.array([c.nspins for c in chains])
    assert sizes.min() >= 8 and sizes.max() <= 14 and len(set(sizes)) == 7  # every size 8..14 occurs
    for c in chains:
        assert 0.5 <= c.drive_ac[0] <= 2.0 and 1.0 <= c.drive_om[0] <= 10.0 and c.drive_as[0] == 0.0
        assert np.all((0.5 <= c.J) & (c.J <= 1.5)) and np.all(np.abs(c.hz) <= 1.0)
        assert c.psi0.shape == (c.dim,) and _unit(c.psi0) and c.h == 0.01 and c.nsteps == 100


def test_control_workload():
    c = mi.workload5()
    assert c.nspins == 16 and c.nsteps == 1000 and c.h == 0.01 and c.extra["T"] == 10.0
    assert np.allclose(c.drive_om, np.pi * np.arange(1, 33) / 10.0)
    assert np.all(c.drive_ac == 0.0) and c.drive_as.shape == (32,) and c.drive_a0 == 0.0
    assert 0.1 < np.std(c.drive_as) < 0.6  # c_k ~ N(0, 0.3)
    assert _unit(c.psi0) and _unit(c.phi) and abs(np.vdot(c.phi, c.psi0)) < 0.05
