"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

Only random draws live here -- no matrix element, coefficient or any other piece
of the method's arithmetic.  Each workload draws with numpy's PCG64
(``default_rng``) seeded with ``1709064830 + workload number``, in the order
couplings J, fields h, drive parameters, initial state(s) psi0, target phi.

Workloads (spin-chain sizes of the paper's Sec. 4 experiments, scaled to GB300):
  1  open XXZ chain, 10 spins (dim 1024), J_i ~ U[0.5,1.5], h_i ~ U[-1,1],
     drive cos(5t) on sum_i sx_i, random normalised complex psi0, step 0.01 on [0,1].
  2  the same chain at 20 spins (dim 1,048,576), step 0.005, 200 steps.
  3  long-range chain, 13 spins (dim 8192), J_ij = 1/|i-j|^1.5 (fixed), h_i ~ U[-1,1],
     drive cos(5t), 64 random initial states.
  4  512 independent XXZ chains, spins ~ U{8..14}, per-chain J, h, drive
     amplitude A ~ U[0.5,2] and frequency w ~ U[1,10] (f = A cos(w t)), step 0.01, 100 steps.
  5  XXZ chain, 16 spins, drive f(t) = sum_{k=1}^{32} c_k sin(k pi t / T), c_k ~ N(0, 0.3),
     T = 10, 1000 steps of 0.01, random target phi.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1709064830


def rng_for(workload: int) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + int(workload))


def random_state(rng: np.random.Generator, dim: int, count: int | None = None) -> np.ndarray:
    """Complex normal entries, each state scaled to unit 2-norm."""
    shape = (dim,) if count is None else (count, dim)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    z /= np.linalg.norm(z, axis=-1, keepdims=True)
    return np.ascontiguousarray(z.astype(np.complex128))


@dataclass
class Chain:
    """One spin chain with static couplings, a drive f(t) on sum_i sx_i and initial state(s)."""
    nspins: int
    J: np.ndarray                 # (nspins-1,) bond couplings (XXZ) -- unused by long-range chains
    hz: np.ndarray                # (nspins,) longitudinal fields
    delta: float                  # zz anisotropy
    drive_a0: float
    drive_ac: np.ndarray          # cosine amplitudes
    drive_as: np.ndarray          # sine amplitudes
    drive_om: np.ndarray          # angular frequencies
    psi0: np.ndarray              # (dim,) or (nvec, dim)
    h: float
    nsteps: int
    t0: float = 0.0
    phi: np.ndarray | None = None
    alpha: float | None = None    # long-range decay exponent, None for nearest-neighbour chains
    extra: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return 1 << self.nspins


def xxz_chain(workload: int, nspins: int, h: float, nsteps: int, nvec: int | None = None) -> Chain:
    """Open XXZ chain with drive cos(5t) (workloads 1 and 2, and smaller test chains)."""
    rng = rng_for(workload)
    J = rng.uniform(0.5, 1.5, nspins - 1)
    hz = rng.uniform(-1.0, 1.0, nspins)
    psi0 = random_state(rng, 1 << nspins, nvec)
    return Chain(nspins, J, hz, 0.5, 0.0, np.array([1.0]), np.array([0.0]), np.array([5.0]), psi0, h, nsteps)


def workload1() -> Chain:
    return xxz_chain(1, 10, 0.01, 100)


def workload2() -> Chain:
    return xxz_chain(2, 20, 0.005, 200)


def workload3(nvec: int = 64, nspins: int = 13, h: float = 0.01, nsteps: int = 100) -> Chain:
    rng = rng_for(3)
    hz = rng.uniform(-1.0, 1.0, nspins)
    psi0 = random_state(rng, 1 << nspins, nvec)
    return Chain(nspins, np.zeros(0), hz, 0.5, 0.0, np.array([1.0]), np.array([0.0]), np.array([5.0]), psi0,
                 h, nsteps, alpha=1.5)


def workload4(count: int = 512, nmin: int = 8, nmax: int = 14, h: float = 0.01, nsteps: int = 100) -> list[Chain]:
    rng = rng_for(4)
    sizes = rng.integers(nmin, nmax + 1, count)
    chains = []
    for n in sizes:
        n = int(n)
        J = rng.uniform(0.5, 1.5, n - 1)
        hz = rng.uniform(-1.0, 1.0, n)
        A = rng.uniform(0.5, 2.0)
        w = rng.uniform(1.0, 10.0)
        chains.append(Chain(n, J, hz, 0.5, 0.0, np.array([A]), np.array([0.0]), np.array([w]), None, h, nsteps))
    for c in chains:
        c.psi0 = random_state(rng, c.dim)
    return chains


def workload5(nspins: int = 16, nmodes: int = 32, T: float = 10.0, h: float = 0.01, nsteps: int = 1000) -> Chain:
    rng = rng_for(5)
    J = rng.uniform(0.5, 1.5, nspins - 1)
    hz = rng.uniform(-1.0, 1.0, nspins)
    ck = rng.normal(0.0, 0.3, nmodes)
    psi0 = random_state(rng, 1 << nspins)
    phi = random_state(rng, 1 << nspins)
    om = np.pi * np.arange(1, nmodes + 1) / T
    return Chain(nspins, J, hz, 0.5, 0.0, np.zeros(nmodes), ck, om, psi0, h, nsteps, phi=phi, extra={"T": T})
