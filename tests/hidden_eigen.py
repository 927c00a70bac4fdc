"""A Hermitian matrix whose largest eigenvalue the Lanczos enclosure does not see (test input).

The Lanczos enclosure (the spectral interval the Leja parameters are taken from, when chosen) runs 48
steps from one fixed start vector: v_i = (2 u_{2i} - 1) + i (2 u_{2i+1} - 1), normalised, u_c the
c-th output of SplitMix64 (Steele, Lea, Flood 2014, counter form) seeded with 1709064830, mapped to
[0, 1) by its top 53 bits.  An eigenvector orthogonal to that vector enters the Krylov space only
through rounding; when its eigenvalue lies just outside the rest of the spectrum, the rounding
error grows too slowly over 48 steps to be resolved, and the enclosure ends below it.
"""
import numpy as np

_MASK = (1 << 64) - 1


def _splitmix64_at(seed, c):
    z = (seed + (c + 1) * 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def lanczos_start(n, seed=1709064830):
    u = [(_splitmix64_at(seed, c) >> 11) * 2.0 ** -53 for c in range(2 * n)]
    v = np.array([(2 * u[2 * i] - 1) + 1j * (2 * u[2 * i + 1] - 1) for i in range(n)])
    return v / np.linalg.norm(v)


def hidden_top(n, lam_top, seed=5):
    """(H, Q): H = Q diag(lam_top, bulk) Q^H with the bulk spread evenly over [-1, 1] and the
    eigenvector of lam_top (Q[:, 0]) orthogonal to the Lanczos start vector."""
    rng = np.random.default_rng(seed)
    v0 = lanczos_start(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x -= np.vdot(v0, x) * v0
    q = x / np.linalg.norm(x)
    A = np.column_stack([q] + [rng.standard_normal(n) + 1j * rng.standard_normal(n) for _ in range(n - 1)])
    Q, _ = np.linalg.qr(A)
    Q[:, 0] = q  # the QR's first column is q up to a phase
    ev = np.concatenate([[lam_top], np.linspace(-1.0, 1.0, n - 1)])
    H = (Q * ev) @ Q.conj().T
    return (H + H.conj().T) / 2, Q
