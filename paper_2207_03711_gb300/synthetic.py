"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's callers.

This module only draws random numbers; it holds none of the method's arithmetic.
The paper's molecules (and their PySCF integrals) are not available, so random
molecule-shaped inputs stand in for them:

  * one-electron integrals h_pq ~ N(0, 1), symmetrised as (h + h^T) / 2;
  * two-electron integrals (pq|rs) ~ N(0, 0.1) (standard deviation 0.1), averaged
    over the 8 index permutations of real orbitals so the 8-fold symmetry holds;
  * UCCSD amplitudes theta ~ N(0, 0.05) (standard deviation 0.05).
"""
import numpy as np


def random_integrals(n_spatial, seed):
    rng = np.random.default_rng(seed)
    h = rng.normal(0.0, 1.0, size=(n_spatial, n_spatial))
    h = 0.5 * (h + h.T)
    g = rng.normal(0.0, 0.1, size=(n_spatial,) * 4)
    g = (g + g.transpose(1, 0, 2, 3) + g.transpose(0, 1, 3, 2) + g.transpose(1, 0, 3, 2)
         + g.transpose(2, 3, 0, 1) + g.transpose(3, 2, 0, 1) + g.transpose(2, 3, 1, 0)
         + g.transpose(3, 2, 1, 0)) / 8.0
    return np.ascontiguousarray(h), np.ascontiguousarray(g)


def random_amplitudes(n_params, seed):
    rng = np.random.default_rng(10_000 + seed)
    return rng.normal(0.0, 0.05, size=n_params)


def h2_shaped_integrals(seed):
    """Two spatial orbitals with only the integrals a real H2-like molecule has:
    h_11, h_22, (11|11), (22|22), (11|22) and the (12|12)-class exchange."""
    rng = np.random.default_rng(seed)
    h = np.diag(rng.normal(0.0, 1.0, size=2))
    g = np.zeros((2, 2, 2, 2))
    g[0, 0, 0, 0], g[1, 1, 1, 1] = rng.normal(0.5, 0.1, size=2)
    g[0, 0, 1, 1] = g[1, 1, 0, 0] = rng.normal(0.5, 0.1)
    x = rng.normal(0.2, 0.05)
    for idx in [(0, 1, 0, 1), (1, 0, 1, 0), (0, 1, 1, 0), (1, 0, 0, 1)]:
        g[idx] = x
    return h, g


def random_mps_gaussians(n, ranks, seed):
    """Complex Gaussian arrays (2 r_k, r_{k-1}) per site for a random MPS with the given
    bond ranks (the orthonormalisation into canonical form is done by the caller)."""
    rng = np.random.default_rng(20_000 + seed)
    r = [1] + list(ranks) + [1]
    return [rng.normal(size=(2 * r[k + 1], r[k])) + 1j * rng.normal(size=(2 * r[k + 1], r[k]))
            for k in range(n)]


def full_ranks(n, chi):
    """Largest bond ranks an n-site MPS with bond cap chi can have."""
    return [min(chi, 2 ** min(b + 1, n - 1 - b)) for b in range(n - 1)]


def random_unitary4(seed):
    rng = np.random.default_rng(30_000 + seed)
    z = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    return z  # the caller orthonormalises (QR) if it needs a unitary


def random_right_canonical_mps(n, chi, seed):
    """Timing/profiling input only: right-canonical random site tensors (QR of complex
    Gaussians) at the largest ranks for (n, chi), with decaying positive lambda of unit
    norm per bond. The lambda are not the Schmidt numbers of this state."""
    rng = np.random.default_rng(40_000 + seed)
    r = [1] + full_ranks(n, chi) + [1]
    B = []
    for k in range(n):
        g = rng.normal(size=(2 * r[k + 1], r[k])) + 1j * rng.normal(size=(2 * r[k + 1], r[k]))
        q, _ = np.linalg.qr(g)
        B.append(q.conj().T.reshape(r[k], 2, r[k + 1]))
    lam = []
    for b in range(n - 1):
        l = np.sort(np.exp(-np.arange(r[b + 1]) / 8.0) * rng.uniform(0.5, 1.0, size=r[b + 1]))[::-1]
        lam.append(l / np.linalg.norm(l))
    return B, lam


def mps_inspired_bonds(n):
    """Bond pattern of the MPS-inspired circuit (unitaries that each entangle four
    consecutive qubits, swept along the chain): for q = 0 .. n-4 a block of five two-site
    gates on bonds q, q+1, q+2, q+1, q, i.e. one unitary on qubits q..q+3."""
    return [b for q in range(n - 3) for b in (q, q + 1, q + 2, q + 1, q)]


def brickwork_bonds(n, layers):
    """Bonds of a brickwork of two-site gates on neighbouring qubits: even bonds, then odd
    bonds, repeated."""
    out = []
    for layer in range(layers):
        out += list(range(layer % 2, n - 1, 2))
    return out


def random_gate_matrices(count, seed):
    """count complex Gaussian 4x4 matrices (the caller orthonormalises them, e.g. by QR)."""
    rng = np.random.default_rng(50_000 + seed)
    return rng.normal(size=(count, 4, 4)) + 1j * rng.normal(size=(count, 4, 4))
