"""Brute-force Fock-space Hamiltonian and the Hartree-Fock energy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

This builds the matrix of Eq. (1), Sec. II-A, directly in the occupation-number
basis by acting with creation/annihilation operators on bit strings and counting
fermionic signs. It uses no Pauli algebra, so it pins ``oracle.pauli`` (the
Jordan-Wigner map of Eq. (2)) from outside.

Basis: index b, bit q of b = occupation of spin orbital q (= qubit q), interleaved
spin p = 2k + s. Sign rule: a_p and a+_p pick up (-1)^(number of occupied orbitals
with index < p), which is the ordering in which the Jordan-Wigner Z strings of the
chosen convention run.
"""
import numpy as np


def _popcount_table(n):
    return np.array([bin(i).count("1") for i in range(2 ** n)], dtype=np.int64)


def _annihilate(states, amp, p, pc):
    occ = (states >> p) & 1
    sign = 1 - 2 * (pc[states & ((1 << p) - 1)] & 1)
    return states ^ (1 << p), amp * sign * occ


def _create(states, amp, p, pc):
    empty = 1 - ((states >> p) & 1)
    sign = 1 - 2 * (pc[states & ((1 << p) - 1)] & 1)
    return states ^ (1 << p), amp * sign * empty


def fock_hamiltonian(h, eri, e_core=0.0):
    """Dense 2^n x 2^n matrix of Eq. (1) with chemist-order (pq|rs), n = 2m qubits."""
    m = h.shape[0]
    n = 2 * m
    dim = 2 ** n
    pc = _popcount_table(n)
    basis = np.arange(dim, dtype=np.int64)
    H = np.zeros((dim, dim))
    H[basis, basis] += e_core
    for p in range(n):
        for q in range(n):
            if p % 2 != q % 2 or h[p // 2, q // 2] == 0.0:
                continue
            st, a = _annihilate(basis, np.ones(dim), q, pc)
            st, a = _create(st, a, p, pc)
            nz = a != 0
            np.add.at(H, (st[nz], basis[nz]), h[p // 2, q // 2] * a[nz])
    for p in range(n):
        for q in range(n):
            if p % 2 != q % 2:
                continue
            for r in range(n):
                for s in range(n):
                    if r % 2 != s % 2:
                        continue
                    g = eri[p // 2, q // 2, r // 2, s // 2]
                    if g == 0.0:
                        continue
                    # a+_p a+_r a_s a_q |b>: rightmost operator acts first
                    st, a = _annihilate(basis, np.ones(dim), q, pc)
                    st, a = _annihilate(st, a, s, pc)
                    st, a = _create(st, a, r, pc)
                    st, a = _create(st, a, p, pc)
                    nz = a != 0
                    np.add.at(H, (st[nz], basis[nz]), 0.5 * g * a[nz])
    return H


def sector_indices(n, n_electrons, sz2=0):
    """Basis indices with the given electron count and 2*S_z (alpha = even qubits)."""
    pc = _popcount_table(n)
    b = np.arange(2 ** n)
    alpha = sum(((b >> q) & 1) for q in range(0, n, 2))
    beta = sum(((b >> q) & 1) for q in range(1, n, 2))
    return b[(pc[b] == n_electrons) & ((alpha - beta) == sz2)]


def hf_energy(h, eri, n_electrons, e_core=0.0):
    """Closed-form energy of the determinant with spin orbitals 0..N_e-1 occupied.

    E_HF = sum_{i in occ} h_ii + 1/2 sum_{i,j in occ} [(ii|jj) - delta_{s_i s_j} (ij|ji)]
    (spin-orbital indices; spatial integrals indexed by i // 2).
    """
    occ = list(range(n_electrons))
    e = e_core
    for i in occ:
        e += h[i // 2, i // 2]
    for i in occ:
        for j in occ:
            e += 0.5 * eri[i // 2, i // 2, j // 2, j // 2]
            if i % 2 == j % 2:
                e -= 0.5 * eri[i // 2, j // 2, j // 2, i // 2]
    return e


def operator_matrix(n, ops):
    """Dense matrix of a product of ladder operators [(p, dagger), ...] (leftmost first)."""
    pc = _popcount_table(n)
    dim = 2 ** n
    basis = np.arange(dim, dtype=np.int64)
    st, a = basis.copy(), np.ones(dim)
    for p, dag in reversed(ops):
        st, a = (_create if dag else _annihilate)(st, a, p, pc)
    out = np.zeros((dim, dim))
    nz = a != 0
    np.add.at(out, (st[nz], basis[nz]), a[nz])
    return out


def number_operator(n):
    pc = _popcount_table(n)
    return np.diag(pc.astype(float))


def sz2_operator(n):
    """2 S_z = N_alpha - N_beta (alpha on even qubits)."""
    b = np.arange(2 ** n)
    alpha = sum(((b >> q) & 1) for q in range(0, n, 2))
    beta = sum(((b >> q) & 1) for q in range(1, n, 2))
    return np.diag((alpha - beta).astype(float))
