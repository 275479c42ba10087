"""UCCSD excitations and their Pauli generators.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages followed:
  * Eq. (3), Sec. II-A: |Psi(theta)> = exp(T - T+) |Phi_0>.
  * Eq. (4), Sec. II-A: T = sum theta^a_i a+_a a_i + 1/4 sum theta^ab_ij a+_a a+_b a_i a_j.
  * Sec. II-A (end): the ansatz is implemented by a (first-order) Suzuki-Trotter
    product of exponentials, i.e. gates.
  * Sec. III-D: |Phi_0> is prepared by X gates on the first N_e qubits.

Readings where the paper is silent: spin-conserving, non-spin-adapted excitations with one
amplitude per i<j, a<b; tau = a+_a a_i (singles) and tau = a+_a a+_b a_i a_j
(doubles); order: all singles by (i, a), then all doubles by ((i, j), (a, b)).
Under Jordan-Wigner, tau - tau+ = i sum_k c_k P_k with real c_k and mutually
commuting P_k; the strings are taken in increasing (x-mask, z-mask) order, and
exp(theta (tau - tau+)) = prod_k exp(i theta c_k P_k) exactly. As a Pauli
rotation exp(-i phi P / 2) that is phi = scale * theta with scale = -2 c_k.
"""
import numpy as np

from . import pauli


def excitations(n_qubits, n_electrons):
    """Canonical list of ('s', (i, a)) and ('d', (i, j, a, b)) excitations."""
    occ = range(n_electrons)
    vir = range(n_electrons, n_qubits)
    out = []
    for i in occ:
        for a in vir:
            if i % 2 == a % 2:
                out.append(("s", (i, a)))
    for i in occ:
        for j in occ:
            if j <= i:
                continue
            for a in vir:
                for b in vir:
                    if b <= a:
                        continue
                    if (i % 2) + (j % 2) == (a % 2) + (b % 2):
                        out.append(("d", (i, j, a, b)))
    return out


def generator_strings(exc, n):
    """Pauli strings and real c_k of tau - tau+ = i sum_k c_k P_k, in (x, z)-mask order."""
    kind, idx = exc
    one = np.ones(1)
    if kind == "s":
        i, a = idx
        c1, k1 = pauli.ladder_product([(np.array([a]), True), (np.array([i]), False)], one, n)
        c2, k2 = pauli.ladder_product([(np.array([i]), True), (np.array([a]), False)], one, n)
    else:
        i, j, a, b = idx
        c1, k1 = pauli.ladder_product([(np.array([a]), True), (np.array([b]), True),
                                       (np.array([i]), False), (np.array([j]), False)], one, n)
        # (a+_a a+_b a_i a_j)+ = a+_j a+_i a_b a_a
        c2, k2 = pauli.ladder_product([(np.array([j]), True), (np.array([i]), True),
                                       (np.array([b]), False), (np.array([a]), False)], one, n)
    codes, coeffs = pauli.combine(np.concatenate([c1, c2]), np.concatenate([k1, -k2]))
    assert np.all(np.abs(coeffs.real) < 1e-14), "generator is not anti-Hermitian"
    c = coeffs.imag
    keys = [pauli.masks(code) for code in codes]
    order = sorted(range(len(keys)), key=lambda t: keys[t])
    return codes[order], c[order]


def uccsd_rotations(n_qubits, n_electrons):
    """All Pauli rotations of the Trotterised UCCSD ansatz, in application order.

    Returns (codes (R, n) uint8, param_idx (R,) int, scale (R,) float): rotation r
    is exp(-i * scale[r] * theta[param_idx[r]] / 2 * P_r). Also returns the
    excitation list.
    """
    exc = excitations(n_qubits, n_electrons)
    codes, pidx, scale = [], [], []
    for e, ex in enumerate(exc):
        cs, c = generator_strings(ex, n_qubits)
        for code, ck in zip(cs, c):
            codes.append(code)
            pidx.append(e)
            scale.append(-2.0 * ck)
    return (np.array(codes, dtype=np.uint8).reshape(-1, n_qubits), np.array(pidx, dtype=np.int64),
            np.array(scale), exc)
