"""c1: exact statevector simulation of the Trotterised ansatz (no gates, no truncation).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper contrasts its MPS simulator with the brute-force state-vector approach
(Sec. II-A, Sec. III-A); here that approach is the exact reference. Qubit q is
bit q of the amplitude index.

  * Reference state (Sec. III-D): X gates on the first N_e qubits, i.e. the basis
    state with bits 0..N_e-1 set.
  * Each Pauli rotation exp(-i phi P / 2) = cos(phi/2) I - i sin(phi/2) P is
    applied by its definition.
  * Energy (Eq. 2, Sec. III-C): E = sum_i a_i <psi|P_i|psi>, summed in term order
    with Neumaier compensation; imaginary parts are returned for checking.
"""
import numpy as np

from . import pauli


def hf_state(n, n_electrons):
    psi = np.zeros(2 ** n, dtype=complex)
    psi[(1 << n_electrons) - 1] = 1.0
    return psi


def apply_rotation(psi, code, phi):
    return np.cos(phi / 2) * psi - 1j * np.sin(phi / 2) * pauli.apply_string(code, psi)


def run_ansatz(n, n_electrons, rot_codes, rot_pidx, rot_scale, theta):
    psi = hf_state(n, n_electrons)
    for code, e, s in zip(rot_codes, rot_pidx, rot_scale):
        psi = apply_rotation(psi, code, s * theta[e])
    return psi


def neumaier_sum(values):
    s = 0.0
    comp = 0.0
    for v in values:
        t = s + v
        if abs(s) >= abs(v):
            comp += (s - t) + v
        else:
            comp += (v - t) + s
        s = t
    return s + comp


def expectations(psi, codes):
    """<psi|P_i|psi> for every string (complex)."""
    return np.array([np.vdot(psi, pauli.apply_string(code, psi)) for code in codes])


def energy(psi, codes, coeffs):
    """E = sum_i a_i <P_i> / <psi|psi>; returns (E, per-term <P_i>)."""
    ev = expectations(psi, codes)
    norm = np.vdot(psi, psi).real
    return neumaier_sum(list(coeffs * ev.real)) / norm, ev / norm
