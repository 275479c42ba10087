"""Native-gate decomposition of Pauli rotations and two-site gate fusion.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages followed:
  * Sec. III-D (H2 example): each Trotter factor is a basis change, a CNOT ladder,
    an Rz carrying the variational parameter, the inverse ladder and the inverse
    basis change (4 + 3 + 1 + 3 + 4 = 15 native gates for a 4-qubit string; 120 for
    the 8 strings of H2's double excitation).
  * Sec. III-A: single-qubit gates are absorbed into two-qubit gates by gate fusion,
    and two-qubit gates act on nearest neighbours (bond n = sites n, n+1).

Readings where the paper does not draw the circuit, for exp(-i phi P / 2) with support S = {q : P_q != I},
lo = min S, hi = max S:
  * basis change B_q = H for X, Rx(pi/2) = exp(-i pi X / 4) for Y, none for Z, so
    that B_q P_q B_q^+ = Z;
  * the parity of S is carried upward bond by bond: at bond (b, b+1), b = lo..hi-1,
    a CNOT(b -> b+1) when b+1 is in S, otherwise a SWAP(b, b+1) that moves the
    carried parity across the identity qubit; Rz(phi) = diag(e^{-i phi/2}, e^{i phi/2})
    on hi; then the same hops in reverse order, then B_q^+;
  * fusion inside one rotation: B_q joins the first two-site gate touching q,
    B_q^+ the last one, and the up hop, Rz and down hop on bond (hi-1, hi) become
    one gate. A rotation thus compiles to 2 (hi - lo) - 1 two-site gates.
  * |S| = 1: the single-qubit rotation becomes one gate on bond (q, q+1), or
    (q-1, q) for the last qubit; |S| = 0 is a global phase and emits nothing.

Two-site gate matrices act on |i_b i_{b+1}> with row index 2 i_b + i_{b+1}.
"""
import numpy as np

I2 = np.eye(2, dtype=complex)
HAD = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
RX90 = (I2 - 1j * np.array([[0, 1], [1, 0]], dtype=complex)) / np.sqrt(2)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)


def rz(phi):
    return np.diag([np.exp(-0.5j * phi), np.exp(0.5j * phi)])


def basis_change(c):
    return {1: HAD, 2: RX90, 3: I2}[int(c)]


def native_gates(code, phi):
    """Unfused native gate list: ('1q', q, 2x2) and ('2q', b, 4x4, 'cnot'|'swap')."""
    S = [q for q, c in enumerate(code) if c != 0]
    if not S:
        return []
    lo, hi = S[0], S[-1]
    out = []
    for q in S:
        if code[q] in (1, 2):
            out.append(("1q", q, basis_change(code[q])))
    up = [("2q", b, CNOT, "cnot") if (b + 1) in S else ("2q", b, SWAP, "swap") for b in range(lo, hi)]
    out += up
    out.append(("1q", hi, rz(phi)))
    out += up[::-1]
    for q in S:
        if code[q] in (1, 2):
            out.append(("1q", q, basis_change(code[q]).conj().T))
    return out


def two_site_gates(code, phi, n):
    """Fused list of (bond, 4x4) for exp(-i phi P / 2), in application order."""
    S = [q for q, c in enumerate(code) if c != 0]
    if not S:
        return []
    B = {q: basis_change(code[q]) for q in S}
    if len(S) == 1:
        q = S[0]
        one = B[q].conj().T @ rz(phi) @ B[q]
        return [(q, np.kron(one, I2))] if q + 1 < n else [(q - 1, np.kron(I2, one))]
    lo, hi = S[0], S[-1]
    Sset = set(S)

    def hop(b):
        return CNOT if (b + 1) in Sset else SWAP

    gates = []
    for b in range(lo, hi - 1):                       # up ladder below the top bond
        pre = np.kron(B[lo] if b == lo else I2, B[b + 1] if (b + 1) in Sset else I2)
        gates.append((b, hop(b) @ pre))
    b = hi - 1                                        # top bond: up hop, Rz, down hop
    pre = np.kron(B[lo] if b == lo else I2, B[hi])
    post = np.kron(B[lo].conj().T if b == lo else I2, B[hi].conj().T)
    gates.append((b, post @ CNOT @ np.kron(I2, rz(phi)) @ CNOT @ pre))
    for b in range(hi - 2, lo - 1, -1):               # down ladder
        post = np.kron(B[lo].conj().T if b == lo else I2,
                       B[b + 1].conj().T if (b + 1) in Sset else I2)
        gates.append((b, post @ hop(b)))
    return gates


def compile_circuit(rot_codes, rot_pidx, rot_scale, theta, n):
    """Whole ansatz as a list of (bond, 4x4) two-site gates for parameters theta."""
    out = []
    for code, e, s in zip(rot_codes, rot_pidx, rot_scale):
        out += two_site_gates(code, s * theta[e], n)
    return out


def apply_two_site_sv(psi, bond, U, n):
    """Apply a two-site gate to a statevector (used only to pin the compiler)."""
    t = psi.reshape((2,) * n)
    ax_q, ax_q1 = n - 1 - bond, n - 2 - bond         # axes of qubits bond and bond+1
    G = U.reshape(2, 2, 2, 2)                         # [i_q, i_q1, i'_q, i'_q1]
    t = np.tensordot(G, t, axes=([2, 3], [ax_q, ax_q1]))
    t = np.moveaxis(t, [0, 1], [ax_q, ax_q1])
    return np.ascontiguousarray(t).reshape(-1)


def apply_one_site_sv(psi, q, g, n):
    t = psi.reshape((2,) * n)
    ax = n - 1 - q
    t = np.tensordot(g, t, axes=([1], [ax]))
    t = np.moveaxis(t, 0, ax)
    return np.ascontiguousarray(t).reshape(-1)


def apply_native_sv(psi, gates, n):
    for g in gates:
        if g[0] == "1q":
            psi = apply_one_site_sv(psi, g[1], g[2], n)
        else:
            psi = apply_two_site_sv(psi, g[1], g[2], n)
    return psi
