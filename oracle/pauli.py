"""Pauli-string algebra and the Jordan-Wigner map, written out plainly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages followed:
  * Eq. (1), Sec. II-A: the second-quantised electronic Hamiltonian
    H = sum_pq h^p_q a+_p a_q + 1/2 sum_pqrs g^pq_rs a+_p a+_q a_r a_s.
  * Eq. (2), Sec. II-A: after a Jordan-Wigner mapping H is a real-weighted sum of
    Pauli strings P in {I, X, Y, Z}^(x)n and E = sum_i a_i <P_i>.
  * Sec. III-C: H = sum_i a_i P_i with each P_i an n-qubit tensor product.

Readings where the paper is silent:
  * Integrals are in chemist order (pq|rs); with interleaved spin orbitals
    p = 2k + s the Hamiltonian is
        H = sum_{pq,s} h_pq a+_{ps} a_{qs}
          + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}  (+ e_core).
  * Jordan-Wigner convention: a_p = Z_0 ... Z_{p-1} (X_p + i Y_p) / 2, so qubit
    value 1 means "occupied" and Y = [[0, -i], [i, 0]].

Representation: a Pauli sum is a pair (codes, coeffs); ``codes`` is a
(T, n) uint8 array with 0=I, 1=X, 2=Y, 3=Z per site (site q = qubit q) and
``coeffs`` a length-T complex array. Products are taken site by site with a
single-qubit product rule that is *derived* here from the 2x2 matrices.
"""
import numpy as np

I2 = np.eye(2, dtype=complex)
SIGMA = np.array([
    I2,
    np.array([[0, 1], [1, 0]], dtype=complex),
    np.array([[0, -1j], [1j, 0]], dtype=complex),
    np.array([[1, 0], [0, -1]], dtype=complex),
])


def _derive_single_qubit_products():
    """sigma_a @ sigma_b = i**k * sigma_c; returns (c, k) tables by matrix search."""
    out_c = np.zeros((4, 4), dtype=np.uint8)
    out_k = np.zeros((4, 4), dtype=np.int64)
    for a in range(4):
        for b in range(4):
            m = SIGMA[a] @ SIGMA[b]
            found = False
            for c in range(4):
                for k in range(4):
                    if np.allclose(m, (1j ** k) * SIGMA[c]):
                        out_c[a, b], out_k[a, b], found = c, k, True
            assert found
    return out_c, out_k


PROD_CODE, PROD_IPOW = _derive_single_qubit_products()


def string_matrix(code):
    """Dense 2^n x 2^n matrix of one Pauli string; qubit q is bit q of the index.

    Built with Kronecker products (site n-1 is the most significant factor), so
    it is an independent check of the site-wise product rule.
    """
    m = np.ones((1, 1), dtype=complex)
    for c in code:           # site 0 first, ends up least significant
        m = np.kron(SIGMA[int(c)], m)
    return m


def sum_matrix(codes, coeffs):
    n = codes.shape[1]
    out = np.zeros((2 ** n, 2 ** n), dtype=complex)
    for code, c in zip(codes, coeffs):
        out += c * string_matrix(code)
    return out


def ladder_branches(p, n, dagger):
    """a_p (or a+_p) under Jordan-Wigner as two Pauli strings.

    p: integer array (T,) of spin-orbital indices. Returns codes (T, 2, n)
    and coefficients (2,): a_p = Z..Z X_p / 2 + i Z..Z Y_p / 2, and the adjoint
    flips the sign of the Y branch.
    """
    p = np.asarray(p)
    T = p.shape[0]
    site = np.arange(n)[None, :]
    base = np.where(site < p[:, None], 3, 0).astype(np.uint8)
    codes = np.empty((T, 2, n), dtype=np.uint8)
    codes[:, 0, :] = np.where(site == p[:, None], 1, base)
    codes[:, 1, :] = np.where(site == p[:, None], 2, base)
    coef = np.array([0.5, -0.5j if dagger else 0.5j])
    return codes, coef


def multiply(codes_a, coef_a, codes_b, coef_b):
    """Row-wise product of two equally long lists of Pauli strings (a_t * b_t)."""
    c = PROD_CODE[codes_a, codes_b]
    k = PROD_IPOW[codes_a, codes_b].sum(axis=1) % 4
    return c, coef_a * coef_b * (1j ** k)


def ladder_product(ops, weight, n):
    """Expand sum_t weight_t * op1(t) op2(t) ... into Pauli strings.

    ops: list of (index array (T,), dagger flag) in operator order (leftmost first).
    Returns (codes (T * 2^k, n), coeffs).
    """
    T = weight.shape[0]
    codes = np.zeros((T, n), dtype=np.uint8)
    coef = weight.astype(complex)
    for idx, dag in ops:
        br_codes, br_coef = ladder_branches(idx, n, dag)
        cur_T = codes.shape[0] // T            # rows per original term so far
        # repeat each current row for both branches of this operator
        rep_codes = np.repeat(codes, 2, axis=0)
        rep_coef = np.repeat(coef, 2)
        op_codes = np.repeat(br_codes, cur_T, axis=0).reshape(T * cur_T, 2, n).reshape(-1, n)
        op_coef = np.tile(br_coef, T * cur_T)
        codes, coef = multiply(rep_codes, rep_coef, op_codes, op_coef)
    return codes, coef


def combine(codes, coeffs, rel_drop=1e-12):
    """Merge identical strings, drop |c| <= rel_drop * max|c|, sort lexicographically
    by (site 0, site 1, ...) with I < X < Y < Z (the prefix-trie order)."""
    codes = np.ascontiguousarray(codes)
    n = codes.shape[1]
    if codes.shape[0] == 0:
        return codes.reshape(0, n), np.zeros(0, dtype=complex)
    keys = codes.view(np.dtype((np.void, n))).ravel()
    uniq, inv = np.unique(keys, return_inverse=True)
    re = np.bincount(inv, weights=coeffs.real, minlength=uniq.shape[0])
    im = np.bincount(inv, weights=coeffs.imag, minlength=uniq.shape[0])
    out_c = re + 1j * im
    out_codes = np.frombuffer(uniq.tobytes(), dtype=np.uint8).reshape(-1, n).copy()
    mx = np.abs(out_c).max() if out_c.size else 0.0
    keep = np.abs(out_c) > rel_drop * mx
    out_codes, out_c = out_codes[keep], out_c[keep]
    order = np.lexsort(out_codes.T[::-1])
    return out_codes[order], out_c[order]


def jordan_wigner_hamiltonian(h, eri, e_core=0.0):
    """Eq. (1) -> Eq. (2): real-weighted Pauli sum of the electronic Hamiltonian.

    h: (m, m) one-electron integrals; eri: (m, m, m, m) chemist-order (pq|rs);
    interleaved spin orbitals p = 2k + s give n = 2m qubits.
    Returns (codes (T, n) uint8 in trie order, real coefficients (T,)).
    """
    m = h.shape[0]
    n = 2 * m
    so = np.arange(n)
    # one-body: a+_p a_q with equal spins
    P, Q = np.meshgrid(so, so, indexing="ij")
    P, Q = P.ravel(), Q.ravel()
    sel = (P % 2) == (Q % 2)
    P, Q = P[sel], Q[sel]
    w1 = h[P // 2, Q // 2]
    c1, k1 = ladder_product([(P, True), (Q, False)], w1, n)
    # two-body: 1/2 (pq|rs) a+_p a+_r a_s a_q with spin(p)=spin(q), spin(r)=spin(s)
    P, Q, R, S = [a.ravel() for a in np.meshgrid(so, so, so, so, indexing="ij")]
    sel = ((P % 2) == (Q % 2)) & ((R % 2) == (S % 2)) & (P != R) & (Q != S)
    P, Q, R, S = P[sel], Q[sel], R[sel], S[sel]
    w2 = 0.5 * eri[P // 2, Q // 2, R // 2, S // 2]
    c2, k2 = ladder_product([(P, True), (R, True), (S, False), (Q, False)], w2, n)
    codes = np.concatenate([c1, c2, np.zeros((1, n), dtype=np.uint8)])
    coeffs = np.concatenate([k1, k2, np.array([e_core], dtype=complex)])
    codes, coeffs = combine(codes, coeffs)
    assert np.all(np.abs(coeffs.imag) <= 1e-10 * max(1.0, np.abs(coeffs).max())), "H not Hermitian"
    return codes, coeffs.real.copy()


def masks(code):
    """(x-mask, z-mask) of one string as Python ints: bit q set when site q has
    X or Y (x) / Y or Z (z)."""
    x = z = 0
    for q, c in enumerate(code):
        c = int(c)
        if c in (1, 2):
            x |= 1 << q
        if c in (2, 3):
            z |= 1 << q
    return x, z


def apply_string(code, psi):
    """P|psi> for one Pauli string on a statevector (qubit q = bit q of the index).

    X|b> = |1-b>, Y|b> = i(-1)^b |1-b>, Z|b> = (-1)^b |b>, applied per qubit on a
    tensor view of psi.
    """
    n = len(code)
    t = psi.reshape((2,) * n)            # axis 0 is the most significant bit = qubit n-1
    for q, c in enumerate(code):
        c = int(c)
        if c == 0:
            continue
        ax = n - 1 - q
        if c == 1:
            t = np.flip(t, axis=ax)
        elif c == 2:
            t = np.flip(t, axis=ax)
            sl0 = [slice(None)] * n
            sl1 = [slice(None)] * n
            sl0[ax], sl1[ax] = 0, 1
            t = t.copy()
            t[tuple(sl0)] *= -1j       # new bit 0 came from old bit 1: -i
            t[tuple(sl1)] *= 1j        # new bit 1 came from old bit 0: +i
        else:
            t = t.copy()
            sl1 = [slice(None)] * n
            sl1[ax] = 1
            t[tuple(sl1)] *= -1
    return np.ascontiguousarray(t).reshape(-1)
