"""Pins of the CPU oracle against facts fixed outside it.

Every check here compares the oracle with something other than itself: the
Pauli matrices' textbook products, a brute-force Fock-space construction that
never touches Pauli algebra, closed forms (Hartree-Fock energy, Eckart-Young
optimal truncation), exact statevectors, finite differences, counts printed in
the paper (Sec. III-D: 15 Pauli strings and 120 ansatz gates for H2), and a few
planted mistakes that the pins must catch.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import circuit, fock, grad, mps, pauli, sv, ucc
from paper_2207_03711_gb300 import synthetic as syn

RNG = np.random.default_rng(1234)


def rand_state(n, rng=RNG):
    v = rng.normal(size=2 ** n) + 1j * rng.normal(size=2 ** n)
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------- Pauli algebra
def test_pauli_products_match_textbook():
    # XY = iZ, YZ = iX, ZX = iY, and squares are the identity
    for a, b, c in [(1, 2, 3), (2, 3, 1), (3, 1, 2)]:
        assert pauli.PROD_CODE[a, b] == c and pauli.PROD_IPOW[a, b] == 1
        assert pauli.PROD_CODE[b, a] == c and pauli.PROD_IPOW[b, a] == 3
        assert pauli.PROD_CODE[a, a] == 0 and pauli.PROD_IPOW[a, a] == 0


def test_string_action_two_routes():
    n = 5
    for _ in range(10):
        code = RNG.integers(0, 4, size=n).astype(np.uint8)
        psi = rand_state(n)
        assert np.allclose(pauli.string_matrix(code) @ psi, pauli.apply_string(code, psi), atol=1e-14)


# ---------------------------------------------------------------- Jordan-Wigner vs Fock space
@pytest.mark.parametrize("m", [2, 3, 4])
def test_jw_equals_fock_space_hamiltonian(m):
    h, g = syn.random_integrals(m, 11 + m)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g, e_core=0.7)
    Hj = pauli.sum_matrix(codes, coeffs)
    Hf = fock.fock_hamiltonian(h, g, e_core=0.7)
    assert np.abs(Hj - Hf).max() < 1e-12


H2 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "h2_structure.json")))


def test_h2_has_15_strings():
    """Sec. III-D: the 4-qubit H2 Hamiltonian has 15 Pauli strings (tests/golden)."""
    for seed in range(3):
        h, g = syn.h2_shaped_integrals(seed)
        codes, _ = pauli.jordan_wigner_hamiltonian(h, g)
        assert len(codes) == H2["pauli_strings"]


def test_string_counts_8q_and_24q():
    h, g = syn.random_integrals(4, 0)
    assert len(pauli.jordan_wigner_hamiltonian(h, g)[0]) == 361


# ---------------------------------------------------------------- HF closed form
@pytest.mark.parametrize("m,ne", [(2, 2), (3, 2), (4, 4), (4, 2)])
def test_hf_energy_closed_form(m, ne):
    h, g = syn.random_integrals(m, 5)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    e_sv, _ = sv.energy(sv.hf_state(2 * m, ne), codes, coeffs)
    e_cf = fock.hf_energy(h, g, ne)
    Hf = fock.fock_hamiltonian(h, g)
    assert abs(e_sv - e_cf) < 1e-12
    assert abs(Hf[(1 << ne) - 1, (1 << ne) - 1] - e_cf) < 1e-12
    # theta = 0 through the truncated-MPS oracle as well
    st = mps.hf_mps(2 * m, ne)
    assert abs(mps.energy(st, codes, coeffs)[0] - e_cf) < 1e-12


# ---------------------------------------------------------------- UCCSD structure
def test_uccsd_counts():
    _, _, _, exc = ucc.uccsd_rotations(8, 4)
    assert len(exc) == 26
    rc, _, _, exc = ucc.uccsd_rotations(24, 12)
    assert len(exc) == 1818 and len(rc) == 14112


def test_h2_double_is_120_native_gates():
    """Sec. III-D: the H2 ansatz circuit has 120 gates, 8 exponentials x 15 (tests/golden);
    the reference state takes 2 X gates."""
    ex = ("d", (0, 1, 2, 3))
    codes, c = ucc.generator_strings(ex, H2["n_qubits"])
    assert len(codes) == H2["exponentials"]
    per = [len(circuit.native_gates(code, 0.3)) for code in codes]
    assert all(k == H2["gates_per_exponential"] for k in per)
    assert sum(per) == H2["ansatz_gates"]
    assert int(np.sum(sv.hf_state(H2["n_qubits"], H2["n_electrons"]) != 0)) == 1
    assert H2["n_electrons"] == H2["reference_x_gates"]


@pytest.mark.parametrize("n,ne", [(6, 2), (8, 4)])
def test_excitation_exponential_equals_fermionic_expm(n, ne):
    """prod_k exp(i theta c_k P_k) == expm(theta (tau - tau+)) with tau built in Fock space."""
    for ex in ucc.excitations(n, ne)[::3]:
        kind, idx = ex
        if kind == "s":
            i, a = idx
            tau = fock.operator_matrix(n, [(a, True), (i, False)])
        else:
            i, j, a, b = idx
            tau = fock.operator_matrix(n, [(a, True), (b, True), (i, False), (j, False)])
        theta = 0.37
        ref = scipy.linalg.expm(theta * (tau - tau.T))
        codes, c = ucc.generator_strings(ex, n)
        # the strings commute
        mats = [pauli.string_matrix(code) for code in codes]
        for A in mats:
            for B in mats:
                assert np.abs(A @ B - B @ A).max() < 1e-14
        U = np.eye(2 ** n, dtype=complex)
        for M, ck in zip(mats, c):
            U = (np.cos(theta * ck) * np.eye(2 ** n) + 1j * np.sin(theta * ck) * M) @ U
        assert np.abs(U - ref).max() < 1e-12


# ---------------------------------------------------------------- gate compiler
@pytest.mark.parametrize("n", [4, 7])
def test_compiled_rotation_equals_definition(n):
    for _ in range(25):
        code = RNG.integers(0, 4, size=n).astype(np.uint8)
        if not code.any():
            continue
        phi = RNG.uniform(-3, 3)
        psi = rand_state(n)
        ref = np.cos(phi / 2) * psi - 1j * np.sin(phi / 2) * pauli.apply_string(code, psi)
        nat = circuit.apply_native_sv(psi, circuit.native_gates(code, phi), n)
        fused = psi
        gates = circuit.two_site_gates(code, phi, n)
        S = np.nonzero(code)[0]
        if len(S) > 1:
            assert len(gates) == 2 * (S[-1] - S[0]) - 1
        for b, U in gates:
            assert np.abs(U.conj().T @ U - np.eye(4)).max() < 1e-14
            fused = circuit.apply_two_site_sv(fused, b, U, n)
        assert np.abs(nat - ref).max() < 1e-13
        assert np.abs(fused - ref).max() < 1e-13


def test_uccsd_8q_two_site_gate_count():
    rc, rp, rs, exc = ucc.uccsd_rotations(8, 4)
    gates = circuit.compile_circuit(rc, rp, rs, np.zeros(len(exc)), 8)
    assert len(gates) == 1568


# ---------------------------------------------------------------- c1 vs c2 and invariants
@pytest.fixture(scope="module")
def uccsd8():
    n, ne = 8, 4
    h, g = syn.random_integrals(4, 0)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    rc, rp, rs, exc = ucc.uccsd_rotations(n, ne)
    theta = syn.random_amplitudes(len(exc), 0)
    psi = sv.run_ansatz(n, ne, rc, rp, rs, theta)
    st = mps.hf_mps(n, ne)
    dw = mps.apply_gates(st, circuit.compile_circuit(rc, rp, rs, theta, n), chi=16)
    return dict(n=n, ne=ne, h=h, g=g, codes=codes, coeffs=coeffs, rc=rc, rp=rp, rs=rs,
                theta=theta, psi=psi, st=st, dw=dw)


def test_untruncated_mps_equals_statevector(uccsd8):
    c = uccsd8
    assert c["dw"] < 1e-20
    psi2 = mps.to_statevector(c["st"])
    assert abs(np.vdot(c["psi"], psi2)) ** 2 >= 1 - 1e-12
    e1, ev1 = sv.energy(c["psi"], c["codes"], c["coeffs"])
    e2, ev2 = mps.energy(c["st"], c["codes"], c["coeffs"])
    assert abs(e1 - e2) < 1e-10
    assert np.abs(ev1 - ev2).max() < 1e-12


def test_invariants(uccsd8):
    c = uccsd8
    n = c["n"]
    assert abs(mps.norm2(c["st"]) - 1) < 1e-12
    _, ev = mps.energy(c["st"], c["codes"], c["coeffs"])
    assert np.abs(ev.imag).max() < 1e-12
    psi = c["psi"]
    assert abs(np.vdot(psi, fock.number_operator(n) @ psi).real - c["ne"]) < 1e-12
    assert abs(np.vdot(psi, fock.sz2_operator(n) @ psi).real) < 1e-12


def test_variational_bound(uccsd8):
    c = uccsd8
    Hf = fock.fock_hamiltonian(c["h"], c["g"])
    sec = fock.sector_indices(c["n"], c["ne"], 0)
    emin = np.linalg.eigvalsh(Hf[np.ix_(sec, sec)])[0]
    for seed in range(4):
        th = syn.random_amplitudes(len(c["theta"]), 100 + seed) * 10
        psi = sv.run_ansatz(c["n"], c["ne"], c["rc"], c["rp"], c["rs"], th)
        assert sv.energy(psi, c["codes"], c["coeffs"])[0] >= emin - 1e-10


def test_schmidt_values_untouched_bonds():
    n = 7
    st = mps.from_statevector(rand_state(n), n)
    before = [l.copy() for l in st.lam]
    U = scipy.linalg.expm(1j * (lambda a: a + a.conj().T)(RNG.normal(size=(4, 4)) + 1j * RNG.normal(size=(4, 4))))
    mps.apply_two_site(st, 3, U, chi=64)
    for b in range(n - 1):
        if b != 3:
            assert np.allclose(st.lam[b], before[b], atol=1e-12)
    # single-site unitaries never change Schmidt numbers
    one = np.kron(scipy.linalg.expm(1j * np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, -0.5]])), np.eye(2))
    lam3 = st.lam[3].copy()
    mps.apply_two_site(st, 3, one, chi=64)
    assert np.allclose(st.lam[3], lam3, atol=1e-12)


# ---------------------------------------------------------------- truncation = Eckart-Young
@pytest.mark.parametrize("bond,chi", [(3, 5), (2, 3), (4, 7), (0, 1)])
def test_truncated_step_is_optimal(bond, chi):
    """From an exact canonical MPS, one Eq. (7)-(10) step with truncation must give the
    best rank-chi approximation of the full state across that bond."""
    n = 8
    psi = rand_state(n)
    st = mps.from_statevector(psi, n)
    U = scipy.linalg.expm(1j * (lambda a: a + a.conj().T)(RNG.normal(size=(4, 4)) + 1j * RNG.normal(size=(4, 4))))
    dw = mps.apply_two_site(st, bond, U, chi)
    out = mps.to_statevector(st)
    full = circuit.apply_two_site_sv(psi, bond, U, n)
    # dense optimal truncation across the bond (sites 0..bond | bond+1..n-1)
    t = full.reshape((2,) * n).transpose(tuple(range(n))[::-1]).reshape(2 ** (bond + 1), -1)
    u, s, vh = np.linalg.svd(t, full_matrices=False)
    k = min(chi, np.count_nonzero(s > 1e-13 * s[0]))
    best = (u[:, :k] * s[:k]) @ vh[:k]
    best = best.reshape((2,) * n).transpose(tuple(range(n))[::-1]).reshape(-1)
    assert np.abs(out - best).max() < 1e-12
    assert abs(dw - np.sum(s[k:] ** 2) / np.sum(s ** 2)) < 1e-12
    assert np.allclose(st.lam[bond], s[:k], atol=1e-12)
    # B_{n+1} <- V has orthonormal rows
    V = st.B[bond + 1].reshape(st.B[bond + 1].shape[0], -1)
    assert np.abs(V @ V.conj().T - np.eye(V.shape[0])).max() < 1e-12


def test_expectation_two_routes_on_truncated_state():
    n = 7
    st = mps.from_statevector(rand_state(n), n)
    for b in [1, 3, 5, 2]:
        U = scipy.linalg.expm(1j * (lambda a: a + a.conj().T)(RNG.normal(size=(4, 4))))
        mps.apply_two_site(st, b, U, chi=3)
    psi = mps.to_statevector(st)
    for _ in range(10):
        code = RNG.integers(0, 4, size=n).astype(np.uint8)
        assert abs(mps.expect_string(st, code) - np.vdot(psi, pauli.apply_string(code, psi))) < 1e-13


# ---------------------------------------------------------------- gradients
def test_parameter_shift_equals_finite_differences():
    n, ne = 6, 2
    h, g = syn.random_integrals(3, 2)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    rc, rp, rs, exc = ucc.uccsd_rotations(n, ne)
    theta = syn.random_amplitudes(len(exc), 3) * 5

    def e_of_angles(phis):
        psi = sv.hf_state(n, ne)
        for code, phi in zip(rc, phis):
            psi = sv.apply_rotation(psi, code, phi)
        return sv.energy(psi, codes, coeffs)[0]

    def e_of_theta(th):
        return e_of_angles(grad.rotation_angles(rp, rs, th))

    sel = [0, 2, len(exc) - 1]
    ps = grad.parameter_shift(e_of_angles, rp, rs, theta, sel)
    hstep = 1e-5
    for e, gval in zip(sel, ps):
        tp, tm = theta.copy(), theta.copy()
        tp[e] += hstep
        tm[e] -= hstep
        fd = (e_of_theta(tp) - e_of_theta(tm)) / (2 * hstep)
        assert abs(fd - gval) < 1e-7


# ---------------------------------------------------------------- planted mistakes
def test_planted_jw_sign_error_is_caught(monkeypatch):
    orig = pauli.ladder_branches

    def wrong(p, n, dagger):
        codes, coef = orig(p, n, dagger)
        return codes, coef.conj()          # a_p <-> a+_p mix-up
    monkeypatch.setattr(pauli, "ladder_branches", wrong)
    h, g = syn.random_integrals(2, 3)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    assert np.abs(pauli.sum_matrix(codes, coeffs) - fock.fock_hamiltonian(h, g)).max() > 1e-3


def test_planted_missing_lambda_is_caught(monkeypatch):
    monkeypatch.setattr(mps, "left_lambda", lambda st, site: np.ones(st.B[site].shape[0]))
    with pytest.raises(AssertionError):
        test_truncated_step_is_optimal(3, 5)


def test_planted_basis_change_error_is_caught(monkeypatch):
    monkeypatch.setattr(circuit, "RX90", circuit.RX90.conj().T)
    with pytest.raises(AssertionError):
        test_compiled_rotation_equals_definition(4)


def _fold_single_qubit_gates(native):
    """Fold every single-qubit gate into the next two-qubit gate touching its qubit (the
    previous one if none follows); two-qubit gates stay separate."""
    twoq = [i for i, g in enumerate(native) if g[0] == "2q"]
    mats = {i: native[i][2].copy() for i in twoq}
    for i, g in enumerate(native):
        if g[0] != "1q":
            continue
        _, q, u = g
        nxt = [j for j in twoq if j > i and native[j][1] in (q, q - 1)]
        prv = [j for j in twoq if j < i and native[j][1] in (q, q - 1)]
        j = nxt[0] if nxt else prv[-1]
        b = native[j][1]
        op = np.kron(u, circuit.I2) if b == q else np.kron(circuit.I2, u)
        mats[j] = mats[j] @ op if nxt else op @ mats[j]
    return [(native[j][1], mats[j]) for j in twoq]


def test_single_qubit_fusion_keeps_truncated_result():
    """Single-qubit unitaries never change Schmidt values, so folding them into two-qubit
    gates leaves a truncated evolution unchanged (lambda on every bond, <P>)."""
    n, chi = 8, 3
    rng = np.random.default_rng(11)
    st_a = mps.random_canonical(n, syn.full_ranks(n, chi), syn.random_mps_gaussians(n, syn.full_ranks(n, chi), 2))
    st_b = st_a.copy()
    codes = rng.integers(0, 4, size=(6, n)).astype(np.uint8)
    codes[:, 2] = 1                                   # every string has support
    for code in codes:
        phi = rng.uniform(-1, 1)
        native = circuit.native_gates(code, phi)
        for g in native:
            if g[0] == "1q":
                _, q, u = g
                st_a.B[q] = np.einsum("st,atb->asb", u, st_a.B[q])
            else:
                mps.apply_two_site(st_a, g[1], g[2], chi)
        for b, U in _fold_single_qubit_gates(native):
            mps.apply_two_site(st_b, b, U, chi)
    for la, lb in zip(st_a.lam, st_b.lam):
        assert len(la) == len(lb) and np.abs(la - lb).max() <= 1e-10
    probe = rng.integers(0, 4, size=(20, n)).astype(np.uint8)
    ea = np.array([mps.expect_string(st_a, c) for c in probe])
    eb = np.array([mps.expect_string(st_b, c) for c in probe])
    assert np.abs(ea - eb).max() <= 1e-10


# ---------------------------------------------------------------- random canonical MPS
@pytest.mark.parametrize("n,chi,seed", [(6, 4, 0), (8, 8, 1), (10, 5, 2), (9, 16, 3)])
def test_random_canonical_has_exact_schmidt_numbers(n, chi, seed):
    """random_canonical must return a right-canonical MPS of unit norm whose lambda on
    every bond are the Schmidt numbers of the state it represents: the singular values
    of the dense amplitudes reshaped across that bond (LAPACK SVD of the statevector,
    a route that shares nothing with the QR + eigh construction)."""
    ranks = syn.full_ranks(n, chi)
    st = mps.random_canonical(n, ranks, syn.random_mps_gaussians(n, ranks, seed))
    # every site right-canonical: sum_i B^i B^{i+} = I
    for k, Bk in enumerate(st.B):
        E = sum(Bk[:, i, :] @ Bk[:, i, :].conj().T for i in range(2))
        assert np.abs(E - np.eye(Bk.shape[0])).max() < 1e-12, k
    psi = mps.to_statevector(st)
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-12
    t = psi.reshape((2,) * n).transpose(tuple(range(n))[::-1]).reshape(-1)   # site 0 slowest
    for b in range(n - 1):
        s = np.linalg.svd(t.reshape(2 ** (b + 1), -1), compute_uv=False)
        r = len(st.lam[b])
        assert r == ranks[b]
        assert np.abs(st.lam[b] - s[:r]).max() < 1e-12, b
        assert np.all(s[r:] < 1e-12)                  # nothing beyond the stored rank
        assert np.all(np.diff(st.lam[b]) <= 1e-15)    # descending


class _SqrtDropped:
    """numpy stand-in for the oracle module with sqrt replaced by the identity."""

    def __getattr__(self, name):
        return getattr(np, name)

    @staticmethod
    def sqrt(x):
        return x


def test_planted_squared_schmidt_numbers_are_caught(monkeypatch):
    monkeypatch.setattr(mps, "np", _SqrtDropped())
    with pytest.raises(AssertionError):
        test_random_canonical_has_exact_schmidt_numbers(8, 8, 1)


# ---------------------------------------------------------------- compensated summation
def test_neumaier_sum_on_known_cancellations():
    """Exact values: 1e16 + 1 - 1e16 = 1 (a plain sum gives 0), and 1 + 1e100 + 1 - 1e100
    = 2 (Kahan's variant gives 0); the compensation term's sign decides both."""
    assert sv.neumaier_sum([1e16, 1.0, -1e16]) == 1.0
    assert sv.neumaier_sum([1.0, 1e100, 1.0, -1e100]) == 2.0
    assert sv.neumaier_sum([]) == 0.0
    assert sv.neumaier_sum([0.1] * 10) == math.fsum([0.1] * 10)


def test_neumaier_sum_matches_correctly_rounded_sum():
    """Against math.fsum (the correctly rounded sum) on long ill-conditioned series: the
    compensated sum is within eps |S| + n eps^2 sum|x| of it (the textbook bound), while
    the plain running sum misses by orders of magnitude more."""
    rng = np.random.default_rng(7)
    eps = np.finfo(float).eps
    for trial in range(5):
        x = rng.normal(size=20000) * 10.0 ** rng.uniform(-8, 8, size=20000)
        x = np.concatenate([x, -x[rng.permutation(len(x))][:19990]])     # heavy cancellation
        x = list(x[rng.permutation(len(x))])
        exact = math.fsum(x)
        bound = 2 * eps * abs(exact) + len(x) * eps ** 2 * sum(abs(v) for v in x)
        assert abs(sv.neumaier_sum(x) - exact) <= bound
        naive = 0.0
        for v in x:
            naive += v
        assert abs(naive - exact) > 100 * bound     # the series really needs compensation
