"""GPU parity: the CUDA path through the C ABI against the independent CPU oracle.

Truncated MPS evolution is chaotic under rounding (the oracle disagrees with
itself at the 1e-2 Ha level after tens of thousands of truncated steps when only
the LAPACK driver changes), so full-circuit energies are compared element-wise only
where the result is unique: untruncated circuits, circuit prefixes, single
truncated steps from oracle-made states, and the measurement stage on a fixed MPS.
Properties that hold at any size (Hartree-Fock energy at theta = 0, batch identity)
are checked at the full 24-qubit size.
"""
import numpy as np
import pytest
import scipy.linalg

import paper_2207_03711_gb300 as G
from oracle import circuit, fock, grad, mps, pauli, sv, ucc
from paper_2207_03711_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

FP64_E_TOL = 1e-9       # Ha, FP64 path vs oracle on a unique result
# Ha, mixed path (complex64 tensors, FP32 SVD with a compensated re-orthonormalisation)
# on the untruncated cases: the 1e-6 target at 8 qubits (1568 gates); at 10 qubits
# (~10^4 gates) complex64 storage alone already costs ~1e-6 (an FP64 SVD on complex64
# tensors reaches 1.1e-6 on these inputs), so the bound stated there is 3e-6
MIXED_E_TOL_8Q = 1e-6
MIXED_E_TOL_10Q = 3e-6


@pytest.fixture(scope="module", autouse=True)
def lib():
    G.build()
    return G.load_library()


def oracle_run(n, ne, chi, theta, rc, rp, rs, codes, coeffs, n_gates=None):
    st = mps.hf_mps(n, ne)
    gates = circuit.compile_circuit(rc, rp, rs, theta, n)
    if n_gates is not None:
        gates = gates[:n_gates]
    dw = mps.apply_gates(st, gates, chi)
    return st, dw


@pytest.fixture(scope="module")
def uccsd8():
    n, ne, chi = 8, 4, 16
    h, g = syn.random_integrals(4, 0)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    rc, rp, rs, exc = ucc.uccsd_rotations(n, ne)
    theta = syn.random_amplitudes(len(exc), 0)
    st, dw = oracle_run(n, ne, chi, theta, rc, rp, rs, codes, coeffs)
    e2, ev2 = mps.energy(st, codes, coeffs)
    psi = sv.run_ansatz(n, ne, rc, rp, rs, theta)
    e1, _ = sv.energy(psi, codes, coeffs)
    return dict(n=n, ne=ne, chi=chi, h=h, g=g, codes=codes, coeffs=coeffs, theta=theta, st=st,
                e1=e1, e2=e2, ev2=ev2, rc=rc, rp=rp, rs=rs)


# ------------------------------------- 8 qubits, 4 electrons, chi = 16 (exact)
def test_uccsd_8q_fp64_energy(uccsd8):
    c = uccsd8
    H = G.ham_jw_from_integrals(c["h"], c["g"])
    C = G.circ_uccsd(c["n"], c["ne"])
    M = G.mps_create(c["n"], c["chi"], G.MPS_FP64)
    e = G.vqe_energy(M, C, H, c["theta"])
    assert abs(e - c["e2"]) <= FP64_E_TOL
    assert abs(e - c["e1"]) <= FP64_E_TOL
    s = G.mps_get_stats(M)
    # the discarded fraction is (|M'|^2 - sum kept sigma^2) / |M'|^2 in FP64: ~1e-15 per gate
    assert s["discarded_weight"] < 1e-11 and s["n_svd_noconv"] == 0
    # per-term expectations on the GPU state against the oracle state
    vals = G.mps_expect_paulis(M, c["codes"])
    assert np.abs(vals - c["ev2"]).max() <= 1e-11
    # Schmidt numbers are gauge invariant
    r, sites, lams = G.mps_get_state(M)
    assert list(r) == c["st"].ranks()
    for a, b in zip(lams, c["st"].lam):
        assert np.abs(a - b).max() <= 1e-12


def test_uccsd_8q_mixed_energy(uccsd8):
    c = uccsd8
    H = G.ham_jw_from_integrals(c["h"], c["g"])
    C = G.circ_uccsd(c["n"], c["ne"])
    M = G.mps_create(c["n"], c["chi"], G.MPS_MIXED)
    e = G.vqe_energy(M, C, H, c["theta"])
    print(f"8-qubit mixed |dE| = {abs(e - c['e2']):.3e} Ha")
    assert abs(e - c["e2"]) <= MIXED_E_TOL_8Q


@pytest.mark.parametrize("prec", [G.MPS_FP64, G.MPS_MIXED])
def test_theta_zero_gives_hartree_fock_24q(prec):
    """Closed form at the full 24-qubit size: at theta = 0 every rotation is the
    identity, so E equals the determinant energy sum of integrals."""
    n, ne, chi = 24, 12, 64
    h, g = syn.random_integrals(12, 0)
    H = G.ham_jw_from_integrals(h, g)
    C = G.circ_uccsd(n, ne)
    M = G.mps_create(n, chi, prec)
    e = G.vqe_energy(M, C, H, np.zeros(C.n_params))
    tol = 1e-10 if prec == G.MPS_FP64 else 1e-4
    assert abs(e - fock.hf_energy(h, g, ne)) <= tol


@pytest.mark.parametrize("prec", [G.MPS_FP64, G.MPS_MIXED])
def test_untruncated_10q_matches_statevector(prec):
    n, ne, chi = 10, 4, 32
    h, g = syn.random_integrals(5, 2)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    rc, rp, rs, exc = ucc.uccsd_rotations(n, ne)
    theta = syn.random_amplitudes(len(exc), 2)
    psi = sv.run_ansatz(n, ne, rc, rp, rs, theta)
    e1, _ = sv.energy(psi, codes, coeffs)
    H = G.ham_jw_from_integrals(h, g)
    C = G.circ_uccsd(n, ne)
    M = G.mps_create(n, chi, prec)
    e = G.vqe_energy(M, C, H, theta)
    print(f"10q untruncated prec={prec} |dE| = {abs(e - e1):.3e} Ha")
    if prec == G.MPS_FP64:
        assert G.mps_get_stats(M)["discarded_weight"] < 1e-11
        assert abs(e - e1) <= FP64_E_TOL
    else:
        assert abs(e - e1) <= MIXED_E_TOL_10Q


# -------------------------------------------------- single truncated steps, 24 q
def _canon_state(n, chi, seed):
    r = syn.full_ranks(n, chi)
    return mps.random_canonical(n, r, syn.random_mps_gaussians(n, r, seed))


def _gate_set(n):
    C = G.circ_uccsd(n, n // 2)
    theta = syn.random_amplitudes(C.n_params, 7) * 10
    bond, U = G.circ_export_gates(C, theta)
    q, _ = np.linalg.qr(syn.random_unitary4(1))
    return [(11, U[np.nonzero(bond == 11)[0][0]]), (11, circuit.SWAP), (10, q),
            (12, np.kron(circuit.HAD, circuit.RX90) @ circuit.CNOT)]


@pytest.mark.parametrize("prec", [G.MPS_FP64, G.MPS_MIXED])
def test_truncated_step_parity_24q(prec):
    n, chi = 24, 64
    st0 = _canon_state(n, chi, 0)
    sample = pauli.jordan_wigner_hamiltonian(*syn.random_integrals(12, 0))[0]
    sample = sample[np.random.default_rng(0).choice(len(sample), 120, replace=False)]
    M = G.mps_create(n, chi, prec)
    lam_tol, blk_tol, ev_tol = (1e-12, 1e-10, 1e-10) if prec == G.MPS_FP64 else (2e-5, 2e-4, 2e-4)
    for bond, U in _gate_set(n):
        st = st0.copy()
        G.mps_set_state(M, st.B, st.lam)
        dw_gpu = G.mps_apply_gates(M, [bond], U[None])
        dw_or = mps.apply_two_site(st, bond, U, chi)
        r, sites, lams = G.mps_get_state(M)
        assert r[bond] == len(st.lam[bond])
        assert np.abs(lams[bond] - st.lam[bond]).max() <= lam_tol
        assert abs(dw_gpu - dw_or) <= max(lam_tol, 1e-12)
        # gauge-invariant truncated block diag(lambda_{n-1}) B_n B_{n+1}
        ll = st.lam[bond - 1]
        blk_g = ll[:, None, None, None] * np.einsum("aib,bjc->aijc", sites[bond], sites[bond + 1])
        blk_o = ll[:, None, None, None] * np.einsum("aib,bjc->aijc", st.B[bond], st.B[bond + 1])
        assert np.linalg.norm(blk_g - blk_o) / np.linalg.norm(blk_o) <= blk_tol
        ev_g = G.mps_expect_paulis(M, sample)
        ev_o = np.array([mps.expect_string(st, c) for c in sample]) / mps.norm2(st)
        assert np.abs(ev_g - ev_o).max() <= ev_tol


@pytest.mark.parametrize("prec", [G.MPS_FP64, G.MPS_MIXED])
def test_truncated_step_parity_chi128(prec):
    """chi = 128: the 256 x 256 M' of the middle bonds lives in global memory (the
    engine's second layout); single steps from an oracle-made canonical state."""
    n, chi = 16, 128
    st0 = _canon_state(n, chi, 4)
    rng = np.random.default_rng(5)
    M = G.mps_create(n, chi, prec)
    lam_tol, blk_tol = (1e-12, 1e-10) if prec == G.MPS_FP64 else (2e-5, 2e-4)
    for bond in (7, 6, 8):
        U, _ = np.linalg.qr(rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)))
        st = st0.copy()
        G.mps_set_state(M, st.B, st.lam)
        dw_gpu = G.mps_apply_gates(M, [bond], U[None])
        dw_or = mps.apply_two_site(st, bond, U, chi)
        r, sites, lams = G.mps_get_state(M)
        assert r[bond] == len(st.lam[bond])
        assert np.abs(lams[bond] - st.lam[bond]).max() <= lam_tol
        assert abs(dw_gpu - dw_or) <= max(lam_tol, 1e-12)
        ll = st.lam[bond - 1]
        blk_g = ll[:, None, None, None] * np.einsum("aib,bjc->aijc", sites[bond], sites[bond + 1])
        blk_o = ll[:, None, None, None] * np.einsum("aib,bjc->aijc", st.B[bond], st.B[bond + 1])
        assert np.linalg.norm(blk_g - blk_o) / np.linalg.norm(blk_o) <= blk_tol
        # the new right site is right-canonical: rows of V orthonormal
        V = sites[bond + 1].reshape(r[bond], -1)
        assert np.abs(V @ V.conj().T - np.eye(r[bond])).max() <= (1e-12 if prec == G.MPS_FP64 else 2e-6)


def test_measurement_parity_full_size():
    """All 29 737 strings of the 24-qubit Hamiltonian on a fixed chi = 64 MPS; a seeded
    sample of 400 terms is checked one by one against the oracle."""
    n, chi = 24, 64
    st = _canon_state(n, chi, 3)
    h, g = syn.random_integrals(12, 0)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    M = G.mps_create(n, chi, G.MPS_FP64)
    G.mps_set_state(M, st.B, st.lam)
    vals = G.mps_expect_paulis(M, codes)
    idx = np.random.default_rng(1).choice(len(codes), 400, replace=False)
    nrm = mps.norm2(st)
    ref = np.array([mps.expect_string(st, codes[i]) for i in idx]) / nrm
    assert np.abs(vals[idx] - ref).max() <= 1e-11
    assert np.abs(vals.imag).max() <= 1e-11
    # the energy of the loaded entangled state through the library's own trie
    # measurement and FP64 compensated sum, against the oracle's plain contraction of
    # every string
    H = G.ham_jw_from_integrals(h, g)
    e_gpu = G.mps_energy(M, H)
    e_ref, _ = mps.energy(st, codes, coeffs)
    print(f"24q chi64 loaded-state energy |dE| = {abs(e_gpu - e_ref):.3e} Ha")
    assert abs(e_gpu - e_ref) <= FP64_E_TOL
    H.close()


@pytest.mark.parametrize("prec,chi,ng", [(G.MPS_FP64, 24, 2500), (G.MPS_MIXED, 64, 3000)])
def test_prefix_parity_24q(prec, chi, ng):
    """The first gates of the 24-qubit circuit (ranks grow to the cap) agree."""
    n, ne = 24, 12
    h, g = syn.random_integrals(12, 0)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    rc, rp, rs, exc = ucc.uccsd_rotations(n, ne)
    theta = syn.random_amplitudes(len(exc), 0)
    st, dw = oracle_run(n, ne, chi, theta, rc, rp, rs, codes, coeffs, n_gates=ng)
    C = G.circ_uccsd(n, ne)
    bond, U = G.circ_export_gates(C, theta)
    M = G.mps_create(n, chi, prec)
    G.mps_reset(M, [1] * ne + [0] * (n - ne))
    dwg = G.mps_apply_gates(M, bond[:ng], U[:ng])
    r, sites, lams = G.mps_get_state(M)
    idx = np.random.default_rng(2).choice(len(codes), 200, replace=False)
    ev_g = G.mps_expect_paulis(M, codes[idx])
    ev_o = np.array([mps.expect_string(st, c) for c in codes[idx]]) / mps.norm2(st)
    print(f"prefix prec={prec} chi={chi} gates={ng} max|d<P>|={np.abs(ev_g - ev_o).max():.3e} "
          f"dw gpu={dwg:.3e} oracle={dw:.3e} ranks={list(r)}")
    if prec == G.MPS_FP64:
        assert list(r) == st.ranks()
        assert abs(dwg - dw) <= 1e-12
        for a, b in zip(lams, st.lam):
            assert np.abs(a - b).max() <= 1e-10
        assert np.abs(ev_g - ev_o).max() <= 1e-9
    else:
        # FP32 SVDs inside a truncated chain: over a long chain the differences grow into
        # the chaos band that FP64-vs-FP64 rounding changes already produce (a 1e-15
        # relative change of every M' moves truncated-chain energies by ~1e-2 Ha at 16
        # qubits, chi = 32); over these first 3000 gates they are still small (1.8e-6
        # measured on a GB300), and the bound keeps a wide margin above that
        assert np.abs(ev_g - ev_o).max() <= 1e-4


# ----------------------------------------------------------------- edge cases
@pytest.mark.parametrize("n,chi", [(2, 2), (2, 1), (5, 1), (6, 3), (7, 4)])
def test_edge_sizes_random_gates(n, chi):
    rng = np.random.default_rng(n * 10 + chi)
    bonds = rng.integers(0, n - 1, size=25).astype(np.int32)
    bonds[:2] = [0, n - 2]
    Us = np.array([np.linalg.qr(rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4)))[0] for _ in bonds])
    st = mps.hf_mps(n, 1)
    M = G.mps_create(n, chi, G.MPS_FP64)
    G.mps_reset(M, [1] + [0] * (n - 1))
    dw_o = 0.0
    ranks_ok = True
    for b, U in zip(bonds, Us):
        dw_o += mps.apply_two_site(st, int(b), U, chi)
    dw_g = G.mps_apply_gates(M, bonds, Us)
    r, sites, lams = G.mps_get_state(M)
    assert list(r) == st.ranks() and ranks_ok
    for a, b in zip(lams, st.lam):
        assert np.abs(a - b).max() <= 1e-11
    assert abs(dw_g - dw_o) <= 1e-11
    strings = rng.integers(0, 4, size=(30, n)).astype(np.uint8)
    strings[0] = 0
    ev_g = G.mps_expect_paulis(M, strings)
    ev_o = np.array([mps.expect_string(st, c) for c in strings]) / mps.norm2(st)
    assert np.abs(ev_g - ev_o).max() <= 1e-11


@pytest.mark.parametrize("prec,dust", [(G.MPS_MIXED, 1e-25), (G.MPS_FP64, 1e-170)])
def test_gate_on_entries_whose_squares_underflow(prec, dust):
    """Rounding dust in a sector that is empty in exact arithmetic can leave a column
    of M' whose entries are tiny but not zero, so small that their squares underflow:
    its norm comes out 0 while its leading entry is not. The reflector of the
    bidiagonalisation must take that column as zero (not divide by it), and the state
    must stay finite: |0>(|0> + i dust |1>) through three identity gates ends as |00>."""
    M = G.mps_create(2, 4, prec)
    s0 = np.array([1.0, 0.0], dtype=complex).reshape(1, 2, 1)
    s1 = np.array([1.0, 1j * dust], dtype=complex).reshape(1, 2, 1)
    G.mps_set_state(M, [s0, s1], [np.array([1.0])])
    G.mps_apply_gates(M, np.zeros(3, dtype=np.int32), np.tile(np.eye(4, dtype=complex), (3, 1, 1)))
    r, sites, lams = G.mps_get_state(M)
    assert all(np.all(np.isfinite(x)) for x in sites) and all(np.all(np.isfinite(x)) for x in lams)
    psi = np.einsum("aib,bjc->ij", sites[0], sites[1])
    assert abs(abs(psi[0, 0]) - 1.0) <= 1e-6
    assert np.abs(psi).ravel()[1:].max() <= 1e-6


def test_empty_circuit_and_duplicate_strings():
    n = 6
    C = G.circ_create(np.zeros((0, n), dtype=np.uint8), np.zeros(0, dtype=np.int32), np.zeros(0))
    occ = np.array([1, 1, 0, 1, 0, 0], dtype=np.uint8)
    G.circ_set_reference(C, occ)
    M = G.mps_create(n, 4, G.MPS_FP64)
    strings = np.array([[3, 0, 0, 0, 0, 0], [0, 0, 0, 0, 0, 0], [3, 0, 0, 0, 0, 0], [0, 0, 3, 3, 0, 0]],
                       dtype=np.uint8)
    H = G.ham_create(strings[[0, 1, 3]], [0.5, 2.0, -1.0])
    e = G.vqe_energy(M, C, H, None)
    # <Z_0> = -1, <Z_2 Z_3> = (+1)(-1) = -1
    assert abs(e - (0.5 * -1 + 2.0 + -1.0 * -1)) <= 1e-14
    vals = G.mps_expect_paulis(M, strings)
    assert np.allclose(vals, [-1, 1, -1, -1], atol=1e-14)


def test_batch_identity():
    """A result computed alone equals the same request computed in a batch."""
    n, ne, chi = 8, 4, 6   # chi < exact rank: truncation active
    h, g = syn.random_integrals(4, 1)
    H = G.ham_jw_from_integrals(h, g)
    C = G.circ_uccsd(n, ne)
    thetas = np.stack([syn.random_amplitudes(C.n_params, s) for s in range(5)])
    M = G.mps_create(n, chi, G.MPS_FP64, n_slots=5)
    batch = G.vqe_energy_batch(M, C, H, thetas)
    alone = np.array([G.vqe_energy(M, C, H, t) for t in thetas])
    assert np.array_equal(batch, alone)
    # and against the oracle (short circuit: unique result)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    rc, rp, rs, _ = ucc.uccsd_rotations(n, ne)
    for t, e in zip(thetas[:2], batch[:2]):
        st, _ = oracle_run(n, ne, chi, t, rc, rp, rs, codes, coeffs)
        assert abs(mps.energy(st, codes, coeffs)[0] - e) <= 1e-8


def test_gradient_parity():
    n, ne, chi = 6, 2, 8
    h, g = syn.random_integrals(3, 4)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    rc, rp, rs, exc = ucc.uccsd_rotations(n, ne)
    theta = syn.random_amplitudes(len(exc), 5) * 8
    sel = [0, 3, len(exc) - 1]

    def e_of_angles(phis):
        st = mps.hf_mps(n, ne)
        gates = []
        for code, phi in zip(rc, phis):
            gates += circuit.two_site_gates(code, phi, n)
        mps.apply_gates(st, gates, chi)
        return mps.energy(st, codes, coeffs)[0]

    ref = grad.parameter_shift(e_of_angles, rp, rs, theta, sel)
    H = G.ham_jw_from_integrals(h, g)
    C = G.circ_uccsd(n, ne)
    one = G.vqe_gradient(G.mps_create(n, chi, G.MPS_FP64, n_slots=1), C, H, theta, sel)
    assert np.abs(one - ref).max() <= 1e-9
    # shared-prefix forks: 4 slots (one rotation per wave) and 9 slots (four per wave)
    for slots in (4, 9):
        gg = G.vqe_gradient(G.mps_create(n, chi, G.MPS_FP64, n_slots=slots), C, H, theta, sel)
        assert np.abs(gg - one).max() <= 1e-13


def test_gradient_forks_match_restarts_under_truncation():
    # chi = 4 truncates: the forked route must still reproduce the from-scratch route
    n, ne, chi = 10, 4, 4
    h, g = syn.random_integrals(5, 6)
    H = G.ham_jw_from_integrals(h, g)
    C = G.circ_uccsd(n, ne)
    theta = syn.random_amplitudes(C.n_params, 7) * 6
    sel = [0, C.n_params // 2, C.n_params - 1]
    for prec, tol in ((G.MPS_FP64, 1e-13), (G.MPS_MIXED, 1e-6)):
        one = G.vqe_gradient(G.mps_create(n, chi, prec, n_slots=1), C, H, theta, sel)
        forked = G.vqe_gradient(G.mps_create(n, chi, prec, n_slots=7), C, H, theta, sel)
        assert np.abs(forked - one).max() <= tol * max(1.0, np.abs(one).max())


def test_state_roundtrip():
    n, chi = 9, 8
    st = _canon_state(n, chi, 5)
    M = G.mps_create(n, chi, G.MPS_FP64)
    G.mps_set_state(M, st.B, st.lam)
    r, sites, lams = G.mps_get_state(M)
    for a, b in zip(sites, st.B):
        assert np.array_equal(a, b)
    for a, b in zip(lams, st.lam):
        assert np.array_equal(a, b)


def test_vqe_loop_reaches_sector_ground_state():
    # 4 spin orbitals, 2 electrons: UCCSD spans the N = 2, Sz = 0 ground state, and
    # chi = 4 holds every state exactly, so the loop must reach the sector minimum
    from paper_2207_03711_gb300 import vqe
    n, ne, chi = 4, 2, 4
    h, g = syn.random_integrals(2, 1)
    Hf = fock.fock_hamiltonian(h, g)
    Hd = Hf.toarray() if hasattr(Hf, "toarray") else np.asarray(Hf)
    idx = fock.sector_indices(n, ne)
    e0 = np.linalg.eigvalsh(Hd[np.ix_(idx, idx)])[0]
    H = G.ham_jw_from_integrals(h, g)
    C = G.circ_uccsd(n, ne)
    M = G.mps_create(n, chi, G.MPS_FP64, n_slots=9)
    theta0 = syn.random_amplitudes(C.n_params, 2)
    theta, e, hist = vqe.minimize(M, C, H, theta0, iters=200, gtol=1e-9)
    assert e >= e0 - 1e-9                      # variational bound
    assert e - e0 <= 1e-8
    assert hist[-1][1] <= hist[0][1]


def test_fused_circuit_variant():
    """The fused gate list (circ_fuse_gates) is the same circuit: untruncated FP64
    energies and parameter-shift gradients equal the canonical list's and the oracle."""
    n, ne, chi = 8, 4, 16
    h, g = syn.random_integrals(4, 0)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    rc, rp, rs, _ = ucc.uccsd_rotations(n, ne)
    H = G.ham_jw_from_integrals(h, g)
    C0, C1 = G.circ_uccsd(n, ne), G.circ_uccsd(n, ne)
    assert G.circ_fuse_gates(C1) < G.circ_num_gates(C0)
    theta = syn.random_amplitudes(C0.n_params, 0)
    e_sv = sv.energy(sv.run_ansatz(n, ne, rc, rp, rs, theta), codes, coeffs)[0]
    M = G.mps_create(n, chi, G.MPS_FP64, n_slots=9)
    e0 = G.vqe_energy(M, C0, H, theta)
    e1 = G.vqe_energy(M, C1, H, theta)
    assert abs(e0 - e_sv) <= FP64_E_TOL and abs(e1 - e_sv) <= FP64_E_TOL
    sel = [0, 5, C0.n_params - 1]
    g0 = G.vqe_gradient(M, C0, H, theta, sel)
    g1 = G.vqe_gradient(M, C1, H, theta, sel)
    assert np.abs(g0 - g1).max() <= 1e-9


@pytest.mark.parametrize("prec,tol", [(G.MPS_FP64, FP64_E_TOL), (G.MPS_MIXED, MIXED_E_TOL_8Q)])
def test_ladder_cancellation_variant(prec, tol):
    """The ladder-cancelling gate list (circ_cancel_ladders, 943 instead of 1568 gates at
    8 qubits) is the same circuit: untruncated energies equal the oracle's within each
    precision's bound, and FP64 parameter-shift gradients equal the canonical list's."""
    n, ne, chi = 8, 4, 16
    h, g = syn.random_integrals(4, 0)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    rc, rp, rs, _ = ucc.uccsd_rotations(n, ne)
    H = G.ham_jw_from_integrals(h, g)
    C0, C1 = G.circ_uccsd(n, ne), G.circ_uccsd(n, ne)
    assert G.circ_cancel_ladders(C1) < 0.7 * G.circ_num_gates(C0)
    theta = syn.random_amplitudes(C0.n_params, 0)
    e_sv = sv.energy(sv.run_ansatz(n, ne, rc, rp, rs, theta), codes, coeffs)[0]
    M = G.mps_create(n, chi, prec, n_slots=9)
    e1 = G.vqe_energy(M, C1, H, theta)
    print(f"8q ladder-cancelled prec={prec} |dE| = {abs(e1 - e_sv):.3e} Ha")
    assert abs(e1 - e_sv) <= tol
    if prec == G.MPS_FP64:
        sel = [0, 5, C0.n_params - 1]
        g0 = G.vqe_gradient(M, C0, H, theta, sel)
        g1 = G.vqe_gradient(M, C1, H, theta, sel)
        assert np.abs(g0 - g1).max() <= 1e-9
