"""CPU tests of the C ABI: the library loads, exports every declared entry point,
and its host preprocessing (Jordan-Wigner, UCCSD, gate compiler, argument checks)
agrees with the independent oracle. No GPU is needed: these calls touch no device."""
import os
import re

import numpy as np
import pytest

import paper_2207_03711_gb300 as G
from oracle import circuit, pauli, sv, ucc
from paper_2207_03711_gb300 import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    G.build()
    return G.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mpsvqe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)) - {"if", "defined"}


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 28
    for name in names:
        assert hasattr(lib, name), name
        assert name in G.SIGNATURES, name


@pytest.mark.parametrize("m,seed", [(2, 0), (4, 0), (5, 3), (12, 0)])
def test_jw_matches_oracle(m, seed):
    h, g = syn.random_integrals(m, seed)
    H = G.ham_jw_from_integrals(h, g, 0.25)
    P, C = G.ham_get_terms(H)
    Po, Co = pauli.jordan_wigner_hamiltonian(h, g, 0.25)
    assert P.shape == Po.shape and (P == Po).all()
    assert np.abs(C - Co).max() <= 1e-12


def test_jw_is_deterministic():
    """The transform runs in parallel over fixed parts merged in a fixed order: two calls
    give the same strings and the same coefficient bits."""
    h, g = syn.random_integrals(10, 4)
    P1, C1 = G.ham_get_terms(G.ham_jw_from_integrals(h, g))
    P2, C2 = G.ham_get_terms(G.ham_jw_from_integrals(h, g))
    assert np.array_equal(P1, P2) and np.array_equal(C1, C2)


def test_h2_shaped_has_15_terms():
    h, g = syn.h2_shaped_integrals(1)
    assert G.ham_get_terms(G.ham_jw_from_integrals(h, g))[0].shape[0] == 15


@pytest.mark.parametrize("n,ne", [(4, 2), (8, 4), (10, 4), (24, 12)])
def test_uccsd_rotations_match_oracle(n, ne):
    C = G.circ_uccsd(n, ne)
    P, pidx, scale = G.circ_get_rotations(C)
    rc, rp, rs, exc = ucc.uccsd_rotations(n, ne)
    assert C.n_params == len(exc)
    assert (P == rc).all() and (pidx == rp).all()
    assert np.abs(scale - rs).max() <= 1e-15


def test_compiled_gates_match_oracle_uccsd():
    n, ne = 8, 4
    C = G.circ_uccsd(n, ne)
    theta = syn.random_amplitudes(C.n_params, 4)
    bond, U = G.circ_export_gates(C, theta)
    rc, rp, rs, _ = ucc.uccsd_rotations(n, ne)
    ref = circuit.compile_circuit(rc, rp, rs, theta, n)
    assert len(ref) == len(bond) == 1568
    assert all(b == r[0] for b, r in zip(bond, ref))
    assert max(np.abs(u - r[1]).max() for u, r in zip(U, ref)) <= 1e-14


def test_compiled_gates_general_rotations():
    rng = np.random.default_rng(5)
    n = 9
    codes = rng.integers(0, 4, size=(60, n)).astype(np.uint8)
    codes[0] = 0
    codes[1] = 0
    codes[1, 4] = 2          # single-qubit rotation
    codes[2] = 0
    codes[2, 8] = 1          # single-qubit rotation on the last qubit
    codes[3] = 0
    codes[3, [0, 8]] = [1, 3]  # long identity gap
    pidx = rng.integers(-1, 5, size=60).astype(np.int32)
    scale = rng.normal(size=60)
    theta = rng.normal(size=5)
    C = G.circ_create(codes, pidx, scale)
    bond, U = G.circ_export_gates(C, theta)
    ref = []
    for code, e, s in zip(codes, pidx, scale):
        phi = s * theta[e] if e >= 0 else s
        ref += circuit.two_site_gates(code, phi, n)
    assert len(ref) == len(bond)
    assert all(b == r[0] for b, r in zip(bond, ref))
    assert max(np.abs(u - r[1]).max() for u, r in zip(U, ref)) <= 1e-14


def test_ham_create_merges_and_sorts():
    P = np.array([[3, 0, 1], [0, 0, 0], [3, 0, 1], [1, 2, 0]], dtype=np.uint8)
    H = G.ham_create(P, [0.5, 1.0, 0.25, -2.0])
    Pq, Cq = G.ham_get_terms(H)
    assert (Pq == np.array([[0, 0, 0], [1, 2, 0], [3, 0, 1]])).all()
    assert np.allclose(Cq, [1.0, -2.0, 0.75])


def test_argument_errors_are_status_codes():
    with pytest.raises(G.MpsError) as e:
        G.circ_uccsd(4, 0)
    assert e.value.code == G.MPS_EINVAL
    with pytest.raises(G.MpsError):
        G.ham_create(np.array([[0, 7]], dtype=np.uint8), [1.0])
    with pytest.raises(G.MpsError):
        G.ham_jw_from_integrals(np.zeros((0, 0)), np.zeros((0, 0, 0, 0)))
    with pytest.raises(G.MpsError):
        G.circ_create(np.array([[0, 5, 1]], dtype=np.uint8), [0], [1.0])
    bad = np.array([[1.0, 2.0], [2.0, 1.0]])
    eri = np.zeros((2,) * 4)
    assert G.ham_get_terms(G.ham_jw_from_integrals(bad, eri))[0].shape[0] > 0


def test_estimate_bytes_host_only():
    """mps_estimate_bytes needs no GPU: it grows with slots, chi and precision, adds the
    circuit and Hamiltonian buffers, and rejects bad sizes."""
    G.load_library()
    base = G.mps_estimate_bytes(12, 16, G.MPS_MIXED, 1)
    assert base > 0
    assert G.mps_estimate_bytes(12, 16, G.MPS_MIXED, 4) > base
    assert G.mps_estimate_bytes(12, 32, G.MPS_MIXED, 1) > base
    assert G.mps_estimate_bytes(12, 16, G.MPS_FP64, 1) > base
    h, g = syn.random_integrals(6, 0)
    H = G.ham_jw_from_integrals(h, g)
    C = G.circ_uccsd(12, 6)
    full = G.mps_estimate_bytes(12, 16, G.MPS_MIXED, 1, C, H)
    assert full > G.mps_estimate_bytes(12, 16, G.MPS_MIXED, 1, C) > base
    # site tensors alone: sum of cap_{k-1} * 2 * cap_k complex64 entries
    caps = [1] + [min(16, 2 ** min(b + 1, 11 - b)) for b in range(11)] + [1]
    assert base >= 8 * sum(caps[k] * 2 * caps[k + 1] for k in range(12))
    with pytest.raises(G.MpsError):
        G.mps_estimate_bytes(12, 0, G.MPS_MIXED, 1)


def test_fused_gate_list_is_the_same_circuit():
    """circ_fuse_gates (a circuit-level variant): fewer gates, the same unitary. Checked
    by applying both gate lists exactly to a statevector and against the oracle's
    product of Pauli exponentials (no GPU)."""
    n, ne = 8, 4
    C = G.circ_uccsd(n, ne)
    theta = syn.random_amplitudes(C.n_params, 3) * 5
    b0, U0 = G.circ_export_gates(C, theta)
    ng = G.circ_fuse_gates(C)
    b1, U1 = G.circ_export_gates(C, theta)
    assert ng == len(b1) < len(b0)
    rc, rp, rs, _ = ucc.uccsd_rotations(n, ne)
    ref = sv.run_ansatz(n, ne, rc, rp, rs, theta)
    for bonds, Us in ((b0, U0), (b1, U1)):
        psi = sv.hf_state(n, ne)
        for b, U in zip(bonds, Us):
            psi = circuit.apply_two_site_sv(psi, int(b), U, n)
        assert np.abs(psi - ref).max() <= 1e-12


@pytest.mark.parametrize("n,ne", [(8, 4), (10, 4)])
def test_ladder_cancellation_is_the_same_circuit(n, ne):
    """circ_cancel_ladders (a circuit-level variant): the commuting rotations of each
    excitation reordered so the CNOT ladders of consecutive ones cancel; far fewer gates
    than the canonical list and than plain fusion, the same unitary. Checked by applying
    the gate list exactly to a statevector against the oracle's product of Pauli
    exponentials in the canonical order (no GPU), and the parameter-carrying gate of
    every rotation still exists (gradients shift those)."""
    C = G.circ_uccsd(n, ne)
    theta = syn.random_amplitudes(C.n_params, 4) * 5
    n_plain = G.circ_num_gates(C)
    C2 = G.circ_uccsd(n, ne)
    n_fused = G.circ_fuse_gates(C2)
    ng = G.circ_cancel_ladders(C)
    b1, U1 = G.circ_export_gates(C, theta)
    assert ng == len(b1) < 0.7 * n_plain and ng < 0.8 * n_fused
    rc, rp, rs, _ = ucc.uccsd_rotations(n, ne)
    ref = sv.run_ansatz(n, ne, rc, rp, rs, theta)
    psi = sv.hf_state(n, ne)
    for b, U in zip(b1, U1):
        psi = circuit.apply_two_site_sv(psi, int(b), U, n)
    assert np.abs(psi - ref).max() <= 1e-12
    # the rotation list is a permutation of the canonical one, inside each excitation
    P, pidx, scale = G.circ_get_rotations(C)
    assert np.array_equal(pidx, np.asarray(rp, dtype=np.int32))
    canon = sorted(zip(rp, map(tuple, np.asarray(rc)), rs))
    assert sorted(zip(pidx.tolist(), map(tuple, P), scale.tolist())) == canon


def _injected_create(monkeypatch, after):
    G.load_library()
    monkeypatch.setenv("MPS_FAULT_ALLOC_AFTER", str(after))
    with pytest.raises(G.MpsError) as e:
        G.mps_create(8, 16, G.MPS_MIXED, n_slots=2)
    assert e.value.code == G.MPS_ENOMEM
    assert "injected" in str(e.value)


def test_injected_allocation_failure_is_a_status_code(monkeypatch):
    """Host-side fault injection (MPS_FAULT_ALLOC_AFTER=0): the first device allocation
    of mps_create fails before any device call; the call returns MPS_ENOMEM."""
    _injected_create(monkeypatch, 0)


@pytest.mark.gpu
@pytest.mark.parametrize("after", [3, 7])
def test_injected_allocation_failure_midway(monkeypatch, after):
    """The same with real allocations before the injected failure: mps_create releases
    what it took and reports MPS_ENOMEM; the next create without injection works."""
    _injected_create(monkeypatch, after)
    monkeypatch.delenv("MPS_FAULT_ALLOC_AFTER")
    M = G.mps_create(8, 16, G.MPS_MIXED, n_slots=2)
    M.close()


def test_ladder_cancellation_reorders_only_commuting_runs():
    """circ_cancel_ladders reorders a run of rotations that share a parameter only if all
    of its strings commute pairwise, never across parameters and never fixed-angle
    rotations (parameter < 0); a run is sorted by its letters from the lowest
    non-identity site up."""
    n = 4
    X, Y, Z = 1, 2, 3
    rots = [
        ([Y, X, 0, 0], 0, 1.0), ([X, Y, 0, 0], 0, -1.0),     # commuting run: reordered (X < Y)
        ([X, 0, 0, 0], 1, 1.0), ([Z, 0, 0, 0], 1, 1.0),      # anticommuting run: kept
        ([0, Y, Z, 0], -1, 0.3), ([0, X, Z, 0], -1, 0.2),    # fixed angles: kept
        ([0, 0, Y, X], 2, 1.0),                              # run of one
    ]
    P = np.array([r[0] for r in rots], dtype=np.uint8)
    pidx = np.array([r[1] for r in rots], dtype=np.int32)
    scale = np.array([r[2] for r in rots])
    C = G.circ_create(P, pidx, scale)
    theta = np.array([0.3, -0.7, 0.5])
    b0, U0 = G.circ_export_gates(C, theta)
    G.circ_cancel_ladders(C)
    P2, pidx2, scale2 = G.circ_get_rotations(C)
    assert P2[0].tolist() == [X, Y, 0, 0] and scale2[0] == -1.0
    assert P2[1].tolist() == [Y, X, 0, 0] and scale2[1] == 1.0
    assert np.array_equal(P2[2:], P[2:]) and np.array_equal(pidx2, pidx) and np.array_equal(scale2[2:], scale[2:])
    # the same unitary: both gate lists applied to a random state agree
    rng = np.random.default_rng(0)
    psi0 = rng.normal(size=2 ** n) + 1j * rng.normal(size=2 ** n)
    b1, U1 = G.circ_export_gates(C, theta)
    outs = []
    for bonds, Us in ((b0, U0), (b1, U1)):
        psi = psi0.copy()
        for b, U in zip(bonds, Us):
            psi = circuit.apply_two_site_sv(psi, int(b), U, n)
        outs.append(psi)
    assert np.abs(outs[0] - outs[1]).max() <= 1e-12
