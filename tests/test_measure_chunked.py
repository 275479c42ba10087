"""The chunked depth-first trie measurement (Eq. 11 generalised to Pauli strings,
Sec. III-C) against the oracle's plain left-to-right contraction of each string.

* The result does not depend on the chunking: a budget that forces chunks of 16 nodes
  per level gives the same expectations as whole levels (bit for bit in FP64, within
  rounding of the tensor-core tiles in mixed precision).
* Mixed precision at the 24-qubit, chi = 64 shape (CUDA-core environments): sampled
  strings and the energy of the loaded state against the FP64 oracle.
* Mixed precision at 20 qubits, chi = 128, where the levels whose bonds are both >= 128
  run on the tensor cores: chunked against whole levels, and against the oracle.
* Bond dimension 256 at 64 qubits (the measurement-bound configuration: a seeded random
  right-canonical MPS with every interior rank at min(256, 2^min(k+1, n-1-k))): seeded
  Jordan-Wigner-shaped strings sharing prefixes, FP64 and mixed, against the oracle.
"""
import numpy as np
import pytest

import paper_2207_03711_gb300 as G
from oracle import mps, pauli
from paper_2207_03711_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    G.build()
    return G.load_library()


def _canon(n, chi, seed, bias=1.0):
    """Random canonical MPS at full ranks; bias > 1 scales the Gaussian rows of physical
    index 0 so that local expectations are O(1) rather than ~2^(-n/2)."""
    r = syn.full_ranks(n, chi)
    g = syn.random_mps_gaussians(n, r, seed)
    rr = [1] + list(r) + [1]
    for k in range(n):
        g[k][:rr[k + 1]] *= bias
    return mps.random_canonical(n, r, g)


def jw_shaped_strings(n, count, seed):
    """Strings shaped like Jordan-Wigner terms: I..I P_p Z..Z P_q I..I and products of two
    such pairs (P in {X, Y}), plus Z_p and Z_p Z_q; many share their leading identities."""
    rng = np.random.default_rng(seed)
    out = set()
    while len(out) < count:
        s = np.zeros(n, dtype=np.uint8)
        kind = rng.integers(0, 4)
        p, q = sorted(rng.choice(n, 2, replace=False))
        if kind == 0:
            s[p] = 3
        elif kind == 1:
            s[p] = s[q] = 3
        else:
            s[p] = rng.integers(1, 3)
            s[p + 1:q] = 3
            s[q] = rng.integers(1, 3)
            if kind == 3 and q + 2 < n:
                r, t = sorted(rng.choice(np.arange(q + 1, n), 2, replace=False))
                s[r] = rng.integers(1, 3)
                s[r + 1:t] = 3
                s[t] = rng.integers(1, 3)
        out.add(s.tobytes())
    return np.array([np.frombuffer(b, dtype=np.uint8) for b in sorted(out)])


@pytest.mark.parametrize("prec", [G.MPS_FP64, G.MPS_MIXED])
def test_chunking_does_not_change_results(prec):
    n, chi = 16, 32
    st = _canon(n, chi, 5, bias=2.0)
    h, g = syn.random_integrals(n // 2, 4)
    codes, _ = pauli.jordan_wigner_hamiltonian(h, g)
    M = G.mps_create(n, chi, prec)
    G.mps_set_state(M, st.B, st.lam)
    whole = G.mps_expect_paulis(M, codes)
    G.mps_set_meas_budget(M, 1)           # 16-node chunks on every level
    chunked = G.mps_expect_paulis(M, codes)
    G.mps_set_meas_budget(M, 0)
    again = G.mps_expect_paulis(M, codes)
    assert np.array_equal(whole, again)
    if prec == G.MPS_FP64:
        assert np.array_equal(whole, chunked)
    else:
        assert np.abs(whole - chunked).max() <= 1e-7
    idx = np.random.default_rng(0).choice(len(codes), 100, replace=False)
    ref = np.array([mps.expect_string(st, codes[i]) for i in idx]) / mps.norm2(st)
    tol = 1e-11 if prec == G.MPS_FP64 else 2e-5
    print(f"16q chi32 prec={prec} max|d<P>| = {np.abs(chunked[idx] - ref).max():.3e}")
    assert np.abs(chunked[idx] - ref).max() <= tol


def test_mixed_measurement_24q():
    n, chi = 24, 64
    st = _canon(n, chi, 3, bias=2.0)
    h, g = syn.random_integrals(12, 0)
    codes, coeffs = pauli.jordan_wigner_hamiltonian(h, g)
    M = G.mps_create(n, chi, G.MPS_MIXED)
    G.mps_set_state(M, st.B, st.lam)
    vals = G.mps_expect_paulis(M, codes)
    idx = np.random.default_rng(1).choice(len(codes), 300, replace=False)
    nrm = mps.norm2(st)
    ref = np.array([mps.expect_string(st, codes[i]) for i in idx]) / nrm
    err = np.abs(vals[idx] - ref).max()
    H = G.ham_jw_from_integrals(h, g)
    e_gpu = G.mps_energy(M, H)
    e_ref = sum(c * mps.expect_string(st, codes[i]).real for i, c in zip(idx, coeffs[idx])) / nrm
    e_sub = float(np.sum(coeffs[idx] * vals[idx].real))
    print(f"24q chi64 mixed: max|d<P>| = {err:.3e}; sampled-energy |dE| = {abs(e_sub - e_ref):.3e} Ha; "
          f"E = {e_gpu:.9f}")
    assert err <= 2e-5
    assert abs(e_sub - e_ref) <= 1e-4
    assert np.isfinite(e_gpu)


def test_tensor_core_levels_20q_chi128():
    n, chi = 20, 128
    st = _canon(n, chi, 11, bias=2.0)
    codes = jw_shaped_strings(n, 400, 12)
    M = G.mps_create(n, chi, G.MPS_MIXED)
    G.mps_set_state(M, st.B, st.lam)
    G.mps_set_kernel_timing(M, True)
    whole = G.mps_expect_paulis(M, codes)
    s = G.mps_get_stats(M)
    assert s["tc_gemm_launches"] > 0 and s["ms_tc_gemm"] > 0      # the tensor-core levels ran
    G.mps_set_meas_budget(M, 1)
    chunked = G.mps_expect_paulis(M, codes)
    ref = np.array([mps.expect_string(st, c) for c in codes]) / mps.norm2(st)
    print(f"20q chi128 mixed: whole vs chunked {np.abs(whole - chunked).max():.3e}, vs oracle "
          f"{np.abs(whole - ref).max():.3e} (max|<P>| {np.abs(ref).max():.3e}), tc launches {s['tc_gemm_launches']}")
    assert np.abs(whole - chunked).max() <= 1e-6
    assert np.abs(whole - ref).max() <= 2e-5


@pytest.mark.parametrize("prec", [G.MPS_FP64, G.MPS_MIXED])
def test_chi256_measurement_64q(prec):
    n, chi = 64, 256
    st = _canon(n, chi, 7, bias=3.0)
    codes = jw_shaped_strings(n, 40, 9)
    M = G.mps_create(n, chi, prec)
    G.mps_set_state(M, st.B, st.lam)
    assert list(G.mps_get_ranks(M)) == syn.full_ranks(n, chi)
    vals = G.mps_expect_paulis(M, codes)
    nrm = mps.norm2(st)
    ref = np.array([mps.expect_string(st, c) for c in codes]) / nrm
    err = np.abs(vals - ref).max()
    print(f"64q chi256 prec={prec}: max|d<P>| = {err:.3e} over {len(codes)} strings, "
          f"max|<P>| = {np.abs(ref).max():.3e}")
    # mixed: complex64 environments through 64 levels of tensor-core contractions
    assert err <= (1e-10 if prec == G.MPS_FP64 else 1e-4)
    with pytest.raises(G.MpsError) as e:       # gates are applied at chi <= 128 only
        G.mps_apply_gates(M, np.array([0], dtype=np.int32), np.eye(4)[None].astype(complex))
    assert e.value.code == G.MPS_EINVAL


def test_ragged_odd_bonds_chi256():
    """A loaded chi = 256 state whose bond ranks are odd where both bonds of a level reach
    128: an odd right bond runs on the tensor cores (GEMM widths, leading dimensions and T
    rows of odd width), an odd left bond goes to the CUDA-core kernels (the tensor-core
    route reads L in place as 16-byte-aligned rows of 2D floats); both precisions agree
    with the oracle."""
    n, chi = 18, 256
    r = [2, 4, 8, 16, 32, 64, 128, 255, 131, 201, 128, 64, 32, 16, 8, 4, 2]
    g = syn.random_mps_gaussians(n, r, 21)
    rr = [1] + r + [1]
    for k in range(n):
        g[k][:rr[k + 1]] *= 2.0
    st = mps.random_canonical(n, r, g)
    codes = jw_shaped_strings(n, 60, 22)
    ref = np.array([mps.expect_string(st, c) for c in codes]) / mps.norm2(st)
    for prec, tol in ((G.MPS_FP64, 1e-10), (G.MPS_MIXED, 2e-5)):
        M = G.mps_create(n, chi, prec)
        G.mps_set_state(M, st.B, st.lam)
        assert list(G.mps_get_ranks(M)) == r
        G.mps_set_kernel_timing(M, True)
        vals = G.mps_expect_paulis(M, codes)
        s = G.mps_get_stats(M)
        err = np.abs(vals - ref).max()
        print(f"18q chi256 odd bonds prec={prec}: max|d<P>| = {err:.3e}, tc launches {s['tc_gemm_launches']}")
        if prec == G.MPS_MIXED:
            assert s["tc_gemm_launches"] > 0
        assert err <= tol
