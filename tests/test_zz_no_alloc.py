"""The allocation-free gate entry point gives the same MPS as the allocating one.

mps_apply_gates_noalloc serves callers that cannot have device memory allocated for
them (runtimes that own all device memory through their own pools, processes held to
a fixed budget, code that may not call cudaMalloc or cudaFree where it runs): the
caller keeps the whole MPS in its own device buffers and the library works inside a
fixed device array. This test applies the same gates through both entry points,
twice in a row, compares the results within the mixed-precision tolerances used by
the other truncated-step tests, checks the result against the oracle, checks that the
second call changes no device memory use, and that a bond outside the chain comes
back as an argument error from the device-side check.
"""
import numpy as np
import pytest

import paper_2207_03711_gb300 as G
from oracle import mps
from paper_2207_03711_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

LAM_TOL, INFIDELITY_TOL = 2e-5, 1e-6
# against the FP64 oracle after 80 truncated steps: complex64 storage and the FP32 SVD
ORACLE_LAM_TOL, ORACLE_INFIDELITY_TOL, ORACLE_P_TOL = 1e-4, 1e-5, 1e-4


def overlap(xs, ys):
    """<x|y> of two MPS given as site tensors (r_{k-1}, 2, r_k), left to right."""
    e = np.ones((1, 1), dtype=np.complex128)
    for x, y in zip(xs, ys):
        x = x.astype(np.complex128)
        y = y.astype(np.complex128)
        e = np.einsum("ab,asc,bsd->cd", e, x.conj(), y)
    return e[0, 0]


def caps(n, chi):
    c = [1] + [min(chi, 2 ** min(b + 1, n - 1 - b)) for b in range(n - 1)] + [1]
    off, o = [], 0
    for k in range(n):
        off.append(o)
        o += c[k] * 2 * c[k + 1]
    return c, off, o


def test_noalloc_matches_allocating_path():
    torch = pytest.importorskip("torch")
    G.build()
    G.load_library()
    n, chi = 24, 64
    r = syn.full_ranks(n, chi)
    st = mps.random_canonical(n, r, syn.random_mps_gaussians(n, r, 11))
    C = G.circ_uccsd(n, n // 2)
    bond, U = G.circ_export_gates(C, syn.random_amplitudes(C.n_params, 3))
    sel = slice(30000, 30080)
    bond, U = bond[sel].copy(), U[sel].copy()

    # allocating path
    M = G.mps_create(n, chi, G.MPS_MIXED)
    G.mps_set_state(M, st.B, st.lam)

    # caller-owned device buffers for the allocation-free path
    cap, off, total = caps(n, chi)
    flat = np.zeros(total, dtype=np.complex64)
    for k in range(n):
        flat[off[k]:off[k] + st.B[k].size] = st.B[k].astype(np.complex64).ravel()
    lam = np.zeros((n - 1, chi))
    for b in range(n - 1):
        lam[b, :len(st.lam[b])] = st.lam[b]
    ranks = np.array([1] + [len(l) for l in st.lam] + [1], dtype=np.int32)
    dev = torch.device("cuda")
    d_B = torch.from_numpy(flat).to(dev)
    d_off = torch.tensor(off, dtype=torch.int64, device=dev)
    d_lam = torch.from_numpy(lam).to(dev)
    d_rank = torch.from_numpy(ranks).to(dev)
    d_bond = torch.from_numpy(bond.astype(np.int32)).to(dev)
    d_U = torch.from_numpy(U.astype(np.complex128)).to(dev)
    torch.cuda.synchronize()

    half = len(bond) // 2
    for call in range(2):                       # two calls in a row on the shared workspace
        a, b = call * half, (call + 1) * half
        dw_ref = G.mps_apply_gates(M, bond[a:b], U[a:b])
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        dw = G.mps_apply_gates_noalloc(n, chi, d_B.data_ptr(), d_off.data_ptr(), d_lam.data_ptr(),
                                       d_rank.data_ptr(), b - a, d_bond.data_ptr() + 4 * a,
                                       d_U.data_ptr() + 256 * a, 0)
        torch.cuda.synchronize()
        if call == 1:       # the first call may load the kernel module; the second allocates nothing
            assert torch.cuda.mem_get_info()[0] == free0
        r_ref, sites_ref, lams_ref = G.mps_get_state(M)
        rk = d_rank.cpu().numpy()[1:-1]
        assert list(rk) == list(r_ref)
        assert abs(dw - dw_ref) <= 1e-6
        fl = d_B.cpu().numpy()
        lm = d_lam.cpu().numpy()
        full = [1] + list(rk) + [1]
        for q in range(n - 1):
            assert np.abs(lm[q, :full[q + 1]] - lams_ref[q]).max() <= LAM_TOL
        # site tensors carry the gauge of every bond (singular-vector phases are not
        # unique), so the states are compared through their overlap
        sites = [fl[off[q]:off[q] + full[q] * 2 * full[q + 1]].reshape(full[q], 2, full[q + 1])
                 for q in range(n)]
        ab, aa, bb = overlap(sites, sites_ref), overlap(sites, sites), overlap(sites_ref, sites_ref)
        assert 1.0 - abs(ab) / np.sqrt(abs(aa) * abs(bb)) <= INFIDELITY_TOL

    # against the oracle: the same 80 truncated steps in FP64 from the same state. Over a
    # short run from an exact canonical state the truncation choices coincide, so the
    # Schmidt numbers, the state and Pauli expectations agree to mixed precision.
    ref = st.copy()
    mps.apply_gates(ref, list(zip(bond, U)), chi)
    for q in range(n - 1):
        assert len(ref.lam[q]) == full[q + 1]
        assert np.abs(lm[q, :full[q + 1]] - ref.lam[q]).max() <= ORACLE_LAM_TOL
    ab, aa, bb = overlap(sites, ref.B), overlap(sites, sites), overlap(ref.B, ref.B)
    assert 1.0 - abs(ab) / np.sqrt(abs(aa) * abs(bb)) <= ORACLE_INFIDELITY_TOL
    from oracle.mps import MPS
    got = MPS([x.astype(np.complex128) for x in sites], [lm[q, :full[q + 1]].copy() for q in range(n - 1)])
    rng = np.random.default_rng(5)
    nrm_g, nrm_r = mps.norm2(got), mps.norm2(ref)
    for _ in range(20):
        code = rng.integers(0, 4, size=n).astype(np.uint8)
        pg = mps.expect_string(got, code) / nrm_g
        pr = mps.expect_string(ref, code) / nrm_r
        assert abs(pg - pr) <= ORACLE_P_TOL


def test_noalloc_reports_a_bond_outside_the_chain():
    """The bonds live in device memory, so only the kernel can check them: a bond past
    the last one stops the call before anything is indexed with it, the state stays as
    it was, and the call returns MPS_EINVAL (the discarded-weight pointer makes it wait
    and read the device status)."""
    torch = pytest.importorskip("torch")
    G.build()
    G.load_library()
    n, chi = 10, 8
    r = syn.full_ranks(n, chi)
    st = mps.random_canonical(n, r, syn.random_mps_gaussians(n, r, 4))
    cap, off, total = caps(n, chi)
    flat = np.zeros(total, dtype=np.complex64)
    for k in range(n):
        flat[off[k]:off[k] + st.B[k].size] = st.B[k].astype(np.complex64).ravel()
    lam = np.zeros((n - 1, chi))
    for b in range(n - 1):
        lam[b, :len(st.lam[b])] = st.lam[b]
    ranks = np.array([1] + [len(l) for l in st.lam] + [1], dtype=np.int32)
    dev = torch.device("cuda")
    d_B = torch.from_numpy(flat).to(dev)
    d_off = torch.tensor(off, dtype=torch.int64, device=dev)
    d_lam = torch.from_numpy(lam).to(dev)
    d_rank = torch.from_numpy(ranks).to(dev)
    d_bond = torch.tensor([n - 1, 0], dtype=torch.int32, device=dev)      # n-1 is not a bond
    d_U = torch.from_numpy(np.stack([np.eye(4, dtype=np.complex128)] * 2)).to(dev)
    torch.cuda.synchronize()
    with pytest.raises(G.MpsError) as e:
        G.mps_apply_gates_noalloc(n, chi, d_B.data_ptr(), d_off.data_ptr(), d_lam.data_ptr(), d_rank.data_ptr(),
                                  2, d_bond.data_ptr(), d_U.data_ptr(), 0)
    assert e.value.code == G.MPS_EINVAL and "bond" in str(e.value)
    assert np.array_equal(d_rank.cpu().numpy(), ranks)
    assert np.array_equal(d_B.cpu().numpy(), flat)


def test_noalloc_rejects_sizes_beyond_the_workspace():
    G.build()
    G.load_library()
    with pytest.raises(G.MpsError) as e:
        G.mps_apply_gates_noalloc(24, 128, 1, 1, 1, 1, 0, 1, 1, 0)
    assert e.value.code == G.MPS_EINVAL and "chi" in str(e.value)
