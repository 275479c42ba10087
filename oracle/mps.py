"""c2: the paper's truncated right-canonical MPS simulator, written out plainly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper passages followed (Sec. III-A):
  * Eq. (6): c_{i_1..i_N} = sum_a B^{i_1}_{a_1} B^{i_2}_{a_1 a_2} ... B^{i_N}_{a_{N-1}};
    site tensors are kept right-canonical and the Schmidt numbers lambda of each
    bond are stored.
  * Eq. (7): M_{a_{n-1} i_n i_{n+1} a_{n+1}} = sum_{a_n} O^{i_n i_{n+1}}_{i_n' i_{n+1}'}
    B^{i_n'}_{a_{n-1} a_n} B^{i_{n+1}'}_{a_n a_{n+1}}.
  * Eq. (8): M' = lambda_{a_{n-1}} M. The printed sum over a_{n-1} is read as an
    element-wise row scaling (the index survives on the left-hand side).
  * Eq. (9): SVD(M') = U lambda' V, keeping the D largest Schmidt numbers; the
    discarded weight is reported ("this error can be monitored").
  * Eq. (10): B_{n+1} <- V and B_n <- sum M V^* (no division by lambda).
  * Eq. (11) generalised to Pauli strings: <P> by a plain left-to-right
    contraction of transfer matrices over all sites, no shortcuts.

Readings where the paper leaves a choice: keep k = min(chi, #{sigma > 1e-13 sigma_0}); the state is
never renormalised; energies are divided by <psi|psi>.

Storage: B[k] has shape (r_{k-1}, 2, r_k); lam[k] holds the Schmidt numbers of the
bond between sites k and k+1; the left edge of site 0 uses lambda = [1].
"""
import numpy as np

from .sv import neumaier_sum
from .pauli import SIGMA

CUTOFF = 1e-13


class MPS:
    def __init__(self, B, lam):
        self.B = B
        self.lam = lam

    @property
    def n(self):
        return len(self.B)

    def ranks(self):
        return [b.shape[2] for b in self.B[:-1]]

    def copy(self):
        return MPS([b.copy() for b in self.B], [l.copy() for l in self.lam])


def hf_mps(n, n_electrons):
    """Product state of the reference determinant (Sec. III-D): site q holds |1> for q < N_e."""
    B = []
    for q in range(n):
        t = np.zeros((1, 2, 1), dtype=complex)
        t[0, 1 if q < n_electrons else 0, 0] = 1.0
        B.append(t)
    return MPS(B, [np.ones(1) for _ in range(n - 1)])


def left_lambda(mps, site):
    return np.ones(1) if site == 0 else mps.lam[site - 1]


def apply_two_site(mps, bond, O, chi, cutoff=CUTOFF):
    """Eqs. (7)-(10) on bond (bond, bond+1). Returns the discarded weight fraction."""
    Bn, Bn1 = mps.B[bond], mps.B[bond + 1]
    rl, rr = Bn.shape[0], Bn1.shape[2]
    # Eq. (7): contract the shared bond, then the gate on the two physical legs
    theta = np.einsum("aib,bjc->aijc", Bn, Bn1)
    M = np.einsum("ijkl,aklc->aijc", O.reshape(2, 2, 2, 2), theta)
    # Eq. (8): scale rows by the Schmidt numbers of the bond to the left
    Mp = left_lambda(mps, bond)[:, None, None, None] * M
    # Eq. (9): SVD of M' as a (2 r_left) x (2 r_right) matrix and truncation
    _, s, Vh = np.linalg.svd(Mp.reshape(2 * rl, 2 * rr), full_matrices=False)
    k = int(min(chi, np.count_nonzero(s > cutoff * s[0])))
    total = np.sum(s ** 2)
    discarded = float(np.sum(s[k:] ** 2) / total) if total > 0 else 0.0
    V = Vh[:k]
    # Eq. (10): B_{n+1} <- V, B_n <- M V^+ (M, not M')
    mps.B[bond + 1] = V.reshape(k, 2, rr)
    mps.B[bond] = (M.reshape(2 * rl, 2 * rr) @ V.conj().T).reshape(rl, 2, k)
    mps.lam[bond] = s[:k].copy()
    return discarded


def apply_gates(mps, gates, chi, cutoff=CUTOFF):
    """Apply a list of (bond, 4x4); returns the summed discarded weight."""
    dw = 0.0
    for bond, O in gates:
        dw += apply_two_site(mps, bond, O, chi, cutoff)
    return dw


def expect_string(mps, code):
    """<psi|P|psi> by transfer matrices L_{k+1} = sum_ij sigma_ij B^{i+} L_k B^j, k = 0..n-1."""
    L = np.ones((1, 1), dtype=complex)
    for k in range(mps.n):
        s = SIGMA[int(code[k])]
        Bk = mps.B[k]
        new = np.zeros((Bk.shape[2], Bk.shape[2]), dtype=complex)
        for i in range(2):
            for j in range(2):
                if s[i, j] != 0:
                    new += s[i, j] * (Bk[:, i, :].conj().T @ L @ Bk[:, j, :])
        L = new
    return L[0, 0]


def norm2(mps):
    return expect_string(mps, np.zeros(mps.n, dtype=np.uint8)).real


def energy(mps, codes, coeffs):
    """E = sum_i a_i Re<P_i> / <psi|psi> (Eq. 2), Neumaier-summed in term order.

    Returns (E, per-term <P_i> / <psi|psi> as complex)."""
    nrm = norm2(mps)
    ev = np.array([expect_string(mps, c) for c in codes]) / nrm
    return neumaier_sum(list(coeffs * ev.real)), ev


def to_statevector(mps):
    """Dense amplitudes (qubit q = bit q of the index) for small checks."""
    t = mps.B[0][0]                                 # (2, r_0): [i_0, a]
    for k in range(1, mps.n):
        t = np.einsum("xa,aib->xib", t, mps.B[k])   # x enumerates (i_0..i_{k-1}), site 0 slowest
        t = t.reshape(-1, mps.B[k].shape[2])
    c = t[:, 0]                                     # index = sum_k i_k 2^(n-1-k)
    n = mps.n
    return c.reshape((2,) * n).transpose(tuple(range(n))[::-1]).reshape(-1)


def from_statevector(psi, n):
    """Exact right-canonical MPS of a dense state by right-to-left SVDs (no truncation
    beyond exact zeros); lam holds the exact Schmidt numbers of each bond."""
    c = psi.reshape((2,) * n).transpose(tuple(range(n))[::-1]).reshape(-1)  # site 0 slowest
    B = [None] * n
    lam = [None] * (n - 1)
    cur = c.reshape(-1, 2)          # (left configurations, i_{n-1}) with right bond 1
    r_right = 1
    for k in range(n - 1, 0, -1):
        mat = cur.reshape(-1, 2 * r_right)
        U, s, Vh = np.linalg.svd(mat, full_matrices=False)
        r = int(np.count_nonzero(s > 1e-14 * s[0]))
        B[k] = Vh[:r].reshape(r, 2, r_right)
        lam[k - 1] = s[:r] / np.linalg.norm(s[:r])
        cur = U[:, :r] * s[:r]
        r_right = r
    B[0] = cur.reshape(1, 2, r_right)
    return MPS(B, lam)


def random_canonical(n, ranks, gauss):
    """A random MPS in exact canonical form from caller-drawn Gaussian arrays.

    ranks: n-1 bond ranks; gauss[k]: complex array of shape (2 r_k, r_{k-1}) for
    site k (r_{-1} = r_{n-1} = 1). Each site is made right-canonical by a QR
    factorisation, then every bond is rotated (left to right) so that the left
    environment sum_i B^{i+} L B^i is diagonal; lam then holds the exact Schmidt
    numbers of each bond and the state has unit norm.
    """
    r = [1] + list(ranks) + [1]
    B = []
    for k in range(n):
        q, _ = np.linalg.qr(gauss[k])                # (2 r_k) x r_{k-1}, orthonormal columns
        B.append(q.conj().T.reshape(r[k], 2, r[k + 1]))
    # normalise: site 0 is a single row of unit norm already (QR of a column)
    lam = []
    L = np.ones((1, 1), dtype=complex)
    for k in range(n - 1):
        L = sum(B[k][:, i, :].conj().T @ L @ B[k][:, i, :] for i in range(2))
        w, W = np.linalg.eigh(L)
        idx = np.argsort(w)[::-1]
        w, W = w[idx], W[:, idx]
        B[k] = np.einsum("aib,bc->aic", B[k], W)
        B[k + 1] = np.einsum("cb,bjd->cjd", W.conj().T, B[k + 1])
        L = np.diag(w).astype(complex)
        lam.append(np.sqrt(np.maximum(w, 0.0)))
    return MPS(B, lam)
