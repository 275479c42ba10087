"""The tensor-core GEMM (tcgen05 + TMEM + TMA, compensated TF32 splits) against an FP64
product computed on the host.

The environment sweeps of the measurement (Eq. 11 generalised to Pauli strings,
Sec. III-C) are dense complex contractions; in mixed precision they run on this
primitive as real GEMMs. Shapes cover one and several 128 x 256 tiles, ragged edges in
every dimension, K that is not a multiple of the 32-wide K tile, and leading
dimensions larger than the logical width. The bound is elementwise,
|C - AB^T| <= 1e-5 (|A||B|^T): a single TF32 product (10-bit mantissa) misses it by
about 50x, so the low-order split products are really applied.
"""
import numpy as np
import pytest

import paper_2207_03711_gb300 as G

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (128, 256, 32), (127, 255, 37), (300, 600, 64), (256, 512, 512),
          (1000, 130, 96), (64, 1024, 128), (513, 257, 4)]


@pytest.fixture(scope="module", autouse=True)
def lib():
    G.build()
    return G.load_library()


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tc_gemm_matches_fp64(M, N, K):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    lda, ldb, ldc = K + 3, K + 5, N + 2
    A = rng.normal(size=(M, lda)).astype(np.float32)
    B = rng.normal(size=(N, ldb)).astype(np.float32) * 1e-3
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.full((M, ldc), -7.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    G.mps_tc_gemm_tf32x3(M, N, K, dA.data_ptr(), lda, dB.data_ptr(), ldb, dC.data_ptr(), ldc)
    C = dC.cpu().numpy()
    a, b = A[:, :K].astype(np.float64), B[:, :K].astype(np.float64)
    ref = a @ b.T
    scale = np.abs(a) @ np.abs(b).T
    err = np.abs(C[:, :N] - ref)
    print(f"M={M} N={N} K={K}: max err / scale = {(err / (scale + 1e-30)).max():.3e}")
    assert np.all(err <= 1e-5 * scale + 1e-30)
    # columns beyond N untouched
    assert np.all(C[:, N:] == -7.0)
    if K >= 32:
        # a single TF32 product would not meet the bound
        t32 = lambda x: (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)
        one = t32(A[:, :K].copy()) @ t32(B[:, :K].copy()).T
        assert (np.abs(one - ref) / (scale + 1e-30)).max() > 1e-5


def test_tc_gemm_rejects_bad_sizes():
    with pytest.raises(G.MpsError) as e:
        G.mps_tc_gemm_tf32x3(4, 4, 8, 1, 4, 1, 8, 1, 4)   # lda < K
    assert e.value.code == G.MPS_EINVAL
