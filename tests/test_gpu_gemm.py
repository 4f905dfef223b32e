"""The contraction engine on the GPU against a plain NumPy FP64 product.

Error measure: max |C - A B| / max (|A| |B|) (the elementwise bound of a dot product).
FP64 CUDA-core GEMM: 1e-14.  Split-BF16 tcgen05 GEMM with FP32 accumulation:
2 slices (3 products) < 1e-4, 3 slices (6 products) < 2e-6, 4 slices (10) < 2e-6;
3xTF32 (two 11-bit TF32 slices, 3 products, FP32 accumulation) < 1e-5;
the 3/4-slice bound is the FP32 accumulation, not the operand split.  Exact-accumulation
digit GEMM (row exponents, 7-bit digits): 4 digits < 1e-7, 5 and 6 digits < 5e-9; the
seven-digit form with four exact levels (precision 8) < 5e-14 (measured 1.1-2.3e-14:
the 49-bit digits cut each operand at 2^-50 of its row or column maximum).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(128, 256, 64, False, False), (300, 200, 1000, False, False),
          (64, 48, 5000, True, False), (1000, 130, 70, False, True),
          (257, 129, 333, True, True), (2048, 512, 4096, False, False)]
BOUND = {0: 1e-14, 1: 1e-4, 2: 2e-6, 3: 2e-6, 4: 1e-7, 5: 5e-9, 6: 5e-9, 7: 1e-5, 8: 5e-14}


@pytest.fixture(scope="module")
def trg(require_gpu):
    import paper_2507_21909_b300 as pkg
    return pkg


@pytest.mark.parametrize("prec", [0, 1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("M,N,K,ta,tb", SHAPES)
def test_gemm_against_numpy(trg, prec, M, N, K, ta, tb):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((N, K) if tb else (K, N))
    opA = A.T if ta else A
    opB = B.T if tb else B
    C0 = rng.standard_normal((M, N))
    ref = 0.5 * (opA @ opB) - 2.0 * C0
    got = trg.trg_gemm(A, B, precision=prec, ta=ta, tb=tb, alpha=0.5, beta=-2.0, C=C0)
    scale = 0.5 * (np.abs(opA) @ np.abs(opB)).max() + 2.0 * np.abs(C0).max()
    err = np.abs(got - ref).max() / scale
    assert err < BOUND[prec], err


@pytest.mark.parametrize("prec,bound", [(2, 2e-6), (5, 5e-9)])
def test_gemm_scaled_rows(trg, prec, bound):
    """Rows spanning 12 orders of magnitude: per-element BF16 exponents (split modes) and
    per-row exponents (digit modes) both keep every row's relative accuracy."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((256, 512)) * np.logspace(-6, 6, 256)[:, None]
    B = rng.standard_normal((512, 384))
    got = trg.trg_gemm(A, B, precision=prec)
    ref = A @ B
    rel = np.abs(got - ref).max(axis=1) / (np.abs(A) @ np.abs(B)).max(axis=1)
    assert rel.max() < bound


THIN = [(48, 48, 100003, True, False), (64, 64, 8192, False, True), (17, 33, 5000, True, True),
        (48, 48, 4096, False, False)]


@pytest.mark.parametrize("M,N,K,ta,tb", THIN)
def test_gemm_f64_thin(trg, M, N, K, ta, tb):
    """FP64 products with an output of at most 64 x 64 over a long inner dimension (the
    split-K micro-tile kernel), including ragged K and sizes off the 16-grid."""
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((N, K) if tb else (K, N))
    opA, opB = (A.T if ta else A), (B.T if tb else B)
    C0 = rng.standard_normal((M, N))
    got = trg.trg_gemm(A, B, precision=0, ta=ta, tb=tb, alpha=0.5, beta=-2.0, C=C0)
    ref = 0.5 * (opA @ opB) - 2.0 * C0
    scale = 0.5 * (np.abs(opA) @ np.abs(opB)).max() + 2.0 * np.abs(C0).max()
    assert np.abs(got - ref).max() / scale < 1e-14


@pytest.mark.parametrize("M,K", [(100003, 48), (5000, 64), (4096, 7)])
def test_gemm_f64_gram_and_tall(trg, M, K):
    """A Gram X^T X passed as one host matrix (the symmetric upper-triangle kernel) is
    exactly symmetric and matches NumPy; a tall X R product (M x K times K x K)."""
    rng = np.random.default_rng(M + K)
    X = rng.standard_normal((M, K))
    G = trg.trg_gemm(X, X, precision=0, ta=True, tb=False)
    ref = X.T @ X
    assert np.array_equal(G, G.T)
    assert np.abs(G - ref).max() / (np.abs(X).T @ np.abs(X)).max() < 1e-14
    R = np.triu(rng.standard_normal((K, K)))
    P = trg.trg_gemm(X, R, precision=0)
    assert np.abs(P - X @ R).max() / (np.abs(X) @ np.abs(R)).max() < 1e-14
