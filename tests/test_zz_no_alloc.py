"""trg_gemm_noalloc: the tensor-core GEMM for callers that cannot allocate device memory
where they need a product (host frameworks that own all device memory through their own
pool, real-time loops that must not risk an allocation stall or failure after start-up,
code that must not let cudaMalloc synchronise the device).  It takes the caller's device
buffers and uses only a fixed scratch array inside the library.

The test calls it through the C ABI on device buffers made by PyTorch, on two calls in a
row with different shapes and data (so that anything the first call leaves in the shared
scratch would show in the second), and checks each result against a plain NumPy FP64
product and against the allocating entry point trg_gemm.  Tolerance: the GEMM tests'
bound for the 6-product split, 2e-6 of max(|alpha| |A| |B| + |beta| |C|) per element.
It also checks that oversized problems and leading dimensions shorter than a row are
rejected before any work is queued.  This file is collected last on purpose: if it
fails, a run that stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BOUND = 2e-6   # 3 BF16 slices (6 products), FP32 accumulation


def _call(lib, prec, ta, tb, M, N, K, alpha, dA, lda, dB, ldb, beta, dC, ldc, stream):
    return lib.trg_gemm_noalloc(prec, int(ta), int(tb), M, N, K, alpha,
                                ctypes.c_void_p(dA.data_ptr()), lda,
                                ctypes.c_void_p(dB.data_ptr()), ldb, beta,
                                ctypes.c_void_p(dC.data_ptr()), ldc,
                                ctypes.c_void_p(stream))


def test_noalloc_matches_numpy_and_allocating_gemm_twice(require_gpu):
    import torch
    import paper_2507_21909_b300 as trg
    lib = trg.lib
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(11)
    shapes = [(300, 200, 1000, False, True), (257, 384, 333, True, False)]
    for call, (M, N, K, ta, tb) in enumerate(shapes):
        A = rng.standard_normal((K, M) if ta else (M, K))
        B = rng.standard_normal((N, K) if tb else (K, N))
        C0 = rng.standard_normal((M, N))
        opA, opB = (A.T if ta else A), (B.T if tb else B)
        exact = 0.5 * (opA @ opB) - 1.0 * C0
        via_alloc = trg.trg_gemm(A, B, precision=trg.TRG_PREC_BF16X6, ta=ta, tb=tb, alpha=0.5,
                                 beta=-1.0, C=C0)
        dA = torch.from_numpy(A).cuda()
        dB = torch.from_numpy(B).cuda()
        dC = torch.from_numpy(C0.copy()).cuda()
        torch.cuda.synchronize()
        rc = _call(lib, trg.TRG_PREC_BF16X6, ta, tb, M, N, K, 0.5, dA, A.shape[1], dB,
                   B.shape[1], -1.0, dC, N, stream.cuda_stream)
        assert rc == 0, lib.trg_last_error().decode()
        torch.cuda.synchronize()
        got = dC.cpu().numpy()
        scale = 0.5 * (np.abs(opA) @ np.abs(opB)).max() + np.abs(C0).max()
        assert np.abs(got - exact).max() / scale < BOUND, call
        assert np.abs(got - via_alloc).max() / scale < BOUND, call


def test_noalloc_rejects_oversized_problem_and_short_rows(require_gpu):
    import torch
    import paper_2507_21909_b300 as trg
    lib = trg.lib
    big = torch.zeros(8, device="cuda", dtype=torch.float64)
    S = 0
    # 8192 x 8192 x 8192 in 6 products needs 3 x 2 x 8192 x 8192 x 2 bytes of slices > 64 MiB
    rc = _call(lib, trg.TRG_PREC_BF16X6, 0, 0, 8192, 8192, 8192, 1.0, big, 8192, big, 8192,
               0.0, big, 8192, S)
    assert rc == -1
    assert b"scratch" in lib.trg_last_error()
    assert _call(lib, trg.TRG_PREC_FP64, 0, 0, 8, 8, 8, 1.0, big, 8, big, 8, 0.0, big, 8,
                 S) == -1
    # leading dimensions shorter than the stored rows (M = 4, N = 6, K = 5)
    for ta, tb, lda, ldb, ldc in [(0, 0, 4, 6, 6), (1, 0, 3, 6, 6), (0, 0, 5, 5, 6),
                                  (0, 1, 5, 4, 6), (0, 0, 5, 6, 5), (0, 0, 0, 6, 6)]:
        rc = _call(lib, trg.TRG_PREC_BF16X6, ta, tb, 4, 6, 5, 1.0, big, lda, big, ldb, 0.0,
                   big, ldc, S)
        assert rc == -1, (ta, tb, lda, ldb, ldc)
        assert b"leading dimension" in lib.trg_last_error()
