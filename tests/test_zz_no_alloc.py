"""trg_gemm_noalloc: the tensor-core GEMM for callers that must not allocate device
memory (for example code running during CUDA graph capture, or inside a host framework
that owns all device memory).  It takes the caller's device buffers and uses only a
fixed scratch array inside the library.

The test calls it through the C ABI on device buffers made by PyTorch and checks the
result against the allocating entry point trg_gemm (host buffers) on two calls in a row
with different data, so that nothing left in the shared scratch by the first call can
leak into the second.  Tolerance: the GEMM tests' bound, 2e-6 of max(|A||B|) for the
6-product split (both entry points run the same kernels, so they agree far closer).
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_gemm_twice(require_gpu):
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
        ref = trg.trg_gemm(A, B, precision=trg.TRG_PREC_BF16X6, ta=ta, tb=tb, alpha=0.5,
                           beta=-1.0, C=C0)
        dA = torch.from_numpy(A).cuda()
        dB = torch.from_numpy(B).cuda()
        dC = torch.from_numpy(C0.copy()).cuda()
        torch.cuda.synchronize()
        rc = lib.trg_gemm_noalloc(trg.TRG_PREC_BF16X6, int(ta), int(tb), M, N, K, 0.5,
                                  ctypes.c_void_p(dA.data_ptr()), A.shape[1],
                                  ctypes.c_void_p(dB.data_ptr()), B.shape[1], -1.0,
                                  ctypes.c_void_p(dC.data_ptr()), N,
                                  ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.trg_last_error().decode()
        torch.cuda.synchronize()
        got = dC.cpu().numpy()
        scale = 0.5 * (np.abs(A.T if ta else A) @ np.abs(B.T if tb else B)).max() + np.abs(C0).max()
        assert np.abs(got - ref).max() / scale < 2e-6, call


def test_noalloc_rejects_oversized_problem(require_gpu):
    import torch
    import paper_2507_21909_b300 as trg
    lib = trg.lib
    big = torch.zeros(8, device="cuda", dtype=torch.float64)
    p = ctypes.c_void_p(big.data_ptr())
    # 8192 x 8192 x 8192 in 6 products needs 3 x 2 x 8192 x 8192 x 2 bytes of slices > 64 MiB
    rc = lib.trg_gemm_noalloc(trg.TRG_PREC_BF16X6, 0, 0, 8192, 8192, 8192, 1.0, p, 8192, p,
                              8192, 0.0, p, 8192, None)
    assert rc == -1
    assert b"scratch" in lib.trg_last_error()
    assert lib.trg_gemm_noalloc(trg.TRG_PREC_FP64, 0, 0, 8, 8, 8, 1.0, p, 8, p, 8, 0.0, p, 8,
                                None) == -1
