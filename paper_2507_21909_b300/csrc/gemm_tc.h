// Split-precision tcgen05 GEMM (see gemm_tc.cu).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace trg {

// device scratch provider (slice buffers, split-K partial tiles)
struct TcScratch {
  virtual void *alloc(size_t bytes) = 0;
  virtual ~TcScratch() = default;
};

// optional CUDA-event timing of the tensor-core kernel launches (launching stream).
// after(): kind 0 = exact-digit GEMM (gemm_oz, 3..6 digits), 1 = split-BF16 / 3xTF32 GEMM
// (gemm_tc), 2 = the seven-digit FP64-equivalent digit GEMM;
// alg_flop = 2 M N K batch (the product the caller asked for, counted once);
// pipe_flop = the BF16 tensor-pipe work of every digit / slice product issued.
struct TcTiming {
  virtual void before(cudaStream_t s) = 0;
  virtual void after(cudaStream_t s, int kind, double alg_flop, double pipe_flop) = 0;
  virtual ~TcTiming() = default;
};

// C (FP64) = alpha * op(A) op(B) + beta * C with A, B split into `ns` BF16 slices (or
// TF32 slices, tf32 = true: 3xTF32 for ns = 2) and the slice products i + j < ns
// accumulated in FP32 on the tensor cores.
void gemm_tc(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
             int64_t lda, int64_t sA, const double *B, int64_t ldb, int64_t sB, double beta,
             double *C, int64_t ldc, int64_t sC, int64_t batch, int ns, TcScratch &scr,
             cudaStream_t s, TcTiming *timing = nullptr, bool tf32 = false);

// 1 if a bounded mbarrier wait of the tensor-core kernel gave up (reset on request)
int tc_error_flag(bool reset);
int64_t tc_launch_count();

}  // namespace trg
