// Exact-accumulation (Ozaki-style digit) tensor-core GEMM, see gemm_oz.cu.
#pragma once
#include "gemm_tc.h"

namespace trg {

// C (FP64) = alpha op(A) op(B) + beta C with `ns` 7-bit digits per row/column (3..6)
void gemm_oz(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
             int64_t lda, int64_t sA, const double *B, int64_t ldb, int64_t sB, double beta,
             double *C, int64_t ldc, int64_t sC, int64_t batch, int ns, TcScratch &scr,
             cudaStream_t s, TcTiming *timing = nullptr);
int oz_error_flag(bool reset);

}  // namespace trg
