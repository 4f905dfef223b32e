// Exact-accumulation (Ozaki-style digit) tensor-core GEMM, see gemm_oz.cu.
#pragma once
#include "gemm_tc.h"

namespace trg {

// Digit planes of one operand op(X) (rows x K; trans: X stored K x rows) as the kernel
// reads them: exponent codes [batch][rows] and planes pre-tiled per (batch, 8-row group,
// 16-wide K block, slice) in 256-byte runs (the MMA's core-matrix layout; gemm_oz.cu).
// An operand that several products share can be split once (oz_prepare) and passed to
// each.
// fl: BF16 pieces of every value (a = a_0 + a_1 + ..., no exponent codes) for the
// split-BF16 products instead of digits under a common exponent.
struct OzOperand {
  const unsigned *e = nullptr;
  const void *planes = nullptr;
  int64_t rows = 0, K = 0, Kp = 0, batch = 0;
  int ns = 0;
  bool fl = false;
};
OzOperand oz_prepare(const double *X, int64_t rows, int64_t K, int64_t ld, int64_t sX,
                     bool trans, int64_t batch, int ns, TcScratch &scr, cudaStream_t s,
                     bool fl = false);

// C (FP64) = alpha op(A) op(B) + beta C with `ns` 7-bit digits per row/column (3..7), or
// with fl, `ns` BF16 pieces per value (2..4: the BF16x3 / x6 / x10 products, FP32
// accumulation, 128 x 256 tiles); pa / pb: planes of op(A) / op(B) prepared by oz_prepare
// (else split here)
void gemm_oz(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
             int64_t lda, int64_t sA, const double *B, int64_t ldb, int64_t sB, double beta,
             double *C, int64_t ldc, int64_t sC, int64_t batch, int ns, TcScratch &scr,
             cudaStream_t s, TcTiming *timing = nullptr, const OzOperand *pa = nullptr,
             const OzOperand *pb = nullptr, bool fl = false);
int oz_error_flag(bool reset);

}  // namespace trg
