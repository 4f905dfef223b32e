// Learned sketch of the triad-isometry range finders: a 3-layer MLP that proposes
// per-leg row weights of the Gaussian sketch (see sketch_mlp.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace trg {

constexpr int kMlpIn = 5, kMlpHid = 256;
// flat parameter vector: W1 (hid x in), b1 (hid), W2 (hid x hid), b2 (hid), W3 (hid), b3
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + kMlpHid * kMlpIn, kOffW2 = kOffB1 + kMlpHid,
                  kOffB2 = kOffW2 + kMlpHid * kMlpHid, kOffW3 = kOffB2 + kMlpHid,
                  kOffB3 = kOffW3 + kMlpHid, kMlpParams = kOffB3 + 1;
constexpr float kQuantStep = 16.f, kQuantMax = 8.f;   // log2 weight code: round(16 u) / 16

struct SketchNet {
  float *w = nullptr;             // FP32 parameters (device)
  __nv_bfloat16 *wb = nullptr;    // BF16 copy used by inference
  float *m = nullptr, *v = nullptr;  // Adam moments
  long long adam_t = 0;
  bool loaded = false;
};

// parameters from the host (FP32, kMlpParams values); refreshes the BF16 copy
void mlp_set(SketchNet &net, const float *host, cudaStream_t s);
void mlp_get(const SketchNet &net, float *host, cudaStream_t s);
// u[r] for rows x kMlpIn inputs (device pointers); bf16 = BF16 inference, else FP32
void mlp_forward(const SketchNet &net, const float *X, int64_t rows, float *u, bool bf16,
                 cudaStream_t s);
// L = mean (u - t)^2 over the rows and its gradient (device, kMlpParams floats)
double mlp_grad(const SketchNet &net, const float *X, const float *t, int64_t rows, float *grad,
                cudaStream_t s);
// Adam over shuffled minibatches of a device-resident set; returns the last epoch's loss
double mlp_train(SketchNet &net, const float *X, const float *t, int64_t rows, int epochs,
                 int batch, float lr, uint64_t seed, cudaStream_t s);

// inputs of every index of the two legs of rho (n x n, n = da db): F rows da + db
void sketch_features(const double *rho, int da, int db, int chi, float *F, cudaStream_t s);
// the same from a factor Fm (n x m, rho = Fm Fm^T): diag(rho) = row norms^2 of Fm
// (diag_scratch: n doubles)
void sketch_features_factor(const double *Fm, int64_t m, int da, int db, int chi,
                            double *diag_scratch, float *F, cudaStream_t s);
// row weights of the sketch, w[(a b)] = 2^(code(u[a]) / 16) 2^(code(u[da + b]) / 16)
void sketch_row_weights(const float *u, int da, int db, double *w, cudaStream_t s);
// training targets t[i] = 0.5 log2(lev_i d) of both legs from an orthonormal Q (n x c)
void leverage_targets(const double *Q, int da, int db, int c, float *t, cudaStream_t s);
// x[r, :] *= w[r] for a rows x cols row-major matrix
void scale_rows(double *x, int64_t rows, int64_t cols, const double *w, cudaStream_t s);
// out = (r_l <= ratio r_p) ? A : B (n doubles); counters[0] += used A, counters[1] += used B
void select_range(const double *A, const double *B, int64_t n, const double *r_l,
                  const double *r_p, double ratio, double *out, unsigned long long *counters,
                  cudaStream_t s);
// FP32 row-major GEMM C = alpha op(A) op(B) + beta C (training path)
void sgemm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, float alpha, const float *A,
           int64_t lda, const float *B, int64_t ldb, float beta, float *C, int64_t ldc,
           cudaStream_t s);

}  // namespace trg
