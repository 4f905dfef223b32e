// Internal declarations of libtrg (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/trg.h"

namespace trg {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define TRG_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      throw ::trg::Error(TRG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
// every kernel launch of the library is followed by this check, which also counts it
// (atomic: batched instances launch from several host threads)
extern std::atomic<int64_t> g_kernel_launches;
#define TRG_LAUNCH_CHECK()        \
  do {                            \
    ++::trg::g_kernel_launches;   \
    TRG_CUDA(cudaGetLastError()); \
  } while (0)

// message returned by trg_last_error()
void set_last_error(const std::string &msg);

// Two environment variables, read once, hold every switch that is not part of the API:
//   TRG_STUDY="key=value,..."  precision and slicing studies; these change how a step is
//       computed (never set by the library's own callers):
//       slice_mb=<MiB>      budget of one coarse-contraction slice (default 1024)
//       decomp_fp64=1       every GEMM inside a decomposition in FP64
//       tc_phases=<mask>    phases whose GEMMs may use the tensor cores (default 0xFF)
//       exact_everywhere=1  impurity-only products in the exact-digit form too
//       tc_min_max=<n>      smallest max(M, N) sent to the tensor cores (default 64)
//       swap_gram_digits=<n> digits of the bond-swap compression Grams (64 = FP64)
//       decomp_cuda_fp64=1  digit forms: decomposition / thin products on the FP64 CUDA
//                           cores instead of the seven-digit FP64-equivalent GEMM
//   TRG_DEBUG="gemm,mem,svd,attr"  diagnostic prints to stderr (no effect on results).
// study_opt returns the value of `key` ("" if unset); debug_opt whether it is listed.
std::string study_opt(const char *key);
bool debug_opt(const char *key);

// ------------------------------------------------------------------ device arena
// Bump allocator over a few large cudaMalloc chunks.  Scratch of one step is released
// at once by reset(); persistent state buffers are separate cudaMalloc'd buffers.
class Arena {
 public:
  struct Mark { size_t top, used, cur; };
  void *alloc(size_t bytes);
  // stack discipline: everything allocated after mark() is released by release(mark)
  Mark mark() const { return {top_, chunks_.empty() ? 0 : chunks_[top_].used, cur_}; }
  void release(const Mark &m);
  size_t in_use() const { return cur_; }
  size_t reserved() const {
    size_t r = 0;
    for (auto &c : chunks_) r += c.cap;
    return r;
  }
  void reset();           // callers must have synchronised the stream first
  void release();         // frees all chunks
  size_t high_water() const { return high_; }
  ~Arena() { release(); }

 private:
  struct Chunk { char *p; size_t cap; size_t used; };
  std::vector<Chunk> chunks_;  // chunks after top_ are empty
  size_t top_ = 0;
  size_t high_ = 0, cur_ = 0;
};

// dense row-major FP64 tensor living in the arena (or in a persistent buffer)
struct Tensor {
  double *p = nullptr;
  std::vector<int64_t> dims;
  int64_t size() const {
    int64_t n = 1;
    for (auto d : dims) n *= d;
    return n;
  }
  int64_t dim(int i) const { return dims[i]; }
};

// --------------------------------------------------------------------- kernels
void permute(const double *in, double *out, const std::vector<int64_t> &dims_in,
             const std::vector<int> &perm, cudaStream_t s);
// C[b] = alpha * op(A[b]) op(B[b]) + beta * C[b], row-major, FP64 on CUDA cores.
// b_upper: the caller guarantees op(B) is upper triangular (lets thin kernels skip zeros).
void gemm_f64(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
              const double *A, int64_t lda, int64_t sA, const double *B, int64_t ldb,
              int64_t sB, double beta, double *C, int64_t ldc, int64_t sC, int64_t batch,
              cudaStream_t s, bool b_upper = false);
// Gaussian sketch: out[r*cols + c] from the counter-based SplitMix64 / Box-Muller rule
void fill_gaussian(double *out, int64_t rows, int64_t cols, uint64_t key, cudaStream_t s);
uint64_t sketch_key(uint64_t seed, int step, int tag);
// out[(j, b), m] = g2[j, m] * g1[b, m]   (Khatri-Rao sketch, rows (J, beta))
void khatri_rao(const double *g2, const double *g1, double *out, int64_t nj, int64_t nb,
                int64_t w, cudaStream_t s);
// x[i] *= f(v[(i / inner) % n])   mode 0: v, 1: pinv(v) (0 if v <= tol*max), 2: 1/sqrt
// (alive), 3: sqrt(max(v,0)); `vmax` is a device scalar (max of v) for modes 1, 2
void scale_axis(double *x, int64_t total, int64_t inner, int64_t n, const double *v,
                int mode, const double *vmax, double tol, cudaStream_t s);
// zero the entries of v (and of the matching columns of up to two matrices with n
// columns) whose value is <= tol * v[0] (v sorted descending, v >= 0)
void kill_dead(double *v, int64_t n, double tol, double *m1, int64_t rows1, double *m2,
               int64_t rows2, cudaStream_t s);
// deterministic dot product into a device scalar: *out = sum a[i] b[i]
void dot(const double *a, const double *b, int64_t n, double *out, double *scratch,
         cudaStream_t s);
// per-column sign gauge of an (rows x cols) row-major matrix (first entry within
// 1e-6 of the column's largest magnitude made positive); applied to m1 and m2
void sign_gauge(double *m1, int64_t rows1, double *m2, int64_t rows2, int64_t cols,
                cudaStream_t s);
void fill_identity(double *out, int64_t n, int64_t cols, cudaStream_t s);
void scale_by_scalar(double *x, int64_t n, const double *scalar, int mode, cudaStream_t s);
void axpby(double *y, const double *x, double a, double b, int64_t n, cudaStream_t s);
// step bookkeeping on device: c = sqrt(max(t, 0)); logsum += ln c * weight; flag non-finite
void norm_update(const double *tr, double *c_out, double *logsum, double weight, int *flag,
                 cudaStream_t s);
void col_max_abs(const double *v, int64_t n, double *out, cudaStream_t s);

// ------------------------------------------------------------- small linear algebra
// Upper Cholesky factor R (R^T R = G + shift_rel * trace(G) * I) and its inverse, one
// CTA per problem; a pivot <= rel_tol * max(diag G) marks the column dead (its rows of
// R and columns of Rinv are zero).  G, R, Rinv: batch x n x n row-major.
void chol_rinv(const double *G, double *R, double *Rinv, int n, int batch, double rel_tol,
               double shift_rel, cudaStream_t s);
// One-sided Jacobi SVD of batch m x n (m >= n) row-major matrices: A = U diag(S) V^T,
// S descending.  U: m x n, V: n x n (row-major).  info[b] = sweeps used, or -1 if the
// sweep limit was reached.  work: batch * (n*m + n*n) doubles.
// One problem with n >= 64 runs as a cooperative launch over many SMs (bounded grid
// barriers; a timed-out wait raises linalg_error_flag).  work: svd_jacobi_work doubles.
void svd_jacobi(const double *A, int m, int n, double *U, double *S, double *V, int batch,
                double *work, int *info, cudaStream_t s);
size_t svd_jacobi_work(int m, int n, int batch);
// nonzero if a grid barrier of the cooperative Jacobi timed out since the last reset
int linalg_error_flag(bool reset);

}  // namespace trg
