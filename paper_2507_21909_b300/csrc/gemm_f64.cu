// FP64 batched GEMM on CUDA cores (the parity form of every contraction).
// C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b], row-major; 64x64 tiles, BK = 16,
// 256 threads with 4x4 register tiles.  Ragged edges are zero-filled on load.
#include <algorithm>
#include <map>
#include <mutex>

#include "trg_internal.h"

namespace trg {

constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256)
gemm_f64_kernel(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                const double *__restrict__ A, int64_t lda, int64_t sA,
                const double *__restrict__ B, int64_t ldb, int64_t sB, double beta,
                double *__restrict__ C, int64_t ldc, int64_t sC, int64_t batch,
                int64_t kchunk, int nsplit, double *__restrict__ ws) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  for (int64_t z = blockIdx.z; z < batch * nsplit; z += gridDim.z) {
    const int64_t b = z / nsplit, sidx = z % nsplit;
    const int64_t kbeg = sidx * kchunk, kend = min(K, kbeg + kchunk);
    const double *Ab = A + b * sA;
    const double *Bb = B + b * sB;
    double acc[4][4] = {};
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
      for (int idx = tid; idx < BM * BK; idx += 256) {
        int mm, kk;
        if (ta) { mm = idx % BM; kk = idx / BM; } else { kk = idx % BK; mm = idx / BK; }
        int64_t gm = m0 + mm, gk = k0 + kk;
        double v = 0.0;
        if (gm < M && gk < kend) v = ta ? Ab[gk * lda + gm] : Ab[gm * lda + gk];
        As[kk][mm] = v;
      }
      for (int idx = tid; idx < BN * BK; idx += 256) {
        int nn, kk;
        if (tb) { kk = idx % BK; nn = idx / BK; } else { nn = idx % BN; kk = idx / BN; }
        int64_t gn = n0 + nn, gk = k0 + kk;
        double v = 0.0;
        if (gn < N && gk < kend) v = tb ? Bb[gn * ldb + gk] : Bb[gk * ldb + gn];
        Bs[kk][nn] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      }
      __syncthreads();
    }
    if (nsplit > 1) {  // partial sums to the split-K workspace [split][batch][M][N]
      double *W = ws + (sidx * batch + b) * M * N;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int64_t gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int64_t gn = n0 + tx + 16 * j;
          if (gn < N) W[gm * N + gn] = acc[i][j];
        }
      }
      continue;
    }
    double *Cb = C + b * sC;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int64_t gm = m0 + ty + 16 * i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int64_t gn = n0 + tx + 16 * j;
        if (gn >= N) continue;
        double *c = Cb + gm * ldc + gn;
        *c = (beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
      }
    }
  }
}

// C = alpha * sum_s W[s] + beta * C, in a fixed order (deterministic)
__global__ void splitk_reduce(const double *__restrict__ W, int nsplit, int64_t batch,
                              int64_t M, int64_t N, double alpha, double beta,
                              double *__restrict__ C, int64_t ldc, int64_t sC) {
  const int64_t total = batch * M * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += W[s * total + i];
    int64_t b = i / (M * N), mn = i % (M * N), m = mn / N, n = mn % N;
    double *c = C + b * sC + m * ldc + n;
    *c = (beta == 0.0) ? alpha * acc : alpha * acc + beta * *c;
  }
}


// ---------------------------------------------------------------- thin shapes
// Products whose output is at most 64 x 64 (CholeskyQR Grams Q^T Q and Q^T Y over
// millions of rows) and tall products with at most 64 inner and output columns (Q R^-1).
// FP64 issues only a few FMA per clock per SM, so these kernels spend it on the output
// that exists: exact R x R micro-tiles (R = ceil(max(M, N) / 16)) instead of 64 x 64
// tiles, the upper triangle of a symmetric Gram, and the nonzero rows of an upper
// triangular right factor.
constexpr int TBK = 32;

template <int R>
__global__ void __launch_bounds__(256)
gemm_f64_thin_kernel(bool ta, bool tb, int M, int N, int64_t K, const double *__restrict__ A,
                     int64_t lda, const double *__restrict__ B, int64_t ldb, int64_t kchunk,
                     int sym, double *__restrict__ ws) {
  __shared__ double As[TBK][64 + 1];
  __shared__ double Bs[TBK][64 + 1];
  const int tid = threadIdx.x;
  const int64_t kbeg = (int64_t)blockIdx.x * kchunk, kend = min(K, kbeg + kchunk);
  // micro-tile (ty, tx) of this thread.  A symmetric Gram needs only the 136 tiles with
  // ty <= tx; they go to the first threads, so that whole warps (not single lanes, which
  // would still cost their warp a slot) fall idle.
  int tx = tid % 16, ty = tid / 16;
  if (sym) {
    int q = tid, cg = 0;
    while (cg < 16 && q > cg) {
      q -= cg + 1;
      ++cg;
    }
    tx = cg;
    ty = cg < 16 ? q : 16;   // threads past the triangle get an empty tile
  }
  const int r0 = ty * R, c0 = tx * R;
  const bool active = r0 < M && c0 < N && ty < 16;
  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;
  for (int64_t k0 = kbeg; k0 < kend; k0 += TBK) {
    for (int idx = tid; idx < TBK * 64; idx += 256) {
      int mm, kk;
      if (ta) { mm = idx % 64; kk = idx / 64; } else { kk = idx % TBK; mm = idx / TBK; }
      const int64_t gk = k0 + kk;
      double v = 0.0;
      if (mm < M && gk < kend) v = ta ? A[gk * lda + mm] : A[(int64_t)mm * lda + gk];
      As[kk][mm] = v;
    }
    if (!sym) {
      for (int idx = tid; idx < TBK * 64; idx += 256) {
        int nn, kk;
        if (tb) { kk = idx % TBK; nn = idx / TBK; } else { nn = idx % 64; kk = idx / 64; }
        const int64_t gk = k0 + kk;
        double v = 0.0;
        if (nn < N && gk < kend) v = tb ? B[(int64_t)nn * ldb + gk] : B[gk * ldb + nn];
        Bs[kk][nn] = v;
      }
    }
    __syncthreads();
    if (active) {
      const double(*Bp)[65] = sym ? As : Bs;
#pragma unroll 4
      for (int kk = 0; kk < TBK; ++kk) {
        double a[R], b[R];
#pragma unroll
        for (int i = 0; i < R; ++i) a[i] = As[kk][r0 + i];
#pragma unroll
        for (int j = 0; j < R; ++j) b[j] = Bp[kk][c0 + j];
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
          for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  if (!active) return;
  double *W = ws + (int64_t)blockIdx.x * M * N;
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int m = r0 + i, n = c0 + j;
      if (m < M && n < N) W[(int64_t)m * N + n] = acc[i][j];
    }
}

// C = alpha * sum_s W[s] + beta * C in split order; a symmetric Gram reads the upper
// triangle for both halves
__global__ void thin_reduce(const double *__restrict__ W, int nsplit, int M, int N, double alpha,
                            double beta, double *__restrict__ C, int64_t ldc, int sym) {
  const int total = M * N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int m = i / N, n = i % N;
    const int src = sym ? min(m, n) * N + max(m, n) : i;
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += W[(int64_t)s * total + src];
    double *c = C + (int64_t)m * ldc + n;
    *c = (beta == 0.0) ? alpha * acc : alpha * acc + beta * *c;
  }
}

// C (M x N) = alpha A (M x K) B (K x N) + beta C with K, N <= 64 and M large; B is read
// once per CTA.  b_upper: B is upper triangular, so column j only needs rows k <= j.
template <int R>
__global__ void __launch_bounds__(256)
gemm_f64_tall_kernel(int64_t M, int N, int K, double alpha, const double *__restrict__ A,
                     int64_t lda, const double *__restrict__ B, int64_t ldb, double beta,
                     double *__restrict__ C, int64_t ldc, int b_upper) {
  extern __shared__ double tall_smem[];  // B (64 x 65) then the A tile (64 x 65)
  double(*Bs)[65] = reinterpret_cast<double(*)[65]>(tall_smem);
  double(*As)[65] = reinterpret_cast<double(*)[65]>(tall_smem + 64 * 65);
  // column group per half-warp (tx), row group per lane (ty): with an upper-triangular B
  // the loop over k stops at the group's last column for the whole half-warp
  const int tid = threadIdx.x, tx = tid / 16, ty = tid % 16;
  for (int idx = tid; idx < 64 * 64; idx += 256) {
    const int kk = idx / 64, nn = idx % 64;
    Bs[kk][nn] = (kk < K && nn < N) ? B[(int64_t)kk * ldb + nn] : 0.0;
  }
  const int c0 = tx * R;
  const int kmax = b_upper ? min(K, c0 + R) : K;
  const int64_t ntiles = (M + 63) / 64;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t m0 = t * 64;
    __syncthreads();
    for (int idx = tid; idx < 64 * 64; idx += 256) {
      const int mm = idx / 64, kk = idx % 64;
      As[mm][kk] = (m0 + mm < M && kk < K) ? A[(m0 + mm) * lda + kk] : 0.0;
    }
    __syncthreads();
    if (c0 >= N) continue;
    double acc[4][R];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[i][j] = 0.0;
    for (int kk = 0; kk < kmax; ++kk) {
      double a[4], b[R];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[ty * 4 + i][kk];
#pragma unroll
      for (int j = 0; j < R; ++j) b[j] = Bs[kk][c0 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t m = m0 + ty * 4 + i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int n = c0 + j;
        if (n >= N) continue;
        double *c = C + m * ldc + n;
        *c = (beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
      }
    }
  }
}

// split-K workspace, one per stream (batched instances run on several streams at once)
struct Workspace {
  double *p = nullptr;
  size_t cap = 0;
};
static std::mutex g_ws_mu;
static std::map<cudaStream_t, Workspace> g_ws;

static double *ensure_ws(size_t need, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  Workspace &w = g_ws[s];
  if (need <= w.cap) return w.p;
  if (w.p) {
    TRG_CUDA(cudaStreamSynchronize(s));
    TRG_CUDA(cudaFree(w.p));
  }
  w.p = nullptr;
  w.cap = std::max(need, size_t(32) << 20);
  if (cudaMalloc(&w.p, w.cap) != cudaSuccess) {
    cudaGetLastError();
    w.cap = 0;
    throw Error(TRG_ERR_OOM, "split-K workspace allocation failed");
  }
  return w.p;
}

template <int R>
static void launch_thin(bool ta, bool tb, int M, int N, int64_t K, const double *A,
                        int64_t lda, const double *B, int64_t ldb, int64_t kchunk, int nsplit,
                        int sym, double *ws, cudaStream_t s) {
  gemm_f64_thin_kernel<R><<<nsplit, 256, 0, s>>>(ta, tb, M, N, K, A, lda, B, ldb, kchunk, sym,
                                                 ws);
}
template <int R>
static void launch_tall(int64_t M, int N, int K, double alpha, const double *A, int64_t lda,
                        const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                        int b_upper, cudaStream_t s) {
  constexpr int kSmem = 2 * 64 * 65 * (int)sizeof(double);
  // thread-safe one-time setup (function-local static initialisation)
  static const bool attr_done = [&] {
    TRG_CUDA(cudaFuncSetAttribute(gemm_f64_tall_kernel<R>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
    return true;
  }();
  (void)attr_done;
  const int64_t tiles = (M + 63) / 64;
  const int grid = (int)std::min<int64_t>(tiles, 148 * 3);
  gemm_f64_tall_kernel<R><<<grid, 256, kSmem, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                   b_upper);
}

void gemm_f64(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
              const double *A, int64_t lda, int64_t sA, const double *B, int64_t ldb,
              int64_t sB, double beta, double *C, int64_t ldc, int64_t sC, int64_t batch,
              cudaStream_t s, bool b_upper) {
  if (M == 0 || N == 0 || batch == 0) return;
  if (batch == 1 && M <= 64 && N <= 64 && K >= 4096) {
    const int sym = (A == B && ta != tb && M == N && lda == ldb) ? 1 : 0;
    const int nsplit = (int)std::min<int64_t>((K + 1023) / 1024, 148 * 4);
    int64_t kchunk = (K + nsplit - 1) / nsplit;
    kchunk = (kchunk + TBK - 1) / TBK * TBK;
    double *ws = ensure_ws((size_t)nsplit * M * N * sizeof(double), s);
    const int R = (int)((std::max(M, N) + 15) / 16);
    switch (R) {
      case 1: launch_thin<1>(ta, tb, (int)M, (int)N, K, A, lda, B, ldb, kchunk, nsplit, sym, ws, s); break;
      case 2: launch_thin<2>(ta, tb, (int)M, (int)N, K, A, lda, B, ldb, kchunk, nsplit, sym, ws, s); break;
      case 3: launch_thin<3>(ta, tb, (int)M, (int)N, K, A, lda, B, ldb, kchunk, nsplit, sym, ws, s); break;
      default: launch_thin<4>(ta, tb, (int)M, (int)N, K, A, lda, B, ldb, kchunk, nsplit, sym, ws, s); break;
    }
    TRG_LAUNCH_CHECK();
    const int blocks = (int)std::min<int64_t>((M * N + 255) / 256, 148);
    thin_reduce<<<blocks, 256, 0, s>>>(ws, nsplit, (int)M, (int)N, alpha, beta, C, ldc, sym);
    TRG_LAUNCH_CHECK();
    return;
  }
  if (batch == 1 && !ta && !tb && K <= 64 && N <= 64 && M >= 4096) {
    const int R = (int)((N + 15) / 16);
    switch (R) {
      case 1: launch_tall<1>(M, (int)N, (int)K, alpha, A, lda, B, ldb, beta, C, ldc, b_upper, s); break;
      case 2: launch_tall<2>(M, (int)N, (int)K, alpha, A, lda, B, ldb, beta, C, ldc, b_upper, s); break;
      case 3: launch_tall<3>(M, (int)N, (int)K, alpha, A, lda, B, ldb, beta, C, ldc, b_upper, s); break;
      default: launch_tall<4>(M, (int)N, (int)K, alpha, A, lda, B, ldb, beta, C, ldc, b_upper, s); break;
    }
    TRG_LAUNCH_CHECK();
    return;
  }
  int64_t gy = (M + BM - 1) / BM, gx = (N + BN - 1) / BN;
  if (gx > 65535) throw Error(TRG_ERR_ARG, "gemm_f64: N too large for one launch");
  // split K when the output tiles alone cannot fill the 148 SMs
  int nsplit = 1;
  const int64_t tiles = gx * gy * batch;
  if (tiles < 296 && K >= 1024) {
    int64_t want = (2 * 296 + tiles - 1) / tiles;
    int64_t maxs = (K + 255) / 256;
    nsplit = (int)std::min<int64_t>(std::min<int64_t>(want, maxs), 256);
    if (nsplit < 2) nsplit = 1;
  }
  int64_t kchunk = (K + nsplit - 1) / nsplit;
  kchunk = ((kchunk + BK - 1) / BK) * BK;
  double *ws = nsplit > 1 ? ensure_ws((size_t)nsplit * batch * M * N * sizeof(double), s) : nullptr;
  int64_t gz = std::min<int64_t>(batch * nsplit, 65535);
  dim3 grid((unsigned)gy, (unsigned)gx, (unsigned)gz);  // M tiles on x (up to 2^31 - 1)
  gemm_f64_kernel<<<grid, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta,
                                       C, ldc, sC, batch, kchunk, nsplit, ws);
  TRG_LAUNCH_CHECK();
  if (nsplit > 1) {
    int64_t total = batch * M * N;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 16);
    splitk_reduce<<<blocks, 256, 0, s>>>(ws, nsplit, batch, M, N, alpha, beta, C, ldc, sC);
    TRG_LAUNCH_CHECK();
  }
}

}  // namespace trg
