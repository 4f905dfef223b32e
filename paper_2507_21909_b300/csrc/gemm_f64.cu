// FP64 batched GEMM on CUDA cores (the parity form of every contraction).
// C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b], row-major; 64x64 tiles, BK = 16,
// 256 threads with 4x4 register tiles.  Ragged edges are zero-filled on load.
#include <algorithm>

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

static double *g_ws = nullptr;
static size_t g_ws_cap = 0;

void gemm_f64(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
              const double *A, int64_t lda, int64_t sA, const double *B, int64_t ldb,
              int64_t sB, double beta, double *C, int64_t ldc, int64_t sC, int64_t batch,
              cudaStream_t s) {
  if (M == 0 || N == 0 || batch == 0) return;
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
  if (nsplit > 1) {
    size_t need = (size_t)nsplit * batch * M * N * sizeof(double);
    if (need > g_ws_cap) {
      if (g_ws) {
        TRG_CUDA(cudaStreamSynchronize(s));
        TRG_CUDA(cudaFree(g_ws));
      }
      g_ws = nullptr;
      g_ws_cap = std::max(need, size_t(32) << 20);
      if (cudaMalloc(&g_ws, g_ws_cap) != cudaSuccess) {
        cudaGetLastError();
        g_ws_cap = 0;
        throw Error(TRG_ERR_OOM, "split-K workspace allocation failed");
      }
    }
  }
  int64_t gz = std::min<int64_t>(batch * nsplit, 65535);
  dim3 grid((unsigned)gy, (unsigned)gx, (unsigned)gz);  // M tiles on x (up to 2^31 - 1)
  gemm_f64_kernel<<<grid, 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta,
                                       C, ldc, sC, batch, kchunk, nsplit, g_ws);
  TRG_LAUNCH_CHECK();
  if (nsplit > 1) {
    int64_t total = batch * M * N;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 16);
    splitk_reduce<<<blocks, 256, 0, s>>>(g_ws, nsplit, batch, M, N, alpha, beta, C, ldc, sC);
    TRG_LAUNCH_CHECK();
  }
}

}  // namespace trg
