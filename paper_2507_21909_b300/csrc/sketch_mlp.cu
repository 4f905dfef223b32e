// Learned sketch for the range finders of the triad isometries (Sec. II B, eq. HOSVD).
//
// The range finder of each Gram rho (n x n over the leg pair, n = da db) starts from a
// Gaussian sketch G (n x chi).  The learned variant rescales the rows of the same G:
//     Omega[(a b), m] = w1[a] w2[b] G[(a b), m],   w_l[i] = 2^(round(16 u_l[i]) / 16),
// where u_l[i] is the output of a 3-layer MLP (5 -> 256 -> 256 -> 1, ReLU) on five
// statistics of index i of leg l: its position, the share of tr(rho) on its diagonal
// entries, both leg sizes and chi / n.  The network is trained on targets the plain
// method produces, 0.5 log2(leverage * d) of each leg index in the converged range.
// Inference runs with BF16 inputs, weights and hidden activations and FP32 sums; the
// training path (forward, backward, Adam) is FP32.  All kernels are deterministic.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>
#include <vector>

#include "sketch_mlp.h"
#include "trg_internal.h"

namespace trg {

// ------------------------------------------------------------------ FP32 GEMM
__global__ void __launch_bounds__(256)
sgemm_kernel(bool ta, bool tb, int64_t M, int64_t N, int64_t K, float alpha,
             const float *__restrict__ A, int64_t lda, const float *__restrict__ B, int64_t ldb,
             float beta, float *__restrict__ C, int64_t ldc) {
  __shared__ float As[16][65], Bs[16][65];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.x * 64, n0 = (int64_t)blockIdx.y * 64;
  float acc[4][4] = {};
  for (int64_t k0 = 0; k0 < K; k0 += 16) {
    for (int idx = tid; idx < 1024; idx += 256) {
      int mm, kk;
      if (ta) { mm = idx % 64; kk = idx / 64; } else { kk = idx % 16; mm = idx / 16; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < K) v = ta ? A[gk * lda + gm] : A[gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int idx = tid; idx < 1024; idx += 256) {
      int nn, kk;
      if (tb) { kk = idx % 16; nn = idx / 16; } else { nn = idx % 64; kk = idx / 64; }
      const int64_t gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < N && gk < K) v = tb ? B[gn * ldb + gk] : B[gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      float *c = C + gm * ldc + gn;
      *c = beta == 0.f ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
    }
  }
}

void sgemm(bool ta, bool tb, int64_t M, int64_t N, int64_t K, float alpha, const float *A,
           int64_t lda, const float *B, int64_t ldb, float beta, float *C, int64_t ldc,
           cudaStream_t s) {
  if (M == 0 || N == 0) return;
  const int64_t gx = (M + 63) / 64, gy = (N + 63) / 64;
  if (gy > 65535) throw Error(TRG_ERR_ARG, "sgemm: N too large");
  sgemm_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(ta, tb, M, N, K, alpha, A, lda,
                                                               B, ldb, beta, C, ldc);
  TRG_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ small kernels
static int blocks_for(int64_t n) {
  return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 148 * 8);
}

// Z[r, j] += b[j]; H = relu(Z) (H may alias nothing)
__global__ void bias_relu_kernel(float *Z, float *H, const float *b, int64_t rows, int cols,
                                 int relu) {
  const int64_t n = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float z = Z[i] + b[i % cols];
    Z[i] = z;
    if (H) H[i] = relu ? fmaxf(z, 0.f) : z;
  }
}

// du = 2 (u - t) / n and per-block partial sums of (u - t)^2
__global__ void loss_grad_kernel(const float *u, const float *t, int64_t n, float *du,
                                 double *partial) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float e = u[i] - t[i];
    du[i] = 2.f * e / (float)n;
    acc += (double)e * e;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// dZ2[r, j] = du[r] W3[j] (Z2[r, j] > 0)
__global__ void dz2_kernel(const float *du, const float *W3, const float *Z2, int64_t rows,
                           int hid, float *dZ2) {
  const int64_t n = rows * hid;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / hid;
    const int j = (int)(i % hid);
    dZ2[i] = Z2[i] > 0.f ? du[r] * W3[j] : 0.f;
  }
}

__global__ void relu_mask_kernel(float *dH, const float *Z, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!(Z[i] > 0.f)) dH[i] = 0.f;
}

// out[j] = sum_r M[r, j] (fixed order per column)
__global__ void colsum_kernel(const float *M, int64_t rows, int cols, float *out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cols; j += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t r = 0; r < rows; ++r) acc += M[r * cols + j];
    out[j] = (float)acc;
  }
}

__global__ void adam_kernel(float *w, const float *g, float *m, float *v, int64_t n, float lr,
                            float b1t, float b2t) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / (1.f - b1t)) / (sqrtf(vi / (1.f - b2t)) + eps);
  }
}

__global__ void to_bf16_kernel(const float *w, __nv_bfloat16 *wb, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}

__global__ void gather_rows_kernel(const float *X, const float *t, const int *idx, int64_t n,
                                   float *Xb, float *tb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx[i];
    for (int k = 0; k < kMlpIn; ++k) Xb[i * kMlpIn + k] = X[r * kMlpIn + k];
    tb[i] = t[r];
  }
}

// ------------------------------------------------------------------ BF16 inference
// One block of 256 threads (thread j = hidden unit j) keeps W2^T in shared memory as
// BF16 and runs tiles of 32 rows: h1 (BF16) -> h2 (FP32 sums, BF16) -> u.
constexpr int kInferRows = 32;
constexpr size_t kInferSmem =
    (size_t)kMlpHid * kMlpHid * 2 + (size_t)kInferRows * kMlpHid * 2 + kInferRows * 8 * 4;

__global__ void __launch_bounds__(kMlpHid)
mlp_infer_kernel(const __nv_bfloat16 *__restrict__ wb, const float *__restrict__ w,
                 const float *__restrict__ X, int64_t rows, float *__restrict__ u) {
  extern __shared__ __align__(16) uint8_t sm[];
  __nv_bfloat16 *W2T = reinterpret_cast<__nv_bfloat16 *>(sm);                 // [k][j]
  __nv_bfloat16 *H1 = W2T + kMlpHid * kMlpHid;                               // [r][k]
  float *red = reinterpret_cast<float *>(H1 + kInferRows * kMlpHid);         // [r][warp]
  const int j = threadIdx.x, lane = j & 31, wrp = j >> 5;
  for (int idx = j; idx < kMlpHid * kMlpHid; idx += kMlpHid) {
    const int jj = idx / kMlpHid, k = idx % kMlpHid;   // W2[jj][k]
    W2T[k * kMlpHid + jj] = wb[kOffW2 + idx];
  }
  float w1[kMlpIn];
#pragma unroll
  for (int i = 0; i < kMlpIn; ++i) w1[i] = __bfloat162float(wb[kOffW1 + j * kMlpIn + i]);
  const float b1 = w[kOffB1 + j], b2 = w[kOffB2 + j], b3 = w[kOffB3];
  const float w3 = __bfloat162float(wb[kOffW3 + j]);
  __syncthreads();
  for (int64_t r0 = (int64_t)blockIdx.x * kInferRows; r0 < rows;
       r0 += (int64_t)gridDim.x * kInferRows) {
    const int nr = rows - r0 < kInferRows ? (int)(rows - r0) : kInferRows;
    for (int r = 0; r < nr; ++r) {
      float z = b1;
#pragma unroll
      for (int i = 0; i < kMlpIn; ++i)
        z = fmaf(w1[i], __bfloat162float(__float2bfloat16_rn(X[(r0 + r) * kMlpIn + i])), z);
      H1[r * kMlpHid + j] = __float2bfloat16_rn(fmaxf(z, 0.f));
    }
    __syncthreads();
    float acc[kInferRows];
#pragma unroll
    for (int r = 0; r < kInferRows; ++r) acc[r] = 0.f;
    for (int k = 0; k < kMlpHid; ++k) {
      const float wk = __bfloat162float(W2T[k * kMlpHid + j]);
#pragma unroll
      for (int r = 0; r < kInferRows; ++r)
        acc[r] = fmaf(wk, __bfloat162float(H1[r * kMlpHid + k]), acc[r]);
    }
#pragma unroll
    for (int r = 0; r < kInferRows; ++r) {
      const float h2 = __bfloat162float(__float2bfloat16_rn(fmaxf(acc[r] + b2, 0.f)));
      float pr = w3 * h2;
      for (int o = 16; o > 0; o >>= 1) pr += __shfl_xor_sync(0xffffffffu, pr, o);
      if (lane == 0) red[r * 8 + wrp] = pr;
    }
    __syncthreads();
    if (j < nr) {
      float sum = b3;
      for (int q = 0; q < 8; ++q) sum += red[j * 8 + q];
      u[r0 + j] = sum;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ scratch
namespace {
struct Buf {
  void *p = nullptr;
  size_t cap = 0;
  void *get(size_t bytes, cudaStream_t s) {
    if (bytes > cap) {
      if (p) {
        TRG_CUDA(cudaStreamSynchronize(s));
        TRG_CUDA(cudaFree(p));
      }
      p = nullptr;
      cap = 0;
      if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        throw Error(TRG_ERR_OOM, "sketch network scratch allocation failed");
      }
      cap = bytes;
    }
    return p;
  }
};
Buf g_z1, g_h1, g_z2, g_h2, g_u, g_du, g_dz2, g_dh1, g_part, g_xb, g_tb, g_idx, g_grad;
}  // namespace

static void ensure_net(SketchNet &net) {
  if (net.w) return;
  const size_t fb = kMlpParams * sizeof(float);
  if (cudaMalloc(&net.w, fb) != cudaSuccess || cudaMalloc(&net.m, fb) != cudaSuccess ||
      cudaMalloc(&net.v, fb) != cudaSuccess ||
      cudaMalloc(&net.wb, kMlpParams * sizeof(__nv_bfloat16)) != cudaSuccess) {
    cudaGetLastError();
    throw Error(TRG_ERR_OOM, "sketch network allocation failed");
  }
}

static void refresh_bf16(SketchNet &net, cudaStream_t s) {
  to_bf16_kernel<<<blocks_for(kMlpParams), 256, 0, s>>>(net.w, net.wb, kMlpParams);
  TRG_LAUNCH_CHECK();
}

void mlp_set(SketchNet &net, const float *host, cudaStream_t s) {
  ensure_net(net);
  const size_t fb = kMlpParams * sizeof(float);
  TRG_CUDA(cudaMemcpyAsync(net.w, host, fb, cudaMemcpyHostToDevice, s));
  TRG_CUDA(cudaMemsetAsync(net.m, 0, fb, s));
  TRG_CUDA(cudaMemsetAsync(net.v, 0, fb, s));
  net.adam_t = 0;
  refresh_bf16(net, s);
  net.loaded = true;
}

void mlp_get(const SketchNet &net, float *host, cudaStream_t s) {
  if (!net.loaded) throw Error(TRG_ERR_NOINIT, "no sketch network loaded");
  TRG_CUDA(cudaMemcpyAsync(host, net.w, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, s));
  TRG_CUDA(cudaStreamSynchronize(s));
}

// FP32 forward; keeps Z1, H1, Z2, H2 in the scratch buffers
static float *forward_f32(const SketchNet &net, const float *X, int64_t rows, cudaStream_t s) {
  const size_t hb = (size_t)rows * kMlpHid * sizeof(float);
  float *Z1 = (float *)g_z1.get(hb, s), *H1 = (float *)g_h1.get(hb, s);
  float *Z2 = (float *)g_z2.get(hb, s), *H2 = (float *)g_h2.get(hb, s);
  float *U = (float *)g_u.get((size_t)rows * sizeof(float), s);
  sgemm(false, true, rows, kMlpHid, kMlpIn, 1.f, X, kMlpIn, net.w + kOffW1, kMlpIn, 0.f, Z1,
        kMlpHid, s);
  bias_relu_kernel<<<blocks_for(rows * kMlpHid), 256, 0, s>>>(Z1, H1, net.w + kOffB1, rows,
                                                              kMlpHid, 1);
  TRG_LAUNCH_CHECK();
  sgemm(false, true, rows, kMlpHid, kMlpHid, 1.f, H1, kMlpHid, net.w + kOffW2, kMlpHid, 0.f, Z2,
        kMlpHid, s);
  bias_relu_kernel<<<blocks_for(rows * kMlpHid), 256, 0, s>>>(Z2, H2, net.w + kOffB2, rows,
                                                              kMlpHid, 1);
  TRG_LAUNCH_CHECK();
  sgemm(false, true, rows, 1, kMlpHid, 1.f, H2, kMlpHid, net.w + kOffW3, kMlpHid, 0.f, U, 1, s);
  bias_relu_kernel<<<blocks_for(rows), 256, 0, s>>>(U, nullptr, net.w + kOffB3, rows, 1, 0);
  TRG_LAUNCH_CHECK();
  return U;
}

void mlp_forward(const SketchNet &net, const float *X, int64_t rows, float *u, bool bf16,
                 cudaStream_t s) {
  if (!net.loaded) throw Error(TRG_ERR_NOINIT, "no sketch network loaded");
  if (rows <= 0) return;
  if (!bf16) {
    float *U = forward_f32(net, X, rows, s);
    TRG_CUDA(cudaMemcpyAsync(u, U, rows * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return;
  }
  // thread-safe one-time setup (function-local static initialisation)
  static const bool attr_done = [&] {
    TRG_CUDA(cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kInferSmem));
    return true;
  }();
  (void)attr_done;
  const int grid = (int)std::min<int64_t>((rows + kInferRows - 1) / kInferRows, 148);
  mlp_infer_kernel<<<grid, kMlpHid, kInferSmem, s>>>(net.wb, net.w, X, rows, u);
  TRG_LAUNCH_CHECK();
}

double mlp_grad(const SketchNet &net, const float *X, const float *t, int64_t rows, float *grad,
                cudaStream_t s) {
  if (!net.loaded) throw Error(TRG_ERR_NOINIT, "no sketch network loaded");
  if (rows <= 0) throw Error(TRG_ERR_ARG, "mlp_grad: no rows");
  float *U = forward_f32(net, X, rows, s);
  float *Z1 = (float *)g_z1.p, *H1 = (float *)g_h1.p, *Z2 = (float *)g_z2.p,
        *H2 = (float *)g_h2.p;
  const size_t hb = (size_t)rows * kMlpHid * sizeof(float);
  float *du = (float *)g_du.get((size_t)rows * sizeof(float), s);
  const int nb = blocks_for(rows);
  double *part = (double *)g_part.get((size_t)nb * sizeof(double), s);
  loss_grad_kernel<<<nb, 256, 0, s>>>(U, t, rows, du, part);
  TRG_LAUNCH_CHECK();
  float *dZ2 = (float *)g_dz2.get(hb, s), *dH1 = (float *)g_dh1.get(hb, s);
  // layer 3: gW3 = du^T H2, gb3 = sum du
  sgemm(true, false, 1, kMlpHid, rows, 1.f, du, 1, H2, kMlpHid, 0.f, grad + kOffW3, kMlpHid, s);
  colsum_kernel<<<1, 32, 0, s>>>(du, rows, 1, grad + kOffB3);
  TRG_LAUNCH_CHECK();
  // layer 2
  dz2_kernel<<<blocks_for(rows * kMlpHid), 256, 0, s>>>(du, net.w + kOffW3, Z2, rows, kMlpHid,
                                                        dZ2);
  TRG_LAUNCH_CHECK();
  sgemm(true, false, kMlpHid, kMlpHid, rows, 1.f, dZ2, kMlpHid, H1, kMlpHid, 0.f,
        grad + kOffW2, kMlpHid, s);
  colsum_kernel<<<1, kMlpHid, 0, s>>>(dZ2, rows, kMlpHid, grad + kOffB2);
  TRG_LAUNCH_CHECK();
  // layer 1
  sgemm(false, false, rows, kMlpHid, kMlpHid, 1.f, dZ2, kMlpHid, net.w + kOffW2, kMlpHid, 0.f,
        dH1, kMlpHid, s);
  relu_mask_kernel<<<blocks_for(rows * kMlpHid), 256, 0, s>>>(dH1, Z1, rows * kMlpHid);
  TRG_LAUNCH_CHECK();
  sgemm(true, false, kMlpHid, kMlpIn, rows, 1.f, dH1, kMlpHid, X, kMlpIn, 0.f, grad + kOffW1,
        kMlpIn, s);
  colsum_kernel<<<1, kMlpHid, 0, s>>>(dH1, rows, kMlpHid, grad + kOffB1);
  TRG_LAUNCH_CHECK();
  std::vector<double> hp(nb);
  TRG_CUDA(cudaMemcpyAsync(hp.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
  TRG_CUDA(cudaStreamSynchronize(s));
  double sum = 0.0;
  for (double v : hp) sum += v;
  return sum / (double)rows;
}

double mlp_train(SketchNet &net, const float *X, const float *t, int64_t rows, int epochs,
                 int batch, float lr, uint64_t seed, cudaStream_t s) {
  if (!net.loaded) throw Error(TRG_ERR_NOINIT, "no sketch network loaded");
  if (rows <= 0 || epochs <= 0 || batch <= 0) throw Error(TRG_ERR_ARG, "mlp_train: bad sizes");
  const int64_t bs = std::min<int64_t>(batch, rows);
  float *Xb = (float *)g_xb.get((size_t)bs * kMlpIn * sizeof(float), s);
  float *tb = (float *)g_tb.get((size_t)bs * sizeof(float), s);
  int *idx = (int *)g_idx.get((size_t)rows * sizeof(int), s);
  float *grad = (float *)g_grad.get(kMlpParams * sizeof(float), s);
  std::vector<int> perm(rows);
  std::mt19937_64 gen(seed);
  double epoch_loss = 0.0;
  for (int e = 0; e < epochs; ++e) {
    std::iota(perm.begin(), perm.end(), 0);
    std::shuffle(perm.begin(), perm.end(), gen);
    TRG_CUDA(cudaMemcpyAsync(idx, perm.data(), rows * sizeof(int), cudaMemcpyHostToDevice, s));
    double acc = 0.0;
    int64_t seen = 0;
    for (int64_t b0 = 0; b0 + bs <= rows; b0 += bs) {
      gather_rows_kernel<<<blocks_for(bs), 256, 0, s>>>(X, t, idx + b0, bs, Xb, tb);
      TRG_LAUNCH_CHECK();
      acc += mlp_grad(net, Xb, tb, bs, grad, s) * (double)bs;
      seen += bs;
      ++net.adam_t;
      adam_kernel<<<blocks_for(kMlpParams), 256, 0, s>>>(
          net.w, grad, net.m, net.v, kMlpParams, lr, (float)std::pow(0.9, (double)net.adam_t),
          (float)std::pow(0.999, (double)net.adam_t));
      TRG_LAUNCH_CHECK();
    }
    epoch_loss = seen ? acc / (double)seen : 0.0;
  }
  refresh_bf16(net, s);
  TRG_CUDA(cudaStreamSynchronize(s));
  return epoch_loss;
}

// ------------------------------------------------------------------ step helpers
// diag[i * stride] is rho's diagonal entry i (stride n + 1 for rho itself, 1 for a
// vector of row norms^2 of a factor F with rho = F F^T)
__global__ void features_kernel(const double *diag, int64_t stride, int da, int db, int chi,
                                float *F) {
  __shared__ double s_tr;
  const int n = da * db;
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += diag[(int64_t)i * stride];
    s_tr = tr;
  }
  __syncthreads();
  const double tr = s_tr;
  for (int row = threadIdx.x; row < da + db; row += blockDim.x) {
    const bool first = row < da;
    const int i = first ? row : row - da;
    const int d = first ? da : db, dother = first ? db : da;
    double m = 0.0;
    for (int o = 0; o < dother; ++o) {
      const int64_t idx = first ? (int64_t)i * db + o : (int64_t)o * db + i;
      m += diag[idx * stride];
    }
    m = tr > 0.0 ? m / tr : 0.0;
    float *f = F + (int64_t)row * kMlpIn;
    f[0] = (float)((i + 0.5) / d);
    f[1] = (float)(log2(fmax(m * d, 0x1.0p-40)) / 8.0);  // floor above rounding noise
    f[2] = (float)(log2((double)d) / 8.0);
    f[3] = (float)(log2((double)dother) / 8.0);
    f[4] = (float)((double)chi / n);
  }
}

void sketch_features(const double *rho, int da, int db, int chi, float *F, cudaStream_t s) {
  features_kernel<<<1, 256, 0, s>>>(rho, (int64_t)da * db + 1, da, db, chi, F);
  TRG_LAUNCH_CHECK();
}

// one warp per row: out[r] = sum_m F[r, m]^2
__global__ void row_sumsq_kernel(const double *F, int64_t n, int64_t m, double *out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nw) {
    double acc = 0.0;
    for (int64_t k = lane; k < m; k += 32) {
      const double v = F[r * m + k];
      acc += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[r] = acc;
  }
}

void sketch_features_factor(const double *Fm, int64_t m, int da, int db, int chi,
                            double *diag_scratch, float *F, cudaStream_t s) {
  const int64_t n = (int64_t)da * db;
  const int blocks = (int)std::min<int64_t>((n * 32 + 255) / 256, 148 * 8);
  row_sumsq_kernel<<<blocks, 256, 0, s>>>(Fm, n, m, diag_scratch);
  TRG_LAUNCH_CHECK();
  features_kernel<<<1, 256, 0, s>>>(diag_scratch, 1, da, db, chi, F);
  TRG_LAUNCH_CHECK();
}

__device__ __forceinline__ double weight_of(float u) {
  const float c = fminf(fmaxf(rintf(u * kQuantStep), -kQuantMax * kQuantStep),
                        kQuantMax * kQuantStep);
  return exp2((double)c / (double)kQuantStep);
}

__global__ void row_weights_kernel(const float *u, int da, int db, double *w) {
  const int n = da * db;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    w[i] = weight_of(u[i / db]) * weight_of(u[da + i % db]);
}

void sketch_row_weights(const float *u, int da, int db, double *w, cudaStream_t s) {
  row_weights_kernel<<<blocks_for((int64_t)da * db), 256, 0, s>>>(u, da, db, w);
  TRG_LAUNCH_CHECK();
}

// one block: column norms -> number of live columns c; leverages of both legs
__global__ void leverage_kernel(const double *Q, int da, int db, int ccols, float *t) {
  __shared__ int s_live;
  const int n = da * db;
  if (threadIdx.x == 0) s_live = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < ccols; k += blockDim.x) {
    double v = 0.0;
    for (int r = 0; r < n; ++r) v += Q[(int64_t)r * ccols + k] * Q[(int64_t)r * ccols + k];
    if (sqrt(v) > 0.5) atomicAdd(&s_live, 1);
  }
  __syncthreads();
  const double c = (double)max(s_live, 1);
  for (int row = threadIdx.x; row < da + db; row += blockDim.x) {
    const bool first = row < da;
    const int i = first ? row : row - da;
    const int d = first ? da : db, dother = first ? db : da;
    double lev = 0.0;
    for (int o = 0; o < dother; ++o) {
      const int64_t r = first ? (int64_t)i * db + o : (int64_t)o * db + i;
      for (int k = 0; k < ccols; ++k) lev += Q[r * ccols + k] * Q[r * ccols + k];
    }
    lev /= c;
    t[row] = (float)(0.5 * log2(fmax(lev * d, 0x1.0p-40)));
  }
}

void leverage_targets(const double *Q, int da, int db, int c, float *t, cudaStream_t s) {
  leverage_kernel<<<1, 256, 0, s>>>(Q, da, db, c, t);
  TRG_LAUNCH_CHECK();
}

__global__ void scale_rows_kernel(double *x, int64_t rows, int64_t cols, const double *w) {
  const int64_t n = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= w[i / cols];
}

void scale_rows(double *x, int64_t rows, int64_t cols, const double *w, cudaStream_t s) {
  scale_rows_kernel<<<blocks_for(rows * cols), 256, 0, s>>>(x, rows, cols, w);
  TRG_LAUNCH_CHECK();
}

__global__ void select_kernel(const double *A, const double *B, int64_t n, const double *r_l,
                              const double *r_p, double ratio, double *out,
                              unsigned long long *counters) {
  const bool use_a = *r_l <= ratio * *r_p;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = use_a ? A[i] : B[i];
  if (blockIdx.x == 0 && threadIdx.x == 0 && counters) atomicAdd(&counters[use_a ? 0 : 1], 1ull);
}

void select_range(const double *A, const double *B, int64_t n, const double *r_l,
                  const double *r_p, double ratio, double *out, unsigned long long *counters,
                  cudaStream_t s) {
  select_kernel<<<blocks_for(n), 256, 0, s>>>(A, B, n, r_l, r_p, ratio, out, counters);
  TRG_LAUNCH_CHECK();
}

}  // namespace trg
