// Small dense FP64 linear algebra, one CTA per problem:
//   * chol_rinv: upper Cholesky factor R of G (+ a relative diagonal shift) and R^{-1},
//     with dead (non-positive) pivots mapped to zero rows/columns;
//   * svd_jacobi: one-sided (Hestenes) Jacobi SVD with round-robin pair ordering, which
//     keeps high relative accuracy of small singular values (Demmel & Veselic 1992).
#include "trg_internal.h"

namespace trg {

// ------------------------------------------------------------------ Cholesky
__global__ void chol_rinv_kernel(const double *G, double *R, double *Rinv, int n,
                                 double rel_tol, double shift_rel) {
  const int64_t off = (int64_t)blockIdx.x * n * n;
  const double *g = G + off;
  double *r = R + off;
  double *x = Rinv + off;
  __shared__ double s_scale, s_shift, s_piv;
  __shared__ int s_dead;
  if (threadIdx.x == 0) {
    double mx = 0.0, tr = 0.0;
    for (int i = 0; i < n; ++i) {
      mx = fmax(mx, g[(int64_t)i * n + i]);
      tr += g[(int64_t)i * n + i];
    }
    s_scale = mx;
    s_shift = shift_rel * tr;
  }
  __syncthreads();
  // working copy of the upper triangle (+ shift) in R
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += blockDim.x) {
    int i = (int)(idx / n), j = (int)(idx % n);
    r[idx] = (j >= i) ? g[idx] + (i == j ? s_shift : 0.0) : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double p = r[(int64_t)j * n + j];
      s_dead = !(p > rel_tol * s_scale && p > 0.0);
      s_piv = s_dead ? 0.0 : sqrt(p);
    }
    __syncthreads();
    const double piv = s_piv;
    if (s_dead) {
      for (int i = j + threadIdx.x; i < n; i += blockDim.x) r[(int64_t)j * n + i] = 0.0;
      __syncthreads();
      continue;
    }
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) r[(int64_t)j * n + i] /= piv;
    __syncthreads();
    if (threadIdx.x == 0) r[(int64_t)j * n + j] = piv;
    const int t = n - j - 1;
    for (int64_t idx = threadIdx.x; idx < (int64_t)t * t; idx += blockDim.x) {
      int a = j + 1 + (int)(idx / t), b = j + 1 + (int)(idx % t);
      if (b >= a) r[(int64_t)a * n + b] -= r[(int64_t)j * n + a] * r[(int64_t)j * n + b];
    }
    __syncthreads();
  }
  // inverse of the upper-triangular R, one thread per column; dead rows give zeros
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    for (int i = 0; i < n; ++i)
      if (i > c) x[(int64_t)i * n + c] = 0.0;
    for (int i = c; i >= 0; --i) {
      double rii = r[(int64_t)i * n + i];
      double v;
      if (rii == 0.0) {
        v = 0.0;
      } else if (i == c) {
        v = 1.0 / rii;
      } else {
        double sum = 0.0;
        for (int k = i + 1; k <= c; ++k) sum += r[(int64_t)i * n + k] * x[(int64_t)k * n + c];
        v = -sum / rii;
      }
      x[(int64_t)i * n + c] = v;
    }
  }
}

// Same factorisation, held in shared memory as a packed upper triangle (row a starts at
// a n - a (a - 1) / 2): the per-column updates run at shared-memory latency instead of L2
// latency, and every entry of R sees the same operations in the same order as in
// chol_rinv_kernel.  The inverse is left to inv_upper_kernel (do_inv = 0), which spreads
// its independent columns over many CTAs.
__device__ __forceinline__ int pk(int a, int b, int n) { return a * n - (a * (a - 1)) / 2 + (b - a); }

__global__ void __launch_bounds__(512)
chol_rinv_smem_kernel(const double *G, double *R, double *Rinv, int n, double rel_tol,
                      double shift_rel, int x_in_smem, int do_inv) {
  extern __shared__ double S[];
  double *X = S + (size_t)n * (n + 1) / 2;   // used when x_in_smem
  const int64_t off = (int64_t)blockIdx.x * n * n;
  const double *g = G + off;
  double *r = R + off;
  double *x = Rinv + off;
  __shared__ double s_scale, s_shift, s_piv;
  __shared__ int s_dead;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) {
    double mx = 0.0, tr = 0.0;
    for (int i = 0; i < n; ++i) {
      mx = fmax(mx, g[(int64_t)i * n + i]);
      tr += g[(int64_t)i * n + i];
    }
    s_scale = mx;
    s_shift = shift_rel * tr;
  }
  __syncthreads();
  for (int a = warp; a < n; a += nw)
    for (int b = a + lane; b < n; b += 32)
      S[pk(a, b, n)] = g[(int64_t)a * n + b] + (a == b ? s_shift : 0.0);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double p = S[pk(j, j, n)];
      s_dead = !(p > rel_tol * s_scale && p > 0.0);
      s_piv = s_dead ? 0.0 : sqrt(p);
    }
    __syncthreads();
    const double piv = s_piv;
    if (s_dead) {
      for (int i = j + tid; i < n; i += blockDim.x) S[pk(j, i, n)] = 0.0;
      __syncthreads();
      continue;
    }
    for (int i = j + 1 + tid; i < n; i += blockDim.x) S[pk(j, i, n)] /= piv;
    __syncthreads();
    if (tid == 0) S[pk(j, j, n)] = piv;
    for (int a = j + 1 + warp; a < n; a += nw) {
      const double ra = S[pk(j, a, n)];
      const int rowa = pk(a, 0, n), rowj = pk(j, 0, n);
      for (int b = a + lane; b < n; b += 32) S[rowa + b] -= ra * S[rowj + b];
    }
    __syncthreads();
  }
  for (int a = warp; a < n; a += nw)
    for (int b = lane; b < n; b += 32) r[(int64_t)a * n + b] = b >= a ? S[pk(a, b, n)] : 0.0;
  if (!do_inv) return;
  // inverse of the upper-triangular R, one thread per column; dead rows give zeros
  for (int c = tid; c < n; c += blockDim.x) {
    for (int i = c + 1; i < n; ++i) x[(int64_t)i * n + c] = 0.0;
    for (int i = c; i >= 0; --i) {
      const double rii = S[pk(i, i, n)];
      double v;
      if (rii == 0.0) {
        v = 0.0;
      } else if (i == c) {
        v = 1.0 / rii;
      } else {
        double sum = 0.0;
        const int rowi = pk(i, 0, n);
        if (x_in_smem) {
          for (int k = i + 1; k <= c; ++k) sum += S[rowi + k] * X[pk(k, c, n)];
        } else {
          for (int k = i + 1; k <= c; ++k) sum += S[rowi + k] * x[(int64_t)k * n + c];
        }
        v = -sum / rii;
      }
      if (x_in_smem) X[pk(i, c, n)] = v;
      x[(int64_t)i * n + c] = v;
    }
  }
}

// X = R^-1 of an upper-triangular n x n R (row-major, batch of them), one warp per
// column c of X (back substitution x_c = 1 / R_cc, x_i = -(sum_{k>i} R_ik x_k) / R_ii for
// i = c-1 .. 0, lanes over k and a shuffle sum; a zero pivot gives x_i = 0, a dead row),
// 8 columns per CTA; the triangle of R those columns need is staged in shared memory
// (packed rows, m = last column + 1), the columns themselves per warp.
constexpr int kInvCols = 8;
__global__ void __launch_bounds__(32 * kInvCols)
inv_upper_kernel(const double *__restrict__ R, double *__restrict__ X, int n) {
  extern __shared__ double sm[];
  const int64_t off = (int64_t)blockIdx.y * n * n;
  const double *r = R + off;
  double *x = X + off;
  const int c0 = blockIdx.x * kInvCols, m = min(n, c0 + kInvCols);
  double *Rs = sm;                                    // packed upper triangle of R[0..m)
  double *xs = sm + (size_t)m * (m + 1) / 2;          // kInvCols columns of length m
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int a = warp; a < m; a += kInvCols)
    for (int b = a + lane; b < m; b += 32) Rs[pk(a, b, m)] = r[(int64_t)a * n + b];
  __syncthreads();
  const int c = c0 + warp;
  if (c >= n) return;
  double *xc = xs + (size_t)warp * m;
  if (lane == 0) {
    const double rcc = Rs[pk(c, c, m)];
    xc[c] = rcc == 0.0 ? 0.0 : 1.0 / rcc;
  }
  __syncwarp();
  for (int i = c - 1; i >= 0; --i) {
    const int row = pk(i, 0, m);
    double sum = 0.0;
    for (int k = i + 1 + lane; k <= c; k += 32) sum += Rs[row + k] * xc[k];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) {
      const double rii = Rs[row + i];
      xc[i] = rii == 0.0 ? 0.0 : -sum / rii;
    }
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) x[(int64_t)i * n + c] = i <= c ? xc[i] : 0.0;
}

void chol_rinv(const double *G, double *R, double *Rinv, int n, int batch, double rel_tol,
               double shift_rel, cudaStream_t s) {
  if (n == 0 || batch == 0) return;
  constexpr size_t kMaxSmem = 220 * 1024;
  const size_t tri = (size_t)n * (n + 1) / 2 * sizeof(double);
  if (tri <= kMaxSmem) {
    static const bool attr_done = [] {
      TRG_CUDA(cudaFuncSetAttribute(chol_rinv_smem_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem));
      return true;
    }();
    (void)attr_done;
    // the triangle of the last CTA's columns plus its column buffers (<= tri + 8 n doubles)
    const size_t inv_smem = tri + (size_t)kInvCols * n * sizeof(double);
    if (inv_smem <= kMaxSmem) {
      static const bool inv_attr_done = [] {
        TRG_CUDA(cudaFuncSetAttribute(inv_upper_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kMaxSmem));
        return true;
      }();
      (void)inv_attr_done;
      chol_rinv_smem_kernel<<<batch, 512, tri, s>>>(G, R, Rinv, n, rel_tol, shift_rel, 0, 0);
      TRG_LAUNCH_CHECK();
      inv_upper_kernel<<<dim3((n + kInvCols - 1) / kInvCols, batch), 32 * kInvCols, inv_smem,
                         s>>>(R, Rinv, n);
      TRG_LAUNCH_CHECK();
      return;
    }
    // no room for the column buffers beside the triangle: the inverse in the factorising
    // kernel's own loop (one thread per column)
    const int x_in_smem = 2 * tri <= kMaxSmem;
    chol_rinv_smem_kernel<<<batch, 512, x_in_smem ? 2 * tri : tri, s>>>(G, R, Rinv, n, rel_tol,
                                                                       shift_rel, x_in_smem, 1);
    TRG_LAUNCH_CHECK();
    return;
  }
  chol_rinv_kernel<<<batch, 256, 0, s>>>(G, R, Rinv, n, rel_tol, shift_rel);
  TRG_LAUNCH_CHECK();
}


// ------------------------------------------------------------ one-sided Jacobi
constexpr int kSvdThreads = 1024;
constexpr int kMaxSweeps = 80;
// the working columns live in shared memory when they fit (n m doubles); otherwise in
// the global work buffer
constexpr size_t kSvdSmemMax = 200 * 1024;

__device__ inline double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kSvdThreads)
svd_jacobi_kernel(const double *A, int m, int n, double *U, double *S, double *V,
                  double *work, int *info, int in_smem) {
  extern __shared__ double s_cols[];
  const int64_t b = blockIdx.x;
  const double *a = A + b * (int64_t)m * n;
  double *wb = work + b * ((int64_t)n * m + (int64_t)n * n);
  double *at = in_smem ? s_cols : wb;  // n rows of length m
  double *vt = wb + (int64_t)n * m;    // n rows of length n
  __shared__ int s_rot;
  __shared__ int s_sweeps;
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * m; idx += blockDim.x) {
    int j = (int)(idx / m), r = (int)(idx % m);
    at[idx] = a[(int64_t)r * n + j];
  }
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += blockDim.x)
    vt[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
  if (threadIdx.x == 0) s_sweeps = -1;
  __syncthreads();
  const int nn = n + (n & 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  // rotation threshold sqrt(m) eps (the usual one-sided Jacobi choice): the rounding
  // error of a length-m dot product is about that large, so a smaller one never settles
  const double tol = sqrt((double)m) * 2.220446049250313e-16;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int rnd = 0; rnd < nn - 1; ++rnd) {
      for (int k = warp; k < nn / 2; k += nwarps) {
        int p = (k == 0) ? 0 : ((k - 1 + rnd) % (nn - 1)) + 1;
        int kk = nn - 1 - k;
        int q = ((kk - 1 + rnd) % (nn - 1)) + 1;
        int i = p < q ? p : q, j = p < q ? q : p;
        if (j >= n) continue;  // dummy partner
        double *ai = at + (int64_t)i * m, *aj = at + (int64_t)j * m;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int r = lane; r < m; r += 32) {
          double x = ai[r], y = aj[r];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = wsum(al);
        be = wsum(be);
        ga = wsum(ga);
        if (!(fabs(ga) > tol * sqrt(al * be))) continue;
        double zeta = (be - al) / (2.0 * ga);
        double t;
        if (fabs(zeta) > 1e150)
          t = 0.5 / zeta;
        else
          t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int r = lane; r < m; r += 32) {
          double x = ai[r], y = aj[r];
          ai[r] = c * x - s * y;
          aj[r] = s * x + c * y;
        }
        double *vi = vt + (int64_t)i * n, *vj = vt + (int64_t)j * n;
        for (int r = lane; r < n; r += 32) {
          double x = vi[r], y = vj[r];
          vi[r] = c * x - s * y;
          vj[r] = s * x + c * y;
        }
        if (lane == 0) atomicAdd(&s_rot, 1);
      }
      __syncthreads();
    }
    if (s_rot == 0) {
      if (threadIdx.x == 0) s_sweeps = sweep + 1;
      break;
    }
    __syncthreads();
  }
  __syncthreads();
  // singular values = column norms; sort descending (stable by index)
  __shared__ double s_norm[1024];
  for (int j = warp; j < n; j += nwarps) {
    double v = 0.0;
    for (int r = lane; r < m; r += 32) v += at[(int64_t)j * m + r] * at[(int64_t)j * m + r];
    v = wsum(v);
    if (lane == 0) s_norm[j] = sqrt(v);
  }
  __syncthreads();
  double *u = U + b * (int64_t)m * n;
  double *sv = S + b * (int64_t)n;
  double *v = V + b * (int64_t)n * n;
  for (int j = warp; j < n; j += nwarps) {
    double sj = s_norm[j];
    int rank = 0;
    for (int k = 0; k < n; ++k)
      if (s_norm[k] > sj || (s_norm[k] == sj && k < j)) ++rank;
    double inv = sj > 0.0 ? 1.0 / sj : 0.0;
    for (int r = lane; r < m; r += 32) u[(int64_t)r * n + rank] = at[(int64_t)j * m + r] * inv;
    for (int r = lane; r < n; r += 32) v[(int64_t)r * n + rank] = vt[(int64_t)j * n + r];
    if (lane == 0) sv[rank] = sj;
  }
  if (threadIdx.x == 0 && info) info[b] = s_sweeps;
}

// ------------------------------------------- one-sided Jacobi across the whole GPU
// FP64 runs at a few FMA per clock per SM, so a single CTA needs ~0.1 s for a 144 x 144
// SVD.  This variant gives every column pair of a round its own CTA (one warp) and
// separates rounds with a grid barrier; the launch is cooperative, so all CTAs are
// resident.  Same pair order, reductions and rotations as svd_jacobi_kernel, hence the
// same result.  The barrier waits are bounded (about 2 s); a CTA that gives up raises
// g_lin_err and leaves, and the others then give up at their next barrier.
__device__ int g_lin_err;

__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned *gen, unsigned nblocks,
                                             unsigned &my_gen) {
  __threadfence();
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    const unsigned g = my_gen;
    if (atomicAdd(count, 1u) == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*(volatile unsigned *)gen == g) {
        if (clock64() - t0 > (1ll << 32)) {
          atomicExch(&g_lin_err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  ++my_gen;
  return __syncthreads_and(ok) != 0;
}

// The rotation that zeroes the (i, j) entry of the 2 x 2 Gram [al ga; ga be] (the
// smaller tangent, as in Hestenes' one-sided Jacobi)
__device__ __forceinline__ void jacobi_rotation(double al, double be, double ga, double &c,
                                                double &s) {
  const double zeta = (be - al) / (2.0 * ga);
  double t;
  if (fabs(zeta) > 1e150)
    t = 0.5 / zeta;
  else
    t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  c = 1.0 / sqrt(1.0 + t * t);
  s = c * t;
}
constexpr int kRegCols = 8;   // column elements per lane kept in registers (m, n <= 256)

__global__ void __launch_bounds__(32)
svd_jacobi_coop_kernel(const double *A, int m, int n, double *U, double *S, double *V,
                       double *work, unsigned *sync, int *info) {
  double *at = work, *vt = work + (int64_t)n * m, *nrm = vt + (int64_t)n * n;
  unsigned *count = sync, *gen = sync + 1;
  int *rot = reinterpret_cast<int *>(sync + 2);  // one counter per sweep
  const unsigned nb = gridDim.x;
  unsigned my_gen = 0;
  const int lane = threadIdx.x;
  const int64_t stride = (int64_t)nb * 32;
  for (int64_t idx = blockIdx.x * 32 + lane; idx < (int64_t)n * m; idx += stride) {
    int j = (int)(idx / m), r = (int)(idx % m);
    __stcg(&at[idx], A[(int64_t)r * n + j]);
  }
  for (int64_t idx = blockIdx.x * 32 + lane; idx < (int64_t)n * n; idx += stride)
    __stcg(&vt[idx], (idx / n == idx % n) ? 1.0 : 0.0);
  if (!grid_barrier(count, gen, nb, my_gen)) return;
  const int nn = n + (n & 1);
  const double tol = sqrt((double)m) * 2.220446049250313e-16;
  int sweeps = -1;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    for (int rnd = 0; rnd < nn - 1; ++rnd) {
      for (int k = blockIdx.x; k < nn / 2; k += nb) {
        int p = (k == 0) ? 0 : ((k - 1 + rnd) % (nn - 1)) + 1;
        int kk = nn - 1 - k;
        int q = ((kk - 1 + rnd) % (nn - 1)) + 1;
        int i = p < q ? p : q, j = p < q ? q : p;
        if (j >= n) continue;  // dummy partner
        double *ai = at + (int64_t)i * m, *aj = at + (int64_t)j * m;
        double *vi = vt + (int64_t)i * n, *vj = vt + (int64_t)j * n;
        if (m <= 32 * kRegCols && n <= 32 * kRegCols) {
          // both column pairs of A and V read once, together, and kept in registers for
          // the rotation (one L2 round trip per round); same operations in the same order
          double xa[kRegCols], ya[kRegCols], xv[kRegCols], yv[kRegCols];
#pragma unroll
          for (int u = 0; u < kRegCols; ++u) {
            const int r = lane + 32 * u;
            xa[u] = r < m ? __ldcg(&ai[r]) : 0.0;
            ya[u] = r < m ? __ldcg(&aj[r]) : 0.0;
            xv[u] = r < n ? __ldcg(&vi[r]) : 0.0;
            yv[u] = r < n ? __ldcg(&vj[r]) : 0.0;
          }
          double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
          for (int u = 0; u < kRegCols; ++u) {
            if (lane + 32 * u < m) {
              al += xa[u] * xa[u];
              be += ya[u] * ya[u];
              ga += xa[u] * ya[u];
            }
          }
          al = wsum(al);
          be = wsum(be);
          ga = wsum(ga);
          if (!(fabs(ga) > tol * sqrt(al * be))) continue;
          double c, s;
          jacobi_rotation(al, be, ga, c, s);
#pragma unroll
          for (int u = 0; u < kRegCols; ++u) {
            const int r = lane + 32 * u;
            if (r < m) {
              __stcg(&ai[r], c * xa[u] - s * ya[u]);
              __stcg(&aj[r], s * xa[u] + c * ya[u]);
            }
            if (r < n) {
              __stcg(&vi[r], c * xv[u] - s * yv[u]);
              __stcg(&vj[r], s * xv[u] + c * yv[u]);
            }
          }
        } else {
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int r = lane; r < m; r += 32) {
            double x = __ldcg(&ai[r]), y = __ldcg(&aj[r]);
            al += x * x;
            be += y * y;
            ga += x * y;
          }
          al = wsum(al);
          be = wsum(be);
          ga = wsum(ga);
          if (!(fabs(ga) > tol * sqrt(al * be))) continue;
          double c, s;
          jacobi_rotation(al, be, ga, c, s);
          for (int r = lane; r < m; r += 32) {
            double x = __ldcg(&ai[r]), y = __ldcg(&aj[r]);
            __stcg(&ai[r], c * x - s * y);
            __stcg(&aj[r], s * x + c * y);
          }
          for (int r = lane; r < n; r += 32) {
            double x = __ldcg(&vi[r]), y = __ldcg(&vj[r]);
            __stcg(&vi[r], c * x - s * y);
            __stcg(&vj[r], s * x + c * y);
          }
        }
        if (lane == 0) atomicAdd(&rot[sweep], 1);
      }
      if (!grid_barrier(count, gen, nb, my_gen)) return;
    }
    if (*(volatile int *)&rot[sweep] == 0) {
      sweeps = sweep + 1;
      break;
    }
  }
  for (int j = blockIdx.x; j < n; j += nb) {
    double v = 0.0;
    for (int r = lane; r < m; r += 32) {
      const double x = __ldcg(&at[(int64_t)j * m + r]);
      v += x * x;
    }
    v = wsum(v);
    if (lane == 0) __stcg(&nrm[j], sqrt(v));
  }
  if (!grid_barrier(count, gen, nb, my_gen)) return;
  for (int j = blockIdx.x; j < n; j += nb) {
    const double sj = __ldcg(&nrm[j]);
    int rank = 0;
    for (int k = 0; k < n; ++k) {
      const double sk = __ldcg(&nrm[k]);
      if (sk > sj || (sk == sj && k < j)) ++rank;
    }
    const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
    for (int r = lane; r < m; r += 32) U[(int64_t)r * n + rank] = __ldcg(&at[(int64_t)j * m + r]) * inv;
    for (int r = lane; r < n; r += 32) V[(int64_t)r * n + rank] = __ldcg(&vt[(int64_t)j * n + r]);
    if (lane == 0) S[rank] = sj;
  }
  if (blockIdx.x == 0 && lane == 0 && info) info[0] = sweeps;
}

int linalg_error_flag(bool reset) {
  int v = 0;
  cudaMemcpyFromSymbol(&v, g_lin_err, sizeof(int));
  if (reset) {
    int z = 0;
    cudaMemcpyToSymbol(g_lin_err, &z, sizeof(int));
  }
  return v;
}

size_t svd_jacobi_work(int m, int n, int batch) {
  return (size_t)batch * ((size_t)n * m + (size_t)n * n) + (size_t)n + 8 + (kMaxSweeps + 8) / 2;
}

void svd_jacobi(const double *A, int m, int n, double *U, double *S, double *V, int batch,
                double *work, int *info, cudaStream_t s) {
  if (n == 0 || batch == 0) return;
  if (m < n) throw Error(TRG_ERR_ARG, "svd_jacobi needs m >= n");
  if (n > 1024) throw Error(TRG_ERR_ARG, "svd_jacobi: n > 1024");
  // thread-safe one-time setup (function-local static initialisation)
  static const bool attr_set_done = [&] {
    TRG_CUDA(cudaFuncSetAttribute(svd_jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSvdSmemMax));
    return true;
  }();
  (void)attr_set_done;
  if (batch == 1 && n >= 24) {
    // cooperative form: work = [at | vt | norms | sync words]
    double *nrm_end = work + (size_t)n * m + (size_t)n * n + n;
    unsigned *sync = reinterpret_cast<unsigned *>(nrm_end);
    TRG_CUDA(cudaMemsetAsync(sync, 0, (2 + kMaxSweeps) * sizeof(unsigned), s));
    int dev = 0, nsm = 0;
    TRG_CUDA(cudaGetDevice(&dev));
    TRG_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int pairs = (n + (n & 1)) / 2;
    const unsigned grid = (unsigned)std::min(pairs, nsm);
    void *args[] = {(void *)&A, (void *)&m, (void *)&n, (void *)&U, (void *)&S, (void *)&V,
                    (void *)&work, (void *)&sync, (void *)&info};
    TRG_CUDA(cudaLaunchCooperativeKernel((const void *)svd_jacobi_coop_kernel, dim3(grid),
                                         dim3(32), args, 0, s));
    ++g_kernel_launches;
    return;
  }
  const size_t bytes = (size_t)n * m * sizeof(double);
  const int in_smem = bytes <= kSvdSmemMax;
  svd_jacobi_kernel<<<batch, kSvdThreads, in_smem ? bytes : 0, s>>>(A, m, n, U, S, V, work, info,
                                                                     in_smem);
  TRG_LAUNCH_CHECK();
}

}  // namespace trg
