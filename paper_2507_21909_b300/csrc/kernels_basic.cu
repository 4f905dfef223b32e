// Elementwise, permutation, reduction and sketch kernels of libtrg (FP64).
#include <algorithm>
#include <cstdlib>
#include <utility>

#include "trg_internal.h"

namespace trg {

std::atomic<int64_t> g_kernel_launches{0};

// ------------------------------------------------------------------ switches
static std::vector<std::pair<std::string, std::string>> parse_list(const char *var) {
  std::vector<std::pair<std::string, std::string>> out;
  const char *e = getenv(var);
  if (!e) return out;
  std::string s(e);
  size_t i = 0;
  while (i <= s.size()) {
    size_t j = s.find(',', i);
    if (j == std::string::npos) j = s.size();
    std::string item = s.substr(i, j - i);
    if (!item.empty()) {
      size_t eq = item.find('=');
      out.emplace_back(item.substr(0, eq), eq == std::string::npos ? "1" : item.substr(eq + 1));
    }
    i = j + 1;
  }
  return out;
}

std::string study_opt(const char *key) {
  for (auto &kv : parse_list("TRG_STUDY"))   // read at every call: tests set it per case
    if (kv.first == key) return kv.second;
  return std::string();
}

bool debug_opt(const char *key) {
  static const auto opts = parse_list("TRG_DEBUG");
  for (auto &kv : opts)
    if (kv.first == key) return true;
  return false;
}

// ------------------------------------------------------------------ permutation
constexpr int kMaxDims = 10;
struct PermArgs {
  int nd;
  int64_t out_dims[kMaxDims];
  int64_t in_stride_of_out[kMaxDims];  // stride in `in` of each output axis
};

__global__ void permute_kernel(const double *__restrict__ in, double *__restrict__ out,
                               int64_t total, PermArgs a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = i, off = 0;
    for (int d = a.nd - 1; d >= 0; --d) {
      int64_t c = rem % a.out_dims[d];
      rem /= a.out_dims[d];
      off += c * a.in_stride_of_out[d];
    }
    out[i] = in[off];
  }
}

static int grid_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 148 * 64) b = 148 * 64;
  if (b < 1) b = 1;
  return (int)b;
}

// Offsets of a mixed-radix index over `nb` axes (innermost last) in two layouts.
struct BatchMap {
  int nb;
  int64_t dims[kMaxDims];
  int64_t s_in[kMaxDims], s_out[kMaxDims];
};
__device__ __forceinline__ void batch_offsets(const BatchMap &m, int64_t idx, int64_t &oi,
                                              int64_t &oo) {
  oi = 0;
  oo = 0;
  for (int d = m.nb - 1; d >= 0; --d) {
    const int64_t c = idx % m.dims[d];
    idx /= m.dims[d];
    oi += c * m.s_in[d];
    oo += c * m.s_out[d];
  }
}

// The innermost axis is kept: rows of L contiguous elements are copied, one block per
// `rpb` rows; the row offsets are decoded once per row (one thread each), then every warp
// copies whole rows with its lanes along the row (no index division per element).
__global__ void permute_rows_kernel(const double *__restrict__ in, double *__restrict__ out,
                                    int64_t rows, int64_t L, int rpb, BatchMap m) {
  __shared__ int64_t s_off[256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int64_t r0 = (int64_t)blockIdx.x * rpb; r0 < rows; r0 += (int64_t)gridDim.x * rpb) {
    __syncthreads();
    if (threadIdx.x < rpb && r0 + threadIdx.x < rows) {
      int64_t oi, oo;
      batch_offsets(m, r0 + threadIdx.x, oi, oo);
      s_off[threadIdx.x] = oi;
    }
    __syncthreads();
    const int nrow = (int)min((int64_t)rpb, rows - r0);
    if (L >= 32) {
      for (int r = warp; r < nrow; r += nwarp) {
        const double *src = in + s_off[r];
        double *dst = out + (r0 + r) * L;
        int64_t j = lane;
        for (; j + 96 < L; j += 128) {   // four loads in flight per lane
          const double v0 = src[j], v1 = src[j + 32], v2 = src[j + 64], v3 = src[j + 96];
          dst[j] = v0;
          dst[j + 32] = v1;
          dst[j + 64] = v2;
          dst[j + 96] = v3;
        }
        for (; j < L; j += 32) dst[j] = src[j];
      }
    } else {   // short rows: threads over the block's rows x L elements (32-bit indices)
      const int n = nrow * (int)L, l = (int)L;
      double *dst = out + r0 * L;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int r = i / l, j = i - r * l;
        dst[i] = in[s_off[r] + j];
      }
    }
  }
}

// 64 x 64 tiles through shared memory: reads run along the input's innermost axis (a),
// writes along the output's innermost axis (b), 16 loads in flight per thread; the other
// axes are a batch whose offsets one thread decodes per tile.
constexpr int kPT = 64;
__global__ void __launch_bounds__(256)
permute_tile_kernel(const double *__restrict__ in, double *__restrict__ out, int64_t na,
                    int64_t nbb, int64_t sa_out, int64_t sb_in, int64_t ntiles, BatchMap m) {
  __shared__ double tile[kPT][kPT + 1];
  __shared__ int64_t s_io[4];   // input offset, output offset, a0, b0 of the tile
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;   // 64 x 4
  const int64_t ta_n = (na + kPT - 1) / kPT, tb_n = (nbb + kPT - 1) / kPT;
  const int64_t per = ta_n * tb_n;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const int64_t bi = t / per, rem = t - bi * per;
      int64_t oi, oo;
      batch_offsets(m, bi, oi, oo);
      s_io[0] = oi;
      s_io[1] = oo;
      s_io[2] = (rem % ta_n) * kPT;
      s_io[3] = (rem / ta_n) * kPT;
    }
    __syncthreads();
    const int64_t oi = s_io[0], oo = s_io[1], a0 = s_io[2], b0 = s_io[3];
    const int64_t a = a0 + tx;
    double v[kPT / 4];
#pragma unroll
    for (int u = 0; u < kPT / 4; ++u) {
      const int64_t b = b0 + ty + 4 * u;
      v[u] = (a < na && b < nbb) ? in[oi + b * sb_in + a] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kPT / 4; ++u) tile[ty + 4 * u][tx] = v[u];
    __syncthreads();
    const int64_t bo = b0 + tx;
#pragma unroll
    for (int u = 0; u < kPT / 4; ++u) {
      const int64_t ao = a0 + ty + 4 * u;
      if (ao < na && bo < nbb) out[oo + ao * sa_out + bo] = tile[tx][ty + 4 * u];
    }
  }
}

void permute(const double *in, double *out, const std::vector<int64_t> &dims_in,
             const std::vector<int> &perm, cudaStream_t s) {
  const int nd0 = (int)dims_in.size();
  if (nd0 > kMaxDims) throw Error(TRG_ERR_ARG, "permute: too many dims");
  int64_t total = 1;
  for (int d = 0; d < nd0; ++d) total *= dims_in[d];
  if (total == 0) return;
  // merge output axes that are also adjacent (and in order) in the input; drop 1-axes
  std::vector<int64_t> st(nd0, 1);
  for (int d = nd0 - 2; d >= 0; --d) st[d] = st[d + 1] * dims_in[d + 1];
  std::vector<int64_t> od, os;   // merged output dims and their input strides
  std::vector<int> first;        // input axis of each merged group's outermost member
  for (int j = 0; j < nd0; ++j) {
    const int ax = perm[j];
    if (dims_in[ax] == 1) continue;
    if (!od.empty() && first.back() >= 0 && os.back() == st[ax] * dims_in[ax]) {
      od.back() *= dims_in[ax];
      os.back() = st[ax];
    } else {
      od.push_back(dims_in[ax]);
      os.push_back(st[ax]);
      first.push_back(ax);
    }
  }
  const int nd = (int)od.size();
  if (nd <= 1 || (os.back() == 1 && nd == 1)) {
    TRG_CUDA(cudaMemcpyAsync(out, in, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return;
  }
  bool identity = true;
  for (int j = 0; j < nd; ++j) {
    int64_t want = 1;
    for (int k = j + 1; k < nd; ++k) want *= od[k];
    if (os[j] != want) identity = false;
  }
  if (identity) {
    TRG_CUDA(cudaMemcpyAsync(out, in, total * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return;
  }
  std::vector<int64_t> ostr(nd, 1);  // output strides of the merged axes
  for (int j = nd - 2; j >= 0; --j) ostr[j] = ostr[j + 1] * od[j + 1];
  if (os[nd - 1] == 1) {
    // innermost axis kept
    const int64_t L = od[nd - 1], rows = total / L;
    BatchMap m;
    m.nb = nd - 1;
    for (int j = 0; j < nd - 1; ++j) {
      m.dims[j] = od[j];
      m.s_in[j] = os[j];
      m.s_out[j] = ostr[j] / L;
    }
    const int rpb = (int)std::max<int64_t>(8, std::min<int64_t>(256, 4096 / L));
    const int64_t blocks = std::min<int64_t>((rows + rpb - 1) / rpb, 148 * 32);
    permute_rows_kernel<<<(int)blocks, 256, 0, s>>>(in, out, rows, L, rpb, m);
    TRG_LAUNCH_CHECK();
    return;
  }
  // the input's innermost axis sits at output position q (stride 1 in the input)
  int q = -1;
  for (int j = 0; j < nd; ++j)
    if (os[j] == 1) q = j;
  const int64_t na = q >= 0 ? od[q] : 0, nbb = od[nd - 1];
  if (q < 0 || na < 8 || nbb < 8) {
    PermArgs a;
    a.nd = nd;
    for (int j = 0; j < nd; ++j) {
      a.out_dims[j] = od[j];
      a.in_stride_of_out[j] = os[j];
    }
    permute_kernel<<<grid_for(total), 256, 0, s>>>(in, out, total, a);
    TRG_LAUNCH_CHECK();
    return;
  }
  BatchMap m;
  m.nb = 0;
  for (int j = 0; j < nd; ++j) {
    if (j == q || j == nd - 1) continue;
    m.dims[m.nb] = od[j];
    m.s_in[m.nb] = os[j];
    m.s_out[m.nb] = ostr[j];
    ++m.nb;
  }
  const int64_t nbatch = total / (na * nbb);
  const int64_t ntiles = nbatch * ((na + kPT - 1) / kPT) * ((nbb + kPT - 1) / kPT);
  const int64_t blocks = std::min<int64_t>(ntiles, 148 * 64);
  permute_tile_kernel<<<(int)blocks, 256, 0, s>>>(in, out, na, nbb, ostr[q], os[nd - 1],
                                                  ntiles, m);
  TRG_LAUNCH_CHECK();
}

// ------------------------------------------------------- counter-based sketches
// SplitMix64 output function (Steele, Lea, Flood 2014) applied to key + n * gamma.
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

uint64_t sketch_key(uint64_t seed, int step, int tag) {
  return mix64(seed + kGolden * (uint64_t)(64 * (int64_t)step + tag + 1));
}

__global__ void gaussian_kernel(double *out, int64_t total, uint64_t key) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t n = (uint64_t)i;
    uint64_t x = mix64(key + kGolden * (2 * n + 1));
    uint64_t y = mix64(key + kGolden * (2 * n + 2));
    double u1 = ((double)(x >> 11) + 1.0) * 0x1.0p-53;  // (0, 1]
    double u2 = (double)(y >> 11) * 0x1.0p-53;          // [0, 1)
    out[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  }
}

void fill_gaussian(double *out, int64_t rows, int64_t cols, uint64_t key, cudaStream_t s) {
  int64_t total = rows * cols;
  if (total == 0) return;
  gaussian_kernel<<<grid_for(total), 256, 0, s>>>(out, total, key);
  TRG_LAUNCH_CHECK();
}

__global__ void khatri_rao_kernel(const double *g2, const double *g1, double *out,
                                  int64_t nj, int64_t nb, int64_t w) {
  int64_t total = nj * nb * w;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t m = i % w, jb = i / w, b = jb % nb, j = jb / nb;
    out[i] = g2[j * w + m] * g1[b * w + m];
  }
}

void khatri_rao(const double *g2, const double *g1, double *out, int64_t nj, int64_t nb,
                int64_t w, cudaStream_t s) {
  int64_t total = nj * nb * w;
  if (total == 0) return;
  khatri_rao_kernel<<<grid_for(total), 256, 0, s>>>(g2, g1, out, nj, nb, w);
  TRG_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ scaling
__device__ inline double scale_fn(double v, int mode, double vmax, double tol) {
  switch (mode) {
    case 0: return v;
    case 1: return (v > tol * vmax && v > 0.0) ? 1.0 / v : 0.0;
    case 2: return (v > tol * vmax && v > 0.0) ? 1.0 / sqrt(v) : 0.0;
    default: return v > 0.0 ? sqrt(v) : 0.0;
  }
}

__global__ void scale_axis_kernel(double *x, int64_t total, int64_t inner, int64_t n,
                                  const double *v, int mode, const double *vmax,
                                  double tol) {
  double mx = vmax ? *vmax : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = (i / inner) % n;
    x[i] *= scale_fn(v[a], mode, mx, tol);
  }
}

void scale_axis(double *x, int64_t total, int64_t inner, int64_t n, const double *v,
                int mode, const double *vmax, double tol, cudaStream_t s) {
  if (total == 0) return;
  scale_axis_kernel<<<grid_for(total), 256, 0, s>>>(x, total, inner, n, v, mode, vmax, tol);
  TRG_LAUNCH_CHECK();
}

__global__ void kill_dead_kernel(const double *v, int64_t n, double tol, double *m1,
                                 int64_t rows1, double *m2, int64_t rows2) {
  double top = v[0];
  int64_t tot1 = rows1 * n, tot2 = rows2 * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot1 + tot2;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < tot1) {
      int64_t c = i % n;
      if (!(v[c] > tol * top && v[c] > 0.0)) m1[i] = 0.0;
    } else {
      int64_t j = i - tot1, c = j % n;
      if (!(v[c] > tol * top && v[c] > 0.0)) m2[j] = 0.0;
    }
  }
}
__global__ void kill_dead_v_kernel(double *v, int64_t n, double tol) {
  double top = v[0];
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    if (!(v[i] > tol * top && v[i] > 0.0)) v[i] = 0.0;
}

void kill_dead(double *v, int64_t n, double tol, double *m1, int64_t rows1, double *m2,
               int64_t rows2, cudaStream_t s) {
  if (n == 0) return;
  if (!m1) rows1 = 0;
  if (!m2) rows2 = 0;
  if (rows1 * n + rows2 * n > 0) {
    kill_dead_kernel<<<grid_for(rows1 * n + rows2 * n), 256, 0, s>>>(v, n, tol, m1, rows1, m2,
                                                                      rows2);
    TRG_LAUNCH_CHECK();
  }
  kill_dead_v_kernel<<<1, 256, 0, s>>>(v, n, tol);
  TRG_LAUNCH_CHECK();
}

// --------------------------------------------------------------- reductions
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

constexpr int kDotBlocks = 256;
__global__ void dot_partial(const double *a, const double *b, int64_t n, double *part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}
__global__ void dot_final(const double *part, int np, double *out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) v += part[i];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    w = warp_sum(w);
    if (threadIdx.x == 0) *out = w;
  }
}

void dot(const double *a, const double *b, int64_t n, double *out, double *scratch,
         cudaStream_t s) {
  dot_partial<<<kDotBlocks, 256, 0, s>>>(a, b, n, scratch);
  TRG_LAUNCH_CHECK();
  dot_final<<<1, 256, 0, s>>>(scratch, kDotBlocks, out);
  TRG_LAUNCH_CHECK();
}

__global__ void col_max_abs_kernel(const double *v, int64_t n, double *out) {
  __shared__ double sh[32];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(v[i]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    w = warp_max(w);
    if (threadIdx.x == 0) *out = w;
  }
}
void col_max_abs(const double *v, int64_t n, double *out, cudaStream_t s) {
  col_max_abs_kernel<<<1, 256, 0, s>>>(v, n, out);
  TRG_LAUNCH_CHECK();
}

// one block per column: max |a|, then the first row within 1e-6 of it decides the sign
__global__ void sign_gauge_kernel(double *m1, int64_t rows1, double *m2, int64_t rows2,
                                  int64_t cols) {
  __shared__ double shm[32];
  __shared__ long long shi[32];
  __shared__ double s_sign;
  int64_t c = blockIdx.x;
  double mx = 0.0;
  for (int64_t r = threadIdx.x; r < rows1; r += blockDim.x) mx = fmax(mx, fabs(m1[r * cols + c]));
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? shm[threadIdx.x] : 0.0;
    w = warp_max(w);
    if (threadIdx.x == 0) shm[0] = w;
  }
  __syncthreads();
  mx = shm[0];
  __syncthreads();
  long long first = (long long)rows1;
  if (mx > 0.0) {
    double thr = (1.0 - 1e-6) * mx;
    for (int64_t r = threadIdx.x; r < rows1; r += blockDim.x)
      if (fabs(m1[r * cols + c]) >= thr) { first = r; break; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    long long other = __shfl_xor_sync(0xffffffffu, first, o);
    first = other < first ? other : first;
  }
  if ((threadIdx.x & 31) == 0) shi[threadIdx.x >> 5] = first;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long f = (long long)rows1;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) f = shi[i] < f ? shi[i] : f;
    s_sign = (f < (long long)rows1 && m1[f * cols + c] < 0.0) ? -1.0 : 1.0;
  }
  __syncthreads();
  if (s_sign < 0.0) {
    for (int64_t r = threadIdx.x; r < rows1; r += blockDim.x) m1[r * cols + c] = -m1[r * cols + c];
    if (m2)
      for (int64_t r = threadIdx.x; r < rows2; r += blockDim.x) m2[r * cols + c] = -m2[r * cols + c];
  }
}

// The same rule for tall row-major matrices in three coalesced passes over all SMs.
// Threads per block are a multiple of `cols`, so every thread stays on one column:
// (1) per-column max |a| (non-negative doubles order like their bit patterns, so
// atomicMax on the bits), (2) per column the first row within 1e-6 of it (atomicMin),
// (3) the sign of that entry flips the column of m1 and of m2.
__global__ void col_absmax_kernel(const double *__restrict__ m, int64_t n, int64_t cols,
                                  unsigned long long *mx) {
  extern __shared__ unsigned long long red[];
  double v = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += stride)
    v = fmax(v, fabs(m[e]));
  red[threadIdx.x] = (unsigned long long)__double_as_longlong(v);
  __syncthreads();
  if (threadIdx.x < cols) {
    unsigned long long b = 0;
    for (int t = threadIdx.x; t < (int)blockDim.x; t += (int)cols) b = max(b, red[t]);
    atomicMax(&mx[threadIdx.x], b);
  }
}

__global__ void col_first_kernel(const double *__restrict__ m, int64_t n, int64_t cols,
                                 const unsigned long long *mx, unsigned long long *first) {
  extern __shared__ unsigned long long red[];
  const int c = (int)(threadIdx.x % cols);
  const double thr = (1.0 - 1e-6) * __longlong_as_double((long long)mx[c]);
  unsigned long long f = ~0ull;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (thr > 0.0)
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += stride)
      if (fabs(m[e]) >= thr) { f = (unsigned long long)(e / cols); break; }
  red[threadIdx.x] = f;
  __syncthreads();
  if (threadIdx.x < cols) {
    unsigned long long b = ~0ull;
    for (int t = threadIdx.x; t < (int)blockDim.x; t += (int)cols) b = min(b, red[t]);
    atomicMin(&first[threadIdx.x], b);
  }
}

__global__ void col_sign_kernel(const double *m1, int64_t cols, const unsigned long long *first,
                                double *sign) {
  const int c = threadIdx.x;
  if (c >= cols) return;
  const unsigned long long f = first[c];
  sign[c] = (f != ~0ull && m1[(int64_t)f * cols + c] < 0.0) ? -1.0 : 1.0;
}

__global__ void col_scale_kernel(double *m, int64_t n, int64_t cols, const double *sign) {
  const int c = (int)(threadIdx.x % cols);
  const double sg = sign[c];
  if (sg > 0.0) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += stride)
    m[e] = -m[e];
}

void sign_gauge(double *m1, int64_t rows1, double *m2, int64_t rows2, int64_t cols,
                cudaStream_t s) {
  if (cols == 0) return;
  if (cols > 256 || rows1 * cols < (int64_t(1) << 20)) {
    sign_gauge_kernel<<<(unsigned)cols, 256, 0, s>>>(m1, rows1, m2, rows2, cols);
    TRG_LAUNCH_CHECK();
    return;
  }
  // workspace: cols max bits, cols first rows, cols signs (4 KB each at most)
  static thread_local unsigned long long *ws = nullptr;
  if (!ws) TRG_CUDA(cudaMalloc(&ws, 3 * 256 * sizeof(unsigned long long)));
  unsigned long long *mx = ws, *first = ws + 256;
  double *sign = reinterpret_cast<double *>(ws + 512);
  TRG_CUDA(cudaMemsetAsync(mx, 0, 256 * sizeof(unsigned long long), s));
  TRG_CUDA(cudaMemsetAsync(first, 0xFF, 256 * sizeof(unsigned long long), s));
  const int threads = (int)(cols * std::max<int64_t>(1, 256 / cols));
  const size_t shm = (size_t)threads * sizeof(unsigned long long);
  const int blocks = 148 * 8;
  col_absmax_kernel<<<blocks, threads, shm, s>>>(m1, rows1 * cols, cols, mx);
  TRG_LAUNCH_CHECK();
  col_first_kernel<<<blocks, threads, shm, s>>>(m1, rows1 * cols, cols, mx, first);
  TRG_LAUNCH_CHECK();
  col_sign_kernel<<<1, 256, 0, s>>>(m1, cols, first, sign);
  TRG_LAUNCH_CHECK();
  col_scale_kernel<<<blocks, threads, 0, s>>>(m1, rows1 * cols, cols, sign);
  TRG_LAUNCH_CHECK();
  if (m2) {
    col_scale_kernel<<<blocks, threads, 0, s>>>(m2, rows2 * cols, cols, sign);
    TRG_LAUNCH_CHECK();
  }
}

__global__ void fill_identity_kernel(double *out, int64_t n, int64_t cols) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * cols;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (i / cols == i % cols) ? 1.0 : 0.0;
}
void fill_identity(double *out, int64_t n, int64_t cols, cudaStream_t s) {
  if (n * cols == 0) return;
  fill_identity_kernel<<<grid_for(n * cols), 256, 0, s>>>(out, n, cols);
  TRG_LAUNCH_CHECK();
}

// mode 0: x *= s; mode 1: x /= s (s > 0, else untouched)
__global__ void scale_by_scalar_kernel(double *x, int64_t n, const double *scalar, int mode) {
  double sc = *scalar;
  double f = mode == 0 ? sc : (sc > 0.0 ? 1.0 / sc : 1.0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= f;
}
void scale_by_scalar(double *x, int64_t n, const double *scalar, int mode, cudaStream_t s) {
  if (n == 0) return;
  scale_by_scalar_kernel<<<grid_for(n), 256, 0, s>>>(x, n, scalar, mode);
  TRG_LAUNCH_CHECK();
}

__global__ void axpby_kernel(double *y, const double *x, double a, double b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
void axpby(double *y, const double *x, double a, double b, int64_t n, cudaStream_t s) {
  if (n == 0) return;
  axpby_kernel<<<grid_for(n), 256, 0, s>>>(y, x, a, b, n);
  TRG_LAUNCH_CHECK();
}

__global__ void norm_update_kernel(const double *tr, double *c_out, double *logsum,
                                   double weight, int *flag) {
  double t = *tr;
  double c = sqrt(t > 0.0 ? t : 0.0);
  if (!(c > 0.0) || !isfinite(c)) {
    *flag = TRG_ERR_NONFINITE;
    c = 1.0;
  }
  *c_out = c;
  *logsum += log(c) * weight;
}
void norm_update(const double *tr, double *c_out, double *logsum, double weight, int *flag,
                 cudaStream_t s) {
  norm_update_kernel<<<1, 1, 0, s>>>(tr, c_out, logsum, weight, flag);
  TRG_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ arena
void *Arena::alloc(size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  for (size_t i = top_; i < chunks_.size(); ++i) {
    Chunk &c = chunks_[i];
    if (c.cap - c.used >= bytes) {
      void *p = c.p + c.used;
      c.used += bytes;
      top_ = i;
      cur_ += bytes;
      if (cur_ > high_) high_ = cur_;
      return p;
    }
  }
  // the empty chunks above the top are all too small for this request: give their
  // memory back before asking for a bigger chunk (cudaFree waits for the device, so no
  // kernel still reads them); otherwise a step that grows in size piles up idle chunks
  if (chunks_.size() > top_ + 1 && !chunks_.empty()) {
    for (size_t i = top_ + 1; i < chunks_.size(); ++i) cudaFree(chunks_[i].p);
    chunks_.resize(top_ + 1);
  }
  // new chunks are sized to the request (at least 1 GiB); reset() merges them into one
  size_t cap = bytes;
  if (cap < (size_t(1) << 30)) cap = size_t(1) << 30;
  char *p = nullptr;
  if (cudaMalloc(&p, cap) != cudaSuccess) {
    cudaGetLastError();
    cap = bytes;
    if (cudaMalloc(&p, cap) != cudaSuccess) {
      cudaGetLastError();
      throw Error(TRG_ERR_OOM, "device allocation of " + std::to_string(bytes) +
                                   " bytes failed (arena in use " + std::to_string(cur_ >> 20) +
                                   " MiB, reserved " + std::to_string(reserved() >> 20) + " MiB)");
    }
  }
  chunks_.push_back({p, cap, bytes});
  top_ = chunks_.size() - 1;
  cur_ += bytes;
  if (cur_ > high_) high_ = cur_;
  return p;
}

void Arena::reset() {
  // merge into one chunk of the high-water size so that the next step needs one chunk
  if (chunks_.size() > 1) {
    for (auto &c : chunks_) cudaFree(c.p);
    chunks_.clear();
    char *p = nullptr;
    if (cudaMalloc(&p, high_) == cudaSuccess)
      chunks_.push_back({p, high_, 0});
    else
      cudaGetLastError();
  }
  for (auto &c : chunks_) c.used = 0;
  top_ = 0;
  cur_ = 0;
}

void Arena::release(const Mark &m) {
  for (size_t i = m.top + 1; i < chunks_.size(); ++i) chunks_[i].used = 0;
  if (m.top < chunks_.size()) chunks_[m.top].used = m.used;
  top_ = m.top;
  cur_ = m.cur;
}

void Arena::release() {
  for (auto &c : chunks_) cudaFree(c.p);
  chunks_.clear();
  top_ = 0;
  cur_ = 0;
}

}  // namespace trg
