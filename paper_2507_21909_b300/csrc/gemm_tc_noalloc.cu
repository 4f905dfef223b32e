// trg_gemm_noalloc: the split-BF16 tensor-core GEMM for callers that must not allocate.
//
// Some callers cannot call cudaMalloc at the point where they need a product: host
// frameworks that own all device memory through their own pool and forbid foreign
// allocations (a second allocator would fragment or overcommit the pool), real-time
// loops that must not risk an allocation stall or an out-of-memory failure after
// start-up, and code that must not let cudaMalloc synchronise the device in the middle
// of its own asynchronous work.  This entry point serves them: inputs and outputs are
// the caller's device buffers, and the only scratch (BF16 slice buffers and split-K
// partial tiles) is a fixed file-scope __device__ array of kScratchBytes.  No
// cudaMalloc, cudaFree or allocating library routine is called.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "gemm_tc.h"
#include "trg_internal.h"

namespace trg {

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB, held by every device that loads the library
constexpr int kMaxDevices = 64;
constexpr int64_t kBM = 128, kBK = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// device address of g_noalloc_scratch, looked up once per device (host code cannot use
// the symbol's host-side name as a device pointer)
void *g_scratch_ptr[kMaxDevices] = {};

void *scratch_for_current_device() {
  int dev = -1;
  TRG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw Error(TRG_ERR_ARG, "device index out of range");
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      throw Error(TRG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

// bump allocator over the fixed array; never grows
struct FixedScratch : TcScratch {
  unsigned char *base;
  size_t used = 0;
  explicit FixedScratch(void *b) : base(static_cast<unsigned char *>(b)) {}
  void *alloc(size_t bytes) override {
    bytes = (bytes + 255) & ~size_t(255);
    if (used + bytes > kScratchBytes) throw Error(TRG_ERR_ARG, "scratch exhausted");
    void *p = base + used;
    used += bytes;
    return p;
  }
};

// the scratch gemm_tc will request for this problem (same tiling rules as gemm_tc)
size_t scratch_needed(int64_t M, int64_t N, int64_t K, int ns) {
  auto r256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  const int64_t Kp = std::max<int64_t>(kBK, (K + kBK - 1) / kBK * kBK);
  size_t need = r256((size_t)ns * M * Kp * 2) + r256((size_t)ns * N * Kp * 2);
  const int64_t BN = N <= 128 ? 128 : 256;
  const int64_t gx = (N + BN - 1) / BN, gy = (M + kBM - 1) / kBM;
  const int nkb = (int)(Kp / kBK);
  int ksplit = 1;
  const int64_t tiles = gx * gy;
  if (tiles < 148 && nkb >= 8) {
    ksplit = (int)std::min<int64_t>(std::min<int64_t>((2 * 148 + tiles - 1) / tiles, nkb / 4), 65535);
    ksplit = std::max(ksplit, 1);
  }
  const int per = (nkb + ksplit - 1) / ksplit;
  ksplit = (nkb + per - 1) / per;
  if (ksplit > 1) need += r256((size_t)ksplit * M * N * sizeof(double));
  return need;
}

}  // namespace
}  // namespace trg

using namespace trg;

extern "C" trg_status trg_gemm_noalloc(int precision, int ta, int tb, long long M, long long N,
                                       long long K, double alpha, const double *A, long long lda,
                                       const double *B, long long ldb, double beta, double *C,
                                       long long ldc, void *stream) {
  try {
    if (precision < TRG_PREC_BF16X3 || precision > TRG_PREC_BF16X10)
      throw Error(TRG_ERR_ARG, "trg_gemm_noalloc: precision must be a split-BF16 mode (1..3)");
    if (!A || !B || !C || M < 1 || N < 1 || K < 1)
      throw Error(TRG_ERR_ARG, "trg_gemm_noalloc: NULL buffer or empty size");
    // row-major op(A) is M x K and op(B) K x N: a leading dimension shorter than the
    // stored row would make the kernels read or write outside the caller's buffers
    if (lda < (ta ? M : K) || ldb < (tb ? K : N) || ldc < N)
      throw Error(TRG_ERR_ARG, "trg_gemm_noalloc: leading dimension shorter than a row "
                               "(need lda >= " + std::to_string(ta ? M : K) + ", ldb >= " +
                               std::to_string(tb ? K : N) + ", ldc >= " + std::to_string(N) +
                               ")");
    const int ns = precision == TRG_PREC_BF16X3 ? 2 : precision == TRG_PREC_BF16X6 ? 3 : 4;
    const size_t need = scratch_needed(M, N, K, ns);
    if (need > kScratchBytes)
      throw Error(TRG_ERR_ARG, "trg_gemm_noalloc: problem needs " + std::to_string(need >> 20) +
                                   " MiB of scratch, more than the fixed " +
                                   std::to_string(kScratchBytes >> 20) + " MiB");
    FixedScratch scr(scratch_for_current_device());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gemm_tc(ta != 0, tb != 0, M, N, K, alpha, A, lda, 0, B, ldb, 0, beta, C, ldc, 0, 1, ns, scr,
            st);
    // wait for the product and report a bounded wait inside the kernel that gave up (the
    // flag is cleared here, so it cannot be blamed on a later call); a stream that is
    // capturing work is not waited on
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
      cudaGetLastError();
      cap = cudaStreamCaptureStatusActive;
    }
    if (cap == cudaStreamCaptureStatusNone) {
      TRG_CUDA(cudaStreamSynchronize(st));
      if (tc_error_flag(true))
        throw Error(TRG_ERR_TIMEOUT, "trg_gemm_noalloc: a tensor-core pipeline wait timed out; "
                                     "C is not valid");
    }
    set_last_error("ok");
    return TRG_OK;
  } catch (const Error &e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception &e) {
    set_last_error(e.what());
    return TRG_ERR_CUDA;
  }
}
