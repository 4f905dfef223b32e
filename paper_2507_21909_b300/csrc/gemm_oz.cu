// Exact-accumulation split GEMM on the tcgen05 tensor cores (Ozaki-style digits).
//
// C (FP64) = alpha * op(A) op(B) + beta * C with ~7*ns bits of every row of op(A) and
// column of op(B).  Each row r of op(A) gets a common exponent e_r (max |a| < 2^e_r) and
// a' = a 2^-e_r in (-1, 1) is cut into integer digits d_s (|d_0| <= 128, |d_s| <= 64):
//     a' = sum_s d_s 2^(-7(s+1)) + O(2^(-7 ns - 1)).
// Slices are stored pre-scaled as BF16 values  ^a_s = d_s 2^(-7(s-1))  (exact: 8-bit
// integers times powers of two), so that  a' b' = 2^-28 sum_{i,j} ^a_i ^b_j  and the
// digit products fall into three levels of tensor-memory accumulators:
//     L0 = sum ^a_0 ^b_0            (integers x 2^14,  |chunk sum| <= 2^37)
//     L1 = sum ^a_0 ^b_1 + ^a_1 ^b_0 (integers x 2^7)
//     H  = sum over i + j in [2, ns-1] of ^a_i ^b_j   (carries 2^-14 of the result)
// Over a chunk of 512 K the FP32 sums L0 / L1 are exact integers (|L0 2^-14| and
// |L1 2^-7| <= 2^23 < 2^24); every chunk they and that chunk's H are drained into one int64
// fixed-point accumulator per output with 12 fractional bits (integer units on the
// ALU: B300 issues few FP64 adds), so only H carries the FP32 rounding of one chunk.
// |acc| <= K 2^41, so K per split stays below 2^21.  H is double-buffered in tensor
// memory (two accumulators, alternating chunks) so the next chunk's products do not
// wait for the drain.  The epilogue forms C = alpha 2^(e_r + e_c - 40) acc + beta C.
//
// Persistent kernel, one CTA (18 warps) per SM walking the output tiles: warp 0 TMA
// producer, warp 1 MMA issuer (M = 128, N = 128, K = 16), warps 2..17 drain TMEM (four
// warps per 32-lane quadrant, 32 columns each) and write the outputs from their
// registers while the next tile's products already run.  A pipeline stage holds one
// 16-wide K block of every digit slice of A and of B, so each slice tile is loaded once
// and serves all pairs (i, j) that use it.  The digit planes are stored pre-tiled in the
// tensor cores' unswizzled K-major layout (8-row x 16-byte core matrices, the two K halves
// of a 16-wide block 128 bytes apart, the digit slices of one 8-row group side by side):
// one TMA box per operand and stage then moves 256-byte contiguous runs, where a
// row-major plane would need one 32-byte request per row and slice, which saturates the
// SM-to-L2 request path before the tensor pipe.  At the first stage of a chunk the
// lower-level pairs are issued before waiting for the drain of the previous chunk's exact
// levels, and the drain warps read those first and signal them separately from the H
// buffer (which is reused two chunks later), so the issuer waits only for the exact
// levels.  Every wait is bounded (2^31 cycles): on a timeout the device flag is set, the
// roles stop, the CTA waits (bounded) for its loads and products in flight and frees its
// tensor memory; the output is then undefined and the host reports TRG_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "gemm_oz.h"
#include "trg_internal.h"

namespace trg {
namespace oz {

constexpr int BM = 128;
constexpr int BK = 64;                      // K padding granule of the digit planes
constexpr int KS = 16;                      // K per pipeline stage (= one MMA, 32-byte rows)
constexpr int CHUNK_K = 512;                // exact chunk of the exact levels
constexpr int CHUNK_KS = CHUNK_K / KS;      // stages per chunk
constexpr uint32_t CHUNK_BYTES = 256;           // one 8-row group x 16 K of one slice
constexpr size_t kSmemOptin = 232448;           // dynamic shared memory per block (opt-in)
constexpr int MAX_STAGES = 8;
// 18 warps: producer, issuer and 16 drain warps (four per 32-lane TMEM quadrant, a
// quarter of the tile's columns each, so that a drain warp's int64 accumulators fit its
// registers: 65536 / 576 threads)
constexpr int NDRAIN = 16, NWARPS = 2 + NDRAIN, THREADS = NWARPS * 32;
constexpr int kGroupM = 12;                 // row tiles per CTA-order group (~sqrt(148))
constexpr uint32_t TMEM_COLS = 512;         // L0 @0, L1 @128, H @256 / @384 (alternating)

struct Params {
  int64_t M, N, Kp, batch;
  int nks;                                  // K stages per split (multiple of CHUNK_KS)
  int ksplit;                               // K splits (tiles per output tile)
  int stages;                               // stages in the ring
  const unsigned *ea, *eb;                  // row exponent codes [batch][M], [batch][N]
  double alpha, beta;
  double *C;
  int64_t ldc, sC;
  int to_ws;
};

__device__ int g_oz_err;

__device__ __forceinline__ uint32_t su32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mb_init(uint32_t b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(n) : "memory");
}
__device__ __forceinline__ void mb_expect(uint32_t b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mb_arrive(uint32_t b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}
__device__ __forceinline__ bool mb_wait(uint32_t b, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > (1ll << 31)) {
      atomicExch(&g_oz_err, 1);
      return false;
    }
  }
}
// one box of the 5-d plane map {256-byte run, slice, K block, 8-row group, batch}: the
// x coordinate is always 0 (16-byte aligned)
__device__ __forceinline__ void tma5(uint32_t dst, const CUtensorMap *m, uint32_t bar, int kb,
                                     int g, int b) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(bar), "r"(0), "r"(0), "r"(kb), "r"(g), "r"(b)
      : "memory");
}
// unswizzled K-major operand: 8 x 16-byte core matrices, the K-adjacent one 128 bytes on
// (leading offset), the next 8-row group `sbo` bytes on (stride offset)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void tld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// row exponent codes: e + 4096, 0 for an all-zero row
__device__ __forceinline__ int decode_exp(unsigned code) { return code ? (int)code - 4096 : 0; }

// Tile shape of a digit form: NL exact levels (one accumulator each), the lower levels in
// one FP32 accumulator per chunk (two buffers, alternating chunks), TBN output columns,
// FRAC fractional bits of the int64 fixed-point accumulator.
//   ns = 3..6: NL = 2, TBN = 128, FRAC = 12   (L0 @ 0, L1 @ 128, H @ 256 / 384)
//   ns = 7:    NL = 4, TBN = 64,  FRAC = 16   (L0..L3 @ 0, 64, 128, 192, H @ 256 / 320)
// The seven-digit form is the FP64-equivalent one: over a 512-deep chunk a level l sums
// l + 1 digit products of at most 128 x 64 per k (<= 1.26e7 < 2^24 for l = 3), so levels
// 0..3 are exact FP32 integers, and the levels >= 4 (2^-14 and below of the result, in
// ^a ^b units) carry the FP32 rounding of one chunk; |acc| <= K 2^44, so K per split stays
// <= 2^18, and the error of a product is about 2^-50 of max|a| max|b| per chunk, the level
// of an FP64 dot product, from 28 digit products.  Its tiles are 128 x 64 so that six
// 64-column accumulators fit the 512 TMEM columns.
template <int NS>
struct Form {
  static constexpr int NL = NS == 7 ? 4 : 2;
  static constexpr int TBN = NS == 7 ? 64 : 128;
  static constexpr int FRAC = NS == 7 ? 16 : 12;
  static constexpr uint32_t A_TILE = BM * KS * 2;            // 4 KB per slice
  static constexpr uint32_t B_TILE = TBN * KS * 2;
  static constexpr uint32_t STAGE = NS * (A_TILE + B_TILE);
  // kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both K-major
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(TBN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};
constexpr int64_t kXMaxKSplit = int64_t(1) << 18;   // K per split of the seven-digit form

// epilogue staging: every drain warp stages 32 rows x kEpiCols doubles at a time
constexpr int kEpiCols = 4;
constexpr uint32_t kEpiBytes = (uint32_t)NDRAIN * 32u * (kEpiCols + 1) * 8u;

__device__ __forceinline__ void umma(uint32_t acc_t, uint64_t da, uint64_t db, uint32_t idesc,
                                     uint32_t accum) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(acc_t),
      "l"(da), "l"(db), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// The digit GEMM as a persistent kernel: one CTA per SM walks the output tiles t =
// blockIdx.x, blockIdx.x + gridDim.x, ... (tile order: per batch member and K split,
// groups of kGroupM row tiles, column tiles within a group, so that the tiles in flight
// at one time share their A and B tiles in L2).  The three roles keep running counters
// across tiles (stages, chunks), so the next tile's loads and products start while the
// drain warps still write the previous tile's outputs from their registers.
template <int NS>
__global__ void __launch_bounds__(THREADS, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const Params p) {
  using F = Form<NS>;
  constexpr int NL = F::NL, TBN = F::TBN, FRAC = F::FRAC, WC = TBN / 4;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  const int nst = p.stages;
  double *epi = reinterpret_cast<double *>(smem + (size_t)nst * F::STAGE);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)nst * F::STAGE + kEpiBytes);
  // bar[0..nst) stage full, bar[nst..2nst) stage empty, bar[2nst] products of a chunk
  // done, bar[2nst+1] exact levels of a chunk drained, bar[2nst+2] every product issued
  // by this CTA done, bar[2nst+3+j] H buffer j drained (drain barriers: NDRAIN warps)
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bar + 2 * MAX_STAGES + 5);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gx = (p.M + BM - 1) / BM, gy = (p.N + TBN - 1) / TBN;
  const int64_t per_z = gx * gy, ntiles = per_z * p.batch * p.ksplit;
  const int nks_total = (int)(p.Kp / KS);
  struct Tile {
    int64_t m0, n0, b, split;
    int ks0, nk, nchunks;
  };
  auto tile_of = [&](int64_t t) {
    Tile o;
    const int64_t z = t / per_z, lin = t - z * per_z;
    const int64_t g = lin / ((int64_t)kGroupM * gy), idx = lin % ((int64_t)kGroupM * gy);
    const int64_t first = g * kGroupM, gsz = min((int64_t)kGroupM, gx - first);
    o.m0 = (first + idx % gsz) * BM;
    o.n0 = (idx / gsz) * TBN;
    o.b = z % p.batch;
    o.split = z / p.batch;
    o.ks0 = (int)o.split * p.nks;
    o.nk = max(min(o.ks0 + p.nks, nks_total) - o.ks0, 0);
    o.nchunks = (o.nk + CHUNK_KS - 1) / CHUNK_KS;
    return o;
  };

  if (threadIdx.x == 0) {
    for (int st = 0; st < nst; ++st) {
      mb_init(su32(&bar[st]), 1);
      mb_init(su32(&bar[nst + st]), 1);
    }
    mb_init(su32(&bar[2 * nst]), 1);
    mb_init(su32(&bar[2 * nst + 1]), NDRAIN * 32);
    mb_init(su32(&bar[2 * nst + 2]), 1);
    mb_init(su32(&bar[2 * nst + 3]), NDRAIN * 32);
    mb_init(su32(&bar[2 * nst + 4]), NDRAIN * 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_holder)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {  // ------------------------------------------ TMA producer
      int it = 0;     // stages loaded by this CTA so far
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const Tile tl = tile_of(t);
        for (int i = 0; i < tl.nk; ++i, ++it) {
          const int st = it % nst;
          if (!mb_wait(su32(&bar[nst + st]), ((uint32_t)(it / nst) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
          const uint32_t base = su32(smem + (size_t)st * F::STAGE);
          const uint32_t full = su32(&bar[st]);
          mb_expect(full, F::STAGE);
          // [16 groups][NS slices][256 B] of A, then [TBN / 8 groups][NS slices][256 B] of B
          tma5(base, &tmA, full, tl.ks0 + i, (int)(tl.m0 >> 3), (int)tl.b);
          tma5(base + NS * F::A_TILE, &tmB, full, tl.ks0 + i, (int)(tl.n0 >> 3), (int)tl.b);
        }
      }
      // the CTA may not exit with loads in flight: wait for the last load of every stage
      for (int j = max(it - nst, 0); j < it; ++j)
        mb_wait(su32(&bar[j % nst]), (uint32_t)(j / nst) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------------------ MMA issuer
      // per stage: every digit pair (i, j) from the resident slices.  The exact levels
      // restart every chunk and are drained by warps 2..17; at the first stage of a chunk
      // the lower-level pairs go first, so they overlap the drain of the previous chunk.
      // Descriptors of slice tiles: the stage base's plus the byte offset / 16 (slices of
      // one 8-row group 256 bytes apart, groups NS x 256 bytes).
      constexpr uint64_t kSl = CHUNK_BYTES >> 4;
      int it = 0, gch = 0;   // stages consumed, chunks issued (all tiles of this CTA)
      bool ok = true, issued = false;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const Tile tl = tile_of(t);
        for (int ch = 0; ch < tl.nchunks && ok; ++ch, ++gch) {
          const int kbeg = ch * CHUNK_KS, kend = min(kbeg + CHUNK_KS, tl.nk);
          for (int ks = kbeg; ks < kend; ++ks, ++it) {
            const int st = it % nst;
            if (!mb_wait(su32(&bar[st]), (uint32_t)(it / nst) & 1u)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sbase = su32(smem + (size_t)st * F::STAGE);
            const uint64_t da = sdesc(sbase, NS * CHUNK_BYTES);
            const uint64_t db = sdesc(sbase + NS * F::A_TILE, NS * CHUNK_BYTES);
            // lower levels into this chunk's H buffer; that buffer last held chunk gch - 2,
            // whose H pass the drain warps finish before they start on the exact levels
            // of chunk gch - 1 (one barrier per H buffer, one completion per use)
            if (ks == kbeg && gch >= 2) {
              if (!mb_wait(su32(&bar[2 * nst + 3 + (gch & 1)]),
                           (uint32_t)((gch - 2) >> 1) & 1u)) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
            const uint32_t acc_h = tmem + (uint32_t)((NL + (gch & 1)) * TBN);
#pragma unroll
            for (int l = NL; l < NS; ++l)
#pragma unroll
              for (int i = 0; i <= l; ++i)
                umma(acc_h, da + i * kSl, db + (l - i) * kSl, F::IDESC,
                     (ks > kbeg || l > NL || i > 0) ? 1u : 0u);
            // exact levels restart every chunk: the previous chunk's must be drained first
            // (its H buffer is drained afterwards, behind these products)
            if (ks == kbeg && gch > 0) {
              if (!mb_wait(su32(&bar[2 * nst + 1]), (uint32_t)(gch - 1) & 1u)) {
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            }
#pragma unroll
            for (int l = 0; l < NL; ++l)
#pragma unroll
              for (int i = 0; i <= l; ++i)
                umma(tmem + (uint32_t)(l * TBN), da + i * kSl, db + (l - i) * kSl, F::IDESC,
                     (ks > kbeg || i > 0) ? 1u : 0u);
            umma_commit(su32(&bar[nst + st]));
            issued = true;
          }
          if (!ok) break;
          umma_commit(su32(&bar[2 * nst]));   // this chunk's products complete -> drain
        }
      }
      // every product has completed before the tensor memory is released
      if (issued) {
        umma_commit(su32(&bar[2 * nst + 2]));
        mb_wait(su32(&bar[2 * nst + 2]), 0);
      }
    }
  } else {  // ------------------------------------------ drain warps 2..17
    const int ew = warp - 2;                  // 0..15
    const int quad = warp & 3;                // TMEM lane quadrant of this warp
    const int qc = ew >> 2;                   // columns [WC qc, WC qc + WC)
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
    double *st = epi + (size_t)ew * 32 * (kEpiCols + 1);
    int gch = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const Tile tl = tile_of(t);
      long long acc[WC];   // fixed point, FRAC fractional bits
#pragma unroll
      for (int j = 0; j < WC; ++j) acc[j] = 0;
      for (int ch = 0; ch < tl.nchunks; ++ch, ++gch) {
        // warp-uniform: the tensor-memory loads below are warp-collective
        ok = __all_sync(0xffffffffu, mb_wait(su32(&bar[2 * nst]), (uint32_t)gch & 1u));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // exact level l holds integers x 2^(14 - 7l): add them at 2^(14 - 7l + FRAC)
#pragma unroll
        for (int c = 0; c < WC / 16; ++c) {
          const uint32_t col = (uint32_t)(qc * WC + c * 16);
#pragma unroll
          for (int l = 0; l < NL; ++l) {
            uint32_t r[16];
            tld16(lane_base + (uint32_t)(l * TBN) + col, r);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const float unit = __int_as_float((127 - 14 + 7 * l) << 23);   // 2^(7l - 14)
#pragma unroll
            for (int j = 0; j < 16; ++j)
              acc[c * 16 + j] += (long long)__float2int_rn(__uint_as_float(r[j]) * unit)
                                 << (14 - 7 * l + FRAC);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mb_arrive(su32(&bar[2 * nst + 1]));
        // this chunk's lower levels, rounded to 2^-FRAC, from H buffer gch & 1
#pragma unroll
        for (int c = 0; c < WC / 16; ++c) {
          const uint32_t col = (uint32_t)(qc * WC + c * 16);
          uint32_t rh[16];
          tld16(lane_base + (uint32_t)((NL + (gch & 1)) * TBN) + col, rh);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; ++j)
            acc[c * 16 + j] += __float2ll_rn(__uint_as_float(rh[j]) * (float)(1 << FRAC));
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mb_arrive(su32(&bar[2 * nst + 3 + (gch & 1)]));
      }
      if (!ok) break;
      // epilogue from registers (the tensor memory is already free for the next tile):
      // C = alpha 2^(e_r + e_c - 28 - FRAC) acc + beta C, or the raw value into the
      // split-K workspace; kEpiCols columns at a time are staged as st[row][kEpiCols + 1]
      // (one row per lane, as the TMEM lane layout delivers it) and leave row-contiguous
      const int64_t row = tl.m0 + quad * 32 + lane;
      double *Cbase = p.to_ws ? p.C + ((tl.split * p.batch + tl.b) * p.M) * p.N
                              : p.C + tl.b * p.sC;
      const int64_t ldc = p.to_ws ? p.N : p.ldc;
      const bool rd = !p.to_ws && p.beta != 0.0;
      const int er = row < p.M ? decode_exp(p.ea[tl.b * p.M + row]) : 0;
      const int64_t col0 = tl.n0 + qc * WC;
      constexpr int RPI = 32 / kEpiCols;                 // rows per store instruction
      const int rs = lane / kEpiCols, cs = lane % kEpiCols;
      // one pass per kEpiCols columns, not unrolled: the accumulators shift down by
      // kEpiCols after each pass, so every pass reads acc[0 .. kEpiCols) (registers)
#pragma unroll 1
      for (int q = 0; q < WC / kEpiCols; ++q) {
        const int64_t cb = col0 + q * kEpiCols;
#pragma unroll
        for (int j = 0; j < kEpiCols; ++j) {
          const int64_t col = cb + j;
          st[lane * (kEpiCols + 1) + j] =
              (row < p.M && col < p.N)
                  ? ldexp((double)acc[j], er + decode_exp(p.eb[tl.b * p.N + col]) - 28 - FRAC)
                  : 0.0;
        }
#pragma unroll
        for (int j = 0; j < WC - kEpiCols; ++j) acc[j] = acc[j + kEpiCols];
        __syncwarp();
        const int64_t col = cb + cs;
        double old[32 / RPI];
#pragma unroll
        for (int u = 0; u < 32 / RPI; ++u) {
          const int64_t rr = tl.m0 + quad * 32 + u * RPI + rs;
          old[u] = (rd && rr < p.M && col < p.N) ? Cbase[rr * ldc + col] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 32 / RPI; ++u) {
          const int lr = u * RPI + rs;
          const int64_t rr = tl.m0 + quad * 32 + lr;
          if (rr < p.M && col < p.N) {
            const double x = st[lr * (kEpiCols + 1) + cs];
            Cbase[rr * ldc + col] =
                p.to_ws ? x : rd ? p.alpha * x + p.beta * old[u] : p.alpha * x;
          }
        }
        __syncwarp();
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

// ------------------------------------------------------------- split-BF16 GEMM
// The split-BF16 products (BF16x3 / x6 / x10: NS BF16 pieces per value, a = a_0 + a_1 +
// ..., the pairs i + j < NS) on the same persistent design and pre-tiled planes, with
// 128 x 256 tiles: every pair accumulates in FP32 over the split's K into one of two TMEM
// accumulators (tiles alternate between columns [0, 256) and [256, 512)), and the 16 drain
// warps write a finished tile from tensor memory while the next tile's products run.
constexpr int SBN = 256;
template <int NS>
struct SForm {
  static constexpr uint32_t A_TILE = BM * KS * 2, B_TILE = SBN * KS * 2;
  static constexpr uint32_t STAGE = NS * (A_TILE + B_TILE);
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                                    ((uint32_t)(SBN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};

template <int NS>
__global__ void __launch_bounds__(THREADS, 1)
split_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                  const __grid_constant__ CUtensorMap tmB, const Params p) {
  using F = SForm<NS>;
  constexpr int WC = SBN / 4;   // columns per drain warp
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  const int nst = p.stages;
  double *epi = reinterpret_cast<double *>(smem + (size_t)nst * F::STAGE);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)nst * F::STAGE + kEpiBytes);
  // bar[0..nst) stage full, bar[nst..2nst) stage empty, bar[2nst+j] accumulator j holds a
  // finished tile, bar[2nst+2+j] accumulator j read out (NDRAIN warps), bar[2nst+4] every
  // product issued by this CTA done
  uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bar + 2 * MAX_STAGES + 5);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gx = (p.M + BM - 1) / BM, gy = (p.N + SBN - 1) / SBN;
  const int64_t per_z = gx * gy, ntiles = per_z * p.batch * p.ksplit;
  const int nks_total = (int)(p.Kp / KS);
  struct Tile {
    int64_t m0, n0, b, split;
    int ks0, nk;
  };
  auto tile_of = [&](int64_t t) {
    Tile o;
    const int64_t z = t / per_z, lin = t - z * per_z;
    const int64_t g = lin / ((int64_t)kGroupM * gy), idx = lin % ((int64_t)kGroupM * gy);
    const int64_t first = g * kGroupM, gsz = min((int64_t)kGroupM, gx - first);
    o.m0 = (first + idx % gsz) * BM;
    o.n0 = (idx / gsz) * SBN;
    o.b = z % p.batch;
    o.split = z / p.batch;
    o.ks0 = (int)o.split * p.nks;
    o.nk = max(min(o.ks0 + p.nks, nks_total) - o.ks0, 0);
    return o;
  };

  if (threadIdx.x == 0) {
    for (int st = 0; st < nst; ++st) {
      mb_init(su32(&bar[st]), 1);
      mb_init(su32(&bar[nst + st]), 1);
    }
    mb_init(su32(&bar[2 * nst]), 1);
    mb_init(su32(&bar[2 * nst + 1]), 1);
    mb_init(su32(&bar[2 * nst + 2]), NDRAIN * 32);
    mb_init(su32(&bar[2 * nst + 3]), NDRAIN * 32);
    mb_init(su32(&bar[2 * nst + 4]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_holder)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {  // ------------------------------------------ TMA producer
      int it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const Tile tl = tile_of(t);
        for (int i = 0; i < tl.nk; ++i, ++it) {
          const int st = it % nst;
          if (!mb_wait(su32(&bar[nst + st]), ((uint32_t)(it / nst) & 1u) ^ 1u)) {
            ok = false;
            break;
          }
          const uint32_t base = su32(smem + (size_t)st * F::STAGE);
          const uint32_t full = su32(&bar[st]);
          mb_expect(full, F::STAGE);
          // [16 groups][NS pieces][256 B] of A, then [32 groups][NS pieces][256 B] of B
          tma5(base, &tmA, full, tl.ks0 + i, (int)(tl.m0 >> 3), (int)tl.b);
          tma5(base + NS * F::A_TILE, &tmB, full, tl.ks0 + i, (int)(tl.n0 >> 3), (int)tl.b);
        }
      }
      for (int j = max(it - nst, 0); j < it; ++j)
        mb_wait(su32(&bar[j % nst]), (uint32_t)(j / nst) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ------------------------------------------ MMA issuer
      constexpr uint64_t kSl = CHUNK_BYTES >> 4;
      int it = 0, lt = 0;   // stages consumed, tiles issued (this CTA)
      bool ok = true, issued = false;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++lt) {
        const Tile tl = tile_of(t);
        const int j = lt & 1;
        // accumulator j last held tile lt - 2: the drain warps must have read it out
        if (lt >= 2) {
          if (!mb_wait(su32(&bar[2 * nst + 2 + j]), (uint32_t)((lt - 2) >> 1) & 1u)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        const uint32_t acc = tmem + (uint32_t)(j * SBN);
        for (int i = 0; i < tl.nk; ++i, ++it) {
          const int st = it % nst;
          if (!mb_wait(su32(&bar[st]), (uint32_t)(it / nst) & 1u)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sbase = su32(smem + (size_t)st * F::STAGE);
          const uint64_t da = sdesc(sbase, NS * CHUNK_BYTES);
          const uint64_t db = sdesc(sbase + NS * F::A_TILE, NS * CHUNK_BYTES);
#pragma unroll
          for (int l = 0; l < NS; ++l)
#pragma unroll
            for (int i2 = 0; i2 <= l; ++i2)
              umma(acc, da + i2 * kSl, db + (l - i2) * kSl, F::IDESC,
                   (i > 0 || l > 0 || i2 > 0) ? 1u : 0u);
          umma_commit(su32(&bar[nst + st]));
          issued = true;
        }
        if (!ok) break;
        umma_commit(su32(&bar[2 * nst + j]));   // this tile's products complete -> write
      }
      if (issued) {
        umma_commit(su32(&bar[2 * nst + 4]));
        mb_wait(su32(&bar[2 * nst + 4]), 0);
      }
    }
  } else {  // ------------------------------------------ drain warps 2..17
    const int ew = warp - 2, quad = warp & 3, qc = ew >> 2;   // columns [WC qc, WC qc + WC)
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
    double *st = epi + (size_t)ew * 32 * (kEpiCols + 1);
    constexpr int RPI = 32 / kEpiCols;
    const int rs = lane / kEpiCols, cs = lane % kEpiCols;
    int lt = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const Tile tl = tile_of(t);
      const int j = lt & 1;
      // warp-uniform (the tensor-memory loads below are warp-collective)
      if (!__all_sync(0xffffffffu, mb_wait(su32(&bar[2 * nst + j]), (uint32_t)(lt >> 1) & 1u)))
        break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t row = tl.m0 + quad * 32 + lane;
      double *Cbase = p.to_ws ? p.C + ((tl.split * p.batch + tl.b) * p.M) * p.N
                              : p.C + tl.b * p.sC;
      const int64_t ldc = p.to_ws ? p.N : p.ldc;
      const bool rd = !p.to_ws && p.beta != 0.0;
#pragma unroll 1
      for (int c = 0; c < WC / 16; ++c) {
        uint32_t r[16];
        tld16(lane_base + (uint32_t)(j * SBN + qc * WC + c * 16), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c == WC / 16 - 1) {   // the accumulator is read out: the issuer may reuse it
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mb_arrive(su32(&bar[2 * nst + 2 + j]));
        }
#pragma unroll
        for (int q = 0; q < 16 / kEpiCols; ++q) {
          const int64_t cb = tl.n0 + qc * WC + c * 16 + q * kEpiCols;
#pragma unroll
          for (int jj = 0; jj < kEpiCols; ++jj)
            st[lane * (kEpiCols + 1) + jj] =
                (row < p.M && cb + jj < p.N) ? (double)__uint_as_float(r[q * kEpiCols + jj])
                                             : 0.0;
          __syncwarp();
          const int64_t col = cb + cs;
          double old[32 / RPI];
#pragma unroll
          for (int u = 0; u < 32 / RPI; ++u) {
            const int64_t rr = tl.m0 + quad * 32 + u * RPI + rs;
            old[u] = (rd && rr < p.M && col < p.N) ? Cbase[rr * ldc + col] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 32 / RPI; ++u) {
            const int lr = u * RPI + rs;
            const int64_t rr = tl.m0 + quad * 32 + lr;
            if (rr < p.M && col < p.N) {
              const double x = st[lr * (kEpiCols + 1) + cs];
              Cbase[rr * ldc + col] =
                  p.to_ws ? x : rd ? p.alpha * x + p.beta * old[u] : p.alpha * x;
            }
          }
          __syncwarp();
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

// common exponent of every row r of op(X): e with max_k |op(X)[r][k]| < 2^e, stored as
// code = e + 4096 (0 for an all-zero row) and combined across blocks with atomicMax.
// Tiles of 32 rows x 1024 k; the read is coalesced along whichever index is contiguous.
__global__ void oz_rowexp_kernel(const double *__restrict__ X, int64_t rows, int64_t K,
                                 int64_t ld, int64_t sX, int trans, int64_t batch,
                                 unsigned *__restrict__ code) {
  constexpr int KT = 1024;
  const int64_t rt = (rows + 31) / 32, kt = (K + KT - 1) / KT;
  const int64_t ntiles = rt * kt * batch;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t b = t / (rt * kt), rem = t % (rt * kt);
    const int64_t r0 = (rem / kt) * 32, k0 = (rem % kt) * KT;
    const int64_t k1 = min(K, k0 + KT);
    const double *Xb = X + b * sX;
    if (!trans) {  // warp per row, lanes along k, eight independent loads in flight
      for (int i = warp; i < 32; i += nw) {
        const int64_t r = r0 + i;
        if (r >= rows) continue;
        const double *x = Xb + r * ld;
        double mm[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int64_t k = k0 + lane;
        for (; k + 224 < k1; k += 256) {
#pragma unroll
          for (int u = 0; u < 8; ++u) mm[u] = fmax(mm[u], fabs(x[k + 32 * u]));
        }
        for (; k < k1; k += 32) mm[0] = fmax(mm[0], fabs(x[k]));
        double m = mm[0];
#pragma unroll
        for (int u = 1; u < 8; ++u) m = fmax(m, mm[u]);
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && m > 0.0) {
          int ex;
          frexp(m, &ex);
          atomicMax(&code[b * rows + r], (unsigned)(ex + 4096));
        }
      }
    } else {  // lanes along r (contiguous), warps split the k range, eight loads in flight
      const int64_t r = r0 + lane;
      double m = 0.0;
      if (r < rows) {
        double mm[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int64_t k = k0 + warp;
        for (; k + 7 * nw < k1; k += 8 * nw) {
#pragma unroll
          for (int u = 0; u < 8; ++u) mm[u] = fmax(mm[u], fabs(Xb[(k + u * nw) * ld + r]));
        }
        for (; k < k1; k += nw) mm[0] = fmax(mm[0], fabs(Xb[k * ld + r]));
        m = mm[0];
#pragma unroll
        for (int u = 1; u < 8; ++u) m = fmax(m, mm[u]);
      }
      if (r < rows && m > 0.0) {
        int ex;
        frexp(m, &ex);
        atomicMax(&code[b * rows + r], (unsigned)(ex + 4096));
      }
    }
  }
}

// Digit planes: a' = a 2^-e (e the row's exponent) times 2^(7 NS), rounded once to the
// integer q (|q| < 2^(7 NS)), is cut into balanced base-128 digits, d_{NS-1} .. d_1 in
// [-64, 63] from the bottom (d_s = ((q + 64) mod 128) - 64, q <- (q - d_s) / 128) and d_0
// the remaining top digit (|d_0| <= 128).  The recursion only reads the low 7 bits and
// divides exact multiples of 128, so the low three digits come from the low 21 bits in
// 32-bit arithmetic and the rest from the high part plus the carry.
//
// Plane layout (pre-tiled for the MMA, zero padded for k >= K and for the rows of the
// last 8-row group beyond `rows`): value (b, r, k) of slice s at BF16 index
//     ((((b G + r/8) KB + k/16) ns + s) 2 + (k/8) % 2) 64 + (r % 8) 8 + k % 8,
// G = ceil(rows / 8), KB = Kp / 16: one 256-byte run per (8-row group, 16-wide K block,
// slice) holding the two 8 x 8 core matrices of the block.
template <int NS>
__device__ __forceinline__ void balanced_digits(long long q, int (&d)[NS]) {
  constexpr int NLOW = NS - 1 < 3 ? NS - 1 : 3;
  int lo = (int)(q & 0x1FFFFF);
#pragma unroll
  for (int t = 0; t < NLOW; ++t) {
    const int dd = ((lo + 64) & 127) - 64;
    d[NS - 1 - t] = dd;
    lo = (lo - dd) >> 7;
  }
  int r = (int)((q >> 21) * (1ll << (21 - 7 * NLOW))) + lo;
#pragma unroll
  for (int s2 = NS - 1 - NLOW; s2 >= 1; --s2) {
    const int dd = ((r + 64) & 127) - 64;
    d[s2] = dd;
    r = (r - dd) >> 7;
  }
  d[0] = r;
}

// ^a_s = d_s 2^(-7(s-1)) as BF16 (exact: at most 8 significant bits)
template <int S>
__device__ __forceinline__ float digit_value(int d) {
  return (float)d * __int_as_float((127 - 7 * (S - 1)) << 23);
}

template <int NS, int S = 0>
__device__ __forceinline__ void store_pairs(__nv_bfloat16 *o, const int (&d0)[NS],
                                            const int (&d1)[NS]) {
  if constexpr (S < NS) {
    *reinterpret_cast<__nv_bfloat162 *>(o + S * (CHUNK_BYTES / 2)) =
        __floats2bfloat162_rn(digit_value<S>(d0[S]), digit_value<S>(d1[S]));
    store_pairs<NS, S + 1>(o, d0, d1);
  }
}

// planes are written in units of one 8-row group x one 8-wide K half: 32 lanes, lane =
// 4 (r % 8) + j, two consecutive k = 8 h + 2 j, 8 h + 2 j + 1, so that each store of a
// slice is one contiguous 128-byte core matrix
// BF16 pieces of a value for the split-BF16 products, a_s = bf16(a - a_0 - ... - a_{s-1}):
// up to three in FP32 (which holds the 24 bits three pieces carry, so the slicing is exact
// there), four with FP64 remainders
template <int NS>
__device__ __forceinline__ void bf_pieces(double v, __nv_bfloat16 (&q)[NS]) {
  if constexpr (NS <= 3) {
    float rem = (float)v;
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) {
      q[sl] = __float2bfloat16_rn(rem);
      rem -= __bfloat162float(q[sl]);
    }
  } else {
    double rem = v;
#pragma unroll
    for (int sl = 0; sl < NS; ++sl) {
      q[sl] = __double2bfloat16(rem);
      rem -= (double)__bfloat162float(q[sl]);
    }
  }
}

// FL: BF16 pieces of every value (no common exponent) instead of digits
template <int NS, bool FL>
__device__ __forceinline__ void split_pair(double v0, double v1, double scale,
                                           __nv_bfloat16 *chunk, int h, int lane) {
  __nv_bfloat16 *o = chunk + h * 64 + (lane >> 2) * 8 + (lane & 3) * 2;
  if constexpr (FL) {
    __nv_bfloat16 q0[NS], q1[NS];
    bf_pieces<NS>(v0, q0);
    bf_pieces<NS>(v1, q1);
#pragma unroll
    for (int sl = 0; sl < NS; ++sl)
      *reinterpret_cast<__nv_bfloat162 *>(o + sl * (CHUNK_BYTES / 2)) =
          __halves2bfloat162(q0[sl], q1[sl]);
  } else {
    int d0[NS], d1[NS];
    balanced_digits<NS>(__double2ll_rn(v0 * scale), d0);
    balanced_digits<NS>(__double2ll_rn(v1 * scale), d1);
    store_pairs<NS>(o, d0, d1);
  }
}

// Digit planes of op(X) = X (rows contiguous along K): one warp per (8-row group, run of
// kSplitSeg K), one K half (8 wide) of the group per step, four steps in flight
constexpr int64_t kSplitSeg = 1024;
template <int NS, bool FL>
__global__ void oz_split_rows_kernel(const double *__restrict__ X, int64_t rows, int64_t K,
                                     int64_t ld, int64_t sX, const unsigned *__restrict__ e,
                                     __nv_bfloat16 *__restrict__ out, int64_t Kp, int64_t batch) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t G = (rows + 7) / 8, KB = Kp / 16;
  const int64_t nseg = (Kp + kSplitSeg - 1) / kSplitSeg;
  for (int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
       item < batch * G * nseg; item += nwarps) {
    const int64_t bg = item / nseg, seg = item - bg * nseg;
    const int64_t b = bg / G, g = bg - b * G;
    const int64_t r = g * 8 + (lane >> 2);
    const bool live = r < rows;
    const double *x = X + b * sX + (live ? r : 0) * ld;
    const int ex = (!FL && live) ? decode_exp(e[b * rows + r]) : 0;
    const double scale = __longlong_as_double((long long)(1023 - ex + 7 * NS) << 52);
    const int64_t h0 = seg * (kSplitSeg / 8), h1 = min(Kp, (seg + 1) * kSplitSeg) / 8;
    for (int64_t hb = h0; hb < h1; hb += 4) {   // K halves hb .. hb + 3 (h1 - h0 is even)
      double v[8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t k = (hb + u) * 8 + (lane & 3) * 2;
        const bool in = live && hb + u < h1;
        v[2 * u] = (in && k < K) ? x[k] : 0.0;
        v[2 * u + 1] = (in && k + 1 < K) ? x[k + 1] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (hb + u >= h1) break;
        const int64_t kb = (hb + u) >> 1;
        __nv_bfloat16 *chunk = out + ((bg * KB + kb) * NS) * (CHUNK_BYTES / 2);
        split_pair<NS, FL>(v[2 * u], v[2 * u + 1], scale, chunk, (int)((hb + u) & 1), lane);
      }
    }
  }
}

// Digit planes of op(X) = X^T (X stored K x rows): 32 rows x 64 k tiles transposed
// through shared memory (loads coalesced along the rows), then each warp writes whole
// core matrices as above
template <int NS, bool FL>
__global__ void oz_split_cols_kernel(const double *__restrict__ X, int64_t rows, int64_t K,
                                     int64_t ld, int64_t sX, const unsigned *__restrict__ e,
                                     __nv_bfloat16 *__restrict__ out, int64_t Kp, int64_t batch) {
  __shared__ double tile[64][33];   // [k][row]
  __shared__ int64_t s_t[3];         // batch member, first row, first k of the tile
  const int64_t G = (rows + 7) / 8, KB = Kp / 16;
  const int64_t rt = (G + 3) / 4, kt = Kp / 64;   // Kp is a multiple of 64
  const int64_t ntiles = rt * kt * batch;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    if (tx == 0 && ty == 0) {   // one thread decodes the tile index
      const int64_t bb = t / (rt * kt), rem = t % (rt * kt);
      s_t[0] = bb;
      s_t[1] = (rem / kt) * 32;
      s_t[2] = (rem % kt) * 64;
    }
    __syncthreads();
    const int64_t b = s_t[0], r0 = s_t[1], k0 = s_t[2];
    const double *Xb = X + b * sX;
    for (int i = ty; i < 64; i += 8) {   // k = k0 + i, lanes along the rows (contiguous)
      const int64_t k = k0 + i, r = r0 + tx;
      tile[i][tx] = (k < K && r < rows) ? Xb[k * ld + r] : 0.0;
    }
    __syncthreads();
    // 4 groups x 8 K halves = 32 core matrices per tile, four per warp
    const int rr = tx >> 2, jj = tx & 3;
    for (int c = ty; c < 32; c += 8) {
      const int gl = c >> 3, hl = c & 7;   // group within the tile, K half within the tile
      const int64_t g = (r0 >> 3) + gl;
      if (g >= G) continue;
      const int64_t r = g * 8 + rr;
      const int ex = (!FL && r < rows) ? decode_exp(e[b * rows + r]) : 0;
      const double scale = __longlong_as_double((long long)(1023 - ex + 7 * NS) << 52);
      const int kl = hl * 8 + jj * 2;
      const int64_t kb = (k0 >> 4) + (hl >> 1);
      __nv_bfloat16 *chunk = out + (((b * G + g) * KB + kb) * NS) * (CHUNK_BYTES / 2);
      split_pair<NS, FL>(tile[kl][gl * 8 + rr], tile[kl + 1][gl * 8 + rr], scale, chunk,
                         hl & 1, tx);
    }
  }
}

template <int NS, bool FL = false>
static void launch_split(const double *X, int64_t rows, int64_t K, int64_t ld, int64_t sX,
                         bool trans, const unsigned *e, __nv_bfloat16 *out, int64_t Kp,
                         int64_t batch, cudaStream_t s) {
  const int64_t G = (rows + 7) / 8;
  if (trans) {
    const int64_t t = ((G + 3) / 4) * (Kp / 64) * batch;
    oz_split_cols_kernel<NS, FL><<<(unsigned)std::min<int64_t>(std::max<int64_t>(t, 1), 148 * 32),
                               dim3(32, 8), 0, s>>>(X, rows, K, ld, sX, e, out, Kp, batch);
  } else {
    const int64_t warps = G * batch * ((Kp + kSplitSeg - 1) / kSplitSeg);
    oz_split_rows_kernel<NS, FL><<<(unsigned)std::min<int64_t>(std::max<int64_t>((warps + 7) / 8, 1),
                                                            148 * 16),
                               256, 0, s>>>(X, rows, K, ld, sX, e, out, Kp, batch);
  }
  TRG_LAUNCH_CHECK();
}

__global__ void oz_ws_reduce(const double *__restrict__ W, int ksplit, int64_t batch, int64_t M,
                             int64_t N, double alpha, double beta, double *__restrict__ C,
                             int64_t ldc, int64_t sC) {
  const int64_t total = batch * M * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < ksplit; ++s) acc += W[s * total + i];
    const int64_t bb = i / (M * N), mn = i % (M * N), m = mn / N, n = mn % N;
    double *c = C + bb * sC + m * ldc + n;
    *c = (beta == 0.0) ? alpha * acc : alpha * acc + beta * *c;
  }
}

static PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void *f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  if (!fn) throw Error(TRG_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  return fn;
}

// the pre-tiled planes as a 5-d tensor {128 BF16 (one 256-byte run), slice, K block,
// 8-row group, batch}; a box is every slice of box_rows / 8 groups at one K block, landing
// in shared memory as [group][slice][256 B]; groups beyond G read as zeros
static CUtensorMap tmap(const void *base, int64_t Kp, int64_t rows, int64_t batch, int ns,
                        int box_rows = 128) {
  CUtensorMap m;
  const int64_t G = (rows + 7) / 8, KB = Kp / 16, run = CHUNK_BYTES;
  cuuint64_t dims[5] = {(cuuint64_t)(CHUNK_BYTES / 2), (cuuint64_t)ns, (cuuint64_t)KB,
                        (cuuint64_t)G, (cuuint64_t)batch};
  cuuint64_t strides[4] = {(cuuint64_t)run, (cuuint64_t)(ns * run), (cuuint64_t)(KB * ns * run),
                           (cuuint64_t)(G * KB * ns * run)};
  cuuint32_t box[5] = {(cuuint32_t)(CHUNK_BYTES / 2), (cuuint32_t)ns, 1, (cuuint32_t)(box_rows / 8),
                       1};
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = encoder()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(base), dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(TRG_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

// alignment slack, barriers and the TMEM address beside the stage ring and the staging
constexpr size_t kSmemFixed = 1024 + 256 + kEpiBytes;

}  // namespace oz

int oz_error_flag(bool reset) {
  int v = 0;
  cudaMemcpyFromSymbol(&v, oz::g_oz_err, sizeof(int));
  if (reset) {
    int z = 0;
    cudaMemcpyToSymbol(oz::g_oz_err, &z, sizeof(int));
  }
  return v;
}

// rows of op(X) per block of the small-K exponent kernel
__global__ void oz_rowexp_small_kernel(const double *__restrict__ X, int64_t rows, int64_t K,
                                       int64_t ld, int64_t sX, int64_t batch,
                                       unsigned *__restrict__ code) {
  // op(X) = X (rows contiguous along K), K <= 128: one thread per row
  const int64_t total = rows * batch;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / rows, r = t % rows;
    const double *x = X + b * sX + r * ld;
    double m = 0.0;
    for (int64_t k = 0; k < K; ++k) m = fmax(m, fabs(x[k]));
    unsigned cd = 0;
    if (m > 0.0) {
      int ex;
      frexp(m, &ex);
      cd = (unsigned)(ex + 4096);
    }
    code[b * rows + r] = cd;
  }
}

OzOperand oz_prepare(const double *X, int64_t rows, int64_t K, int64_t ld, int64_t sX,
                     bool trans, int64_t batch, int ns, TcScratch &scr, cudaStream_t s,
                     bool fl) {
  using namespace oz;
  OzOperand o;
  o.rows = rows;
  o.K = K;
  o.Kp = std::max<int64_t>(BK, (K + BK - 1) / BK * BK);
  o.batch = batch;
  o.ns = ns;
  o.fl = fl;
  __nv_bfloat16 *pl =
      (__nv_bfloat16 *)scr.alloc((size_t)ns * batch * ((rows + 7) / 8 * 8) * o.Kp * 2);
  if (fl) {   // BF16 pieces of every value: no common exponents
    switch (ns) {
      case 2: launch_split<2, true>(X, rows, K, ld, sX, trans, nullptr, pl, o.Kp, batch, s); break;
      case 3: launch_split<3, true>(X, rows, K, ld, sX, trans, nullptr, pl, o.Kp, batch, s); break;
      default: launch_split<4, true>(X, rows, K, ld, sX, trans, nullptr, pl, o.Kp, batch, s); break;
    }
    o.planes = pl;
    return o;
  }
  unsigned *e = (unsigned *)scr.alloc((size_t)batch * rows * sizeof(unsigned));
  if (!trans && K <= 128) {
    const int64_t t = (rows * batch + 255) / 256;
    oz_rowexp_small_kernel<<<(unsigned)std::min<int64_t>(std::max<int64_t>(t, 1), 148 * 64),
                             256, 0, s>>>(X, rows, K, ld, sX, batch, e);
    TRG_LAUNCH_CHECK();
  } else {
    TRG_CUDA(cudaMemsetAsync(e, 0, (size_t)batch * rows * sizeof(unsigned), s));
    const int64_t t = ((rows + 31) / 32) * ((K + 1023) / 1024) * batch;
    oz_rowexp_kernel<<<(unsigned)std::min<int64_t>(std::max<int64_t>(t, 1), 148 * 32), 256, 0,
                       s>>>(X, rows, K, ld, sX, trans ? 1 : 0, batch, e);
    TRG_LAUNCH_CHECK();
  }
  switch (ns) {
    case 3: launch_split<3>(X, rows, K, ld, sX, trans, e, pl, o.Kp, batch, s); break;
    case 4: launch_split<4>(X, rows, K, ld, sX, trans, e, pl, o.Kp, batch, s); break;
    case 5: launch_split<5>(X, rows, K, ld, sX, trans, e, pl, o.Kp, batch, s); break;
    case 6: launch_split<6>(X, rows, K, ld, sX, trans, e, pl, o.Kp, batch, s); break;
    default: launch_split<7>(X, rows, K, ld, sX, trans, e, pl, o.Kp, batch, s); break;
  }
  o.e = e;
  o.planes = pl;
  return o;
}

void gemm_oz(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
             int64_t lda, int64_t sA, const double *B, int64_t ldb, int64_t sB, double beta,
             double *C, int64_t ldc, int64_t sC, int64_t batch, int ns, TcScratch &scr,
             cudaStream_t s, TcTiming *timing, const OzOperand *pa, const OzOperand *pb,
             bool fl) {
  using namespace oz;
  if (M == 0 || N == 0 || batch == 0) return;
  if (!fl && (ns < 3 || ns > 7)) throw Error(TRG_ERR_ARG, "gemm_oz: 3 <= digits <= 7");
  if (fl && (ns < 2 || ns > 4)) throw Error(TRG_ERR_ARG, "gemm_oz: 2 <= BF16 pieces <= 4");
  const bool x7 = !fl && ns == 7;   // the FP64-equivalent form: its own tile width
  const int bn = fl ? SBN : x7 ? Form<7>::TBN : Form<5>::TBN;
  const size_t stage_bytes = (size_t)ns * (BM + bn) * KS * 2;
  const int64_t Kp = std::max<int64_t>(BK, (K + BK - 1) / BK * BK);
  auto fits = [&](const OzOperand *o, int64_t rows) {
    return o && o->rows == rows && o->K == K && o->Kp == Kp && o->batch == batch && o->ns == ns &&
           o->fl == fl;
  };
  if ((pa && !fits(pa, M)) || (pb && !fits(pb, N)))
    throw Error(TRG_ERR_ARG, "gemm_oz: prepared operand does not match the product");
  // a Gram (op(A) = X^T, op(B) = X, or op(A) = X, op(B) = X^T) has identical digit planes
  const bool gram = A == B && ta != tb && M == N && lda == ldb && sA == sB;
  OzOperand oa = pa ? *pa : oz_prepare(A, M, K, lda, sA, ta, batch, ns, scr, s, fl);
  OzOperand ob = pb ? *pb : gram ? oa : oz_prepare(B, N, K, ldb, sB, !tb, batch, ns, scr, s, fl);
  Params p{};
  p.M = M;
  p.N = N;
  p.Kp = Kp;
  p.batch = batch;
  p.alpha = alpha;
  p.beta = beta;
  p.ea = oa.e;
  p.eb = ob.e;
  const int npairs = ns * (ns + 1) / 2;    // digit (piece) pairs i + j <= ns - 1
  const int64_t gx = (M + BM - 1) / BM, gy = (N + bn - 1) / bn;
  const int nks_total = (int)(Kp / KS);
  // thread-safe one-time setup (function-local static initialisation): the shared-memory
  // opt-in and the number of SMs (one persistent CTA each)
  static const int n_sm = [] {
    for (const void *k : {(const void *)oz_gemm_kernel<3>, (const void *)oz_gemm_kernel<4>,
                          (const void *)oz_gemm_kernel<5>, (const void *)oz_gemm_kernel<6>,
                          (const void *)oz_gemm_kernel<7>, (const void *)split_gemm_kernel<2>,
                          (const void *)split_gemm_kernel<3>, (const void *)split_gemm_kernel<4>})
      TRG_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmemOptin));
    int dev = 0, n = 0;
    TRG_CUDA(cudaGetDevice(&dev));
    TRG_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    return std::max(n, 1);
  }();
  // K splits: the count that minimises the estimated time, in K stages (about 0.5 us
  // each), of ceil(tiles / SMs) rounds of (stages per split + 8 for a tile's fixed cost),
  // plus the split-K workspace round trip at HBM speed; a further split must gain 3 %
  const int64_t tiles = gx * gy * batch;
  auto est = [&](int ks) {
    int per = (nks_total + ks - 1) / ks;
    per = (per + CHUNK_KS - 1) / CHUNK_KS * CHUNK_KS;
    const int kse = (nks_total + per - 1) / per;
    const double rounds = std::ceil((double)(tiles * kse) / n_sm);
    const double ws = kse > 1 ? (2.0 * kse + 1) * (double)(batch * M * N) * 8 / 6e12 / 0.5e-6 : 0;
    return rounds * (per + 8.0) + ws;
  };
  int ksplit = 1;
  double t_best = est(1);
  const int ks_hi = (int)std::min<int64_t>(
      nks_total / CHUNK_KS, std::max<int64_t>(16, (2 * n_sm + tiles - 1) / tiles));
  for (int ks = 2; ks <= ks_hi; ++ks) {
    const double t = est(ks);
    if (t < 0.97 * t_best) {
      t_best = t;
      ksplit = ks;
    }
  }
  // the fixed-point accumulator holds K 2^41 < 2^63 (K 2^44 in the seven-digit form): at
  // most 2^21 (2^18) K per split; BF16 pieces accumulate in FP32 (no limit)
  const int64_t kmax = fl ? (int64_t(1) << 40) : x7 ? kXMaxKSplit : (int64_t(1) << 21);
  ksplit = std::max<int>(ksplit, (int)((Kp + kmax - 1) / kmax));
  int per = (nks_total + ksplit - 1) / ksplit;
  per = (per + CHUNK_KS - 1) / CHUNK_KS * CHUNK_KS;
  ksplit = (nks_total + per - 1) / per;
  p.nks = per;
  p.ksplit = ksplit;
  p.stages = (int)std::min<size_t>(MAX_STAGES, (kSmemOptin - kSmemFixed) / stage_bytes);
  const size_t smem = (size_t)p.stages * stage_bytes + kSmemFixed;
  if (ksplit > 1) {
    p.C = (double *)scr.alloc((size_t)ksplit * batch * M * N * sizeof(double));
    p.to_ws = 1;
    p.ldc = N;
    p.sC = M * N;
  } else {
    p.C = C;
    p.to_ws = 0;
    p.ldc = ldc;
    p.sC = sC;
  }
  CUtensorMap ma = tmap(oa.planes, Kp, M, batch, ns), mb = tmap(ob.planes, Kp, N, batch, ns, bn);
  const int64_t ntiles = gx * gy * batch * ksplit;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, n_sm);
  if (debug_opt("attr")) {
    const void *fns[4] = {(const void *)oz_gemm_kernel<5>, (const void *)oz_rowexp_kernel,
                          (const void *)oz_split_rows_kernel<5, false>,
                          (const void *)oz_ws_reduce};
    for (int i = 0; i < 4; ++i) {
      cudaFuncAttributes fa;
      cudaFuncGetAttributes(&fa, fns[i]);
      fprintf(stderr, "oz kernel %d: regs %d maxThreads %d static smem %zu max dyn smem %d local %zu\n",
              i, fa.numRegs, fa.maxThreadsPerBlock, fa.sharedSizeBytes,
              fa.maxDynamicSharedSizeBytes, fa.localSizeBytes);
    }
    fprintf(stderr, "launch: tiles %lld x %lld x %lld, grid %u threads %d smem %zu stages %d\n",
            (long long)gx, (long long)gy, (long long)(batch * ksplit), grid, THREADS, smem,
            p.stages);
  }
  if (timing) timing->before(s);
  if (fl) {
    switch (ns) {
      case 2: split_gemm_kernel<2><<<grid, THREADS, smem, s>>>(ma, mb, p); break;
      case 3: split_gemm_kernel<3><<<grid, THREADS, smem, s>>>(ma, mb, p); break;
      default: split_gemm_kernel<4><<<grid, THREADS, smem, s>>>(ma, mb, p); break;
    }
  } else {
    switch (ns) {
      case 3: oz_gemm_kernel<3><<<grid, THREADS, smem, s>>>(ma, mb, p); break;
      case 4: oz_gemm_kernel<4><<<grid, THREADS, smem, s>>>(ma, mb, p); break;
      case 5: oz_gemm_kernel<5><<<grid, THREADS, smem, s>>>(ma, mb, p); break;
      case 6: oz_gemm_kernel<6><<<grid, THREADS, smem, s>>>(ma, mb, p); break;
      default: oz_gemm_kernel<7><<<grid, THREADS, smem, s>>>(ma, mb, p); break;
    }
  }
  TRG_LAUNCH_CHECK();
  // timing kinds: 0 digit GEMM, 1 split-BF16 GEMM, 2 seven-digit GEMM
  if (timing)
    timing->after(s, fl ? 1 : x7 ? 2 : 0, 2.0 * (double)M * N * K * batch,
                  2.0 * (double)M * N * K * batch * npairs);
  if (ksplit > 1) {
    const int64_t total = batch * M * N;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 148 * 16);
    oz_ws_reduce<<<blocks, 256, 0, s>>>(p.C, ksplit, batch, M, N, alpha, beta, C, ldc, sC);
    TRG_LAUNCH_CHECK();
  }
}

}  // namespace trg
