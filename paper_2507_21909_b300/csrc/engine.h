// Engine of libtrg (internal): the per-context state of a coarse-graining run and the
// building blocks of a step, shared by the 4D and 3D triad steps, the batched lanes and
// the plain-ATRG comparator: GEMM routing (FP64 cores, split GEMM, digit GEMMs), tensor
// helpers, decompositions (CholeskyQR, Jacobi SVD, range finders, squeezer roots) and
// the sliced coarse contraction.  Definitions in engine.cu; the steps in triad_step.cu;
// contexts and the C ABI in context.cu, batch.cu, atrg.cu.
#pragma once

#include <algorithm>
#include <thread>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <utility>

#include "gemm_oz.h"
#include "gemm_tc.h"
#include "sketch_mlp.h"
#include "trg_internal.h"

namespace trg {


constexpr double kRankTol = 1e-13;     // singular values <= kRankTol * max are zeros
constexpr double kShiftRel = 1e-14;    // relative shift of the first CholeskyQR pass
constexpr double kPivotTol = 1e-13;    // dead-pivot threshold of the later passes

// sketch tags of one step (same numbering in every implementation of the method)
enum { TAG_SWAP_G1 = 1, TAG_SWAP_G2 = 2, TAG_RHO_A = 3, TAG_RHO_X = 4, TAG_RHO_Y = 5,
       TAG_RHO_D = 6, TAG_SQ_F2 = 7, TAG_SQ_B2 = 10, TAG_PROBE_A = 13 };

struct Ctx {
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  Arena arena;
  bool init = false;
  bool have_imp = false;
  // two-impurity network (Sec. III D): 1 = the impurity stands on both sites of the next
  // step's unit cell (merged by that step), 2 = merged nearest-neighbour pair
  int imp_pair = 0;
  bool ising = false;          // the model is Ising (internal energy from the pair)
  double beta = 0.0;
  double *phi = nullptr, *psi = nullptr, *psi_imp = nullptr;  // persistent state
  std::vector<int64_t> dims;                                   // d1..d4, r
  int axes[4] = {0, 1, 2, 3};
  int d = 4;                   // lattice dimension (3 or 4)
  int nsteps = 0;
  double *dscal = nullptr;  // [0] logsum [1] c [2] trace [3] trace2; [8..] dot scratch
  int *dflag = nullptr;
  int q_swap = 4, q_rho = 4, precision = TRG_PREC_FP64;
  int r_bond = 1;              // ILO: re-split and swapped bonds keep r_bond D (Sec. II C)
  bool mixed_now = false;      // this step runs its bulk GEMMs on the tensor cores
  int crit_depth = 0;          // > 0 inside decompositions (QR, re-split, squeezer roots)
  bool crit_fp64 = false;      // route GEMMs inside decompositions to FP64
  unsigned phase_mask = 0xFFu; // phases whose GEMMs may use the tensor cores
  int bulk_cheap = 0;          // > 0: range-finder / impurity products (see gemm())
  // smallest GEMM sides sent to the tensor cores: thin products (max side < 64, e.g. the
  // re-split Grams) and Q R^-1 with a narrow R stay FP64, because a per-column exponent
  // cannot hold the dynamic range of a triangular inverse
  int64_t tc_min_mn = 16, tc_min_max = 64;
  bool cheap_policy = true;    // exact-digit forms use BF16x6 for those products
  // exact-digit forms: the products kept off the bulk digit GEMM (orthonormalisations,
  // squeezer roots, thin products) use the seven-digit FP64-equivalent GEMM, else FP64
  bool x7_policy = true;
  // digit planes of operands that several products of one scope share (PlaneScope)
  struct PlaneEntry {
    const double *ptr;
    int64_t rows, K, ld, stride, batch;
    bool trans;
    int ns;
    OzOperand op;
  };
  std::vector<PlaneEntry> plane_cache;
  bool b_upper = false;        // the next GEMM's right factor is upper triangular (R^-1)
  int ortho = 0;               // > 0: Grams and R^-1 products of an orthonormalisation (FP64)
  int digits_override = 0;     // > 0: digit count of the next digit-form GEMMs
  // digits of the bond swap's compression Grams G^C, G^B in the digit forms (0: the
  // form's own; 64: FP64), for precision studies (study switch swap_gram_digits)
  int swap_gram_digits = 0;
  // learned sketch of the triad-isometry range finders
  SketchNet net;
  int sketch_mode = 0;                      // 0 Gaussian, 1 learned (plain as fallback)
  unsigned long long *d_sketch_cnt = nullptr;  // [0] learned kept, [1] fell back
  float *col_x = nullptr, *col_t = nullptr;    // collected (features, target) rows
  long long col_cap = 0, col_rows = 0, col_dropped = 0;
  uint64_t seed = 0x5EED;
  double last_logc = 0.0, last_gap = INFINITY;
  static constexpr int kPhases = 8;
  cudaEvent_t ev[kPhases + 1] = {};
  double phase_ms[kPhases] = {};
  int phase = 0;
  void mark(int i) {
    phase = i;
    if (!ev[i]) TRG_CUDA(cudaEventCreate(&ev[i]));
    TRG_CUDA(cudaEventRecord(ev[i], stream));
    static const bool dbg = debug_opt("mem");
    if (dbg)
      fprintf(stderr, "phase %d: scratch in use %.2f GB, high water %.2f GB\n", i,
              arena.in_use() / 1073741824.0, arena.high_water() / 1073741824.0);
  }

  // CUDA-event timing of the tensor-core kernel launches inside a step
  struct Timing : TcTiming {
    std::vector<cudaEvent_t> pool;
    struct Rec { int kind; double alg, pipe; };
    std::vector<Rec> rec;
    size_t used = 0;
    void before(cudaStream_t s) override {
      if (pool.size() < 2 * used + 2) {
        for (int i = 0; i < 2; ++i) {
          cudaEvent_t e;
          TRG_CUDA(cudaEventCreate(&e));
          pool.push_back(e);
        }
      }
      TRG_CUDA(cudaEventRecord(pool[2 * used], s));
    }
    void after(cudaStream_t s, int kind, double alg, double pipe) override {
      TRG_CUDA(cudaEventRecord(pool[2 * used + 1], s));
      if (rec.size() <= used) rec.resize(used + 1);
      rec[used] = {kind, alg, pipe};
      ++used;
    }
  } timing;
  // per kind (0 exact-digit GEMM, 1 split-BF16 / 3xTF32 GEMM, 2 seven-digit GEMM): device
  // ms, algorithmic flop (2 M N K, counted once), tensor-pipe flop (every digit / slice
  // product), launches
  double k_ms[3] = {}, k_alg[3] = {}, k_pipe[3] = {};
  int64_t k_launches[3] = {};
  void collect_tc() {  // after a stream synchronise
    for (size_t i = 0; i < timing.used; ++i) {
      float ms = 0.f;
      TRG_CUDA(cudaEventElapsedTime(&ms, timing.pool[2 * i], timing.pool[2 * i + 1]));
      const int k = std::min(std::max(timing.rec[i].kind, 0), 2);
      k_ms[k] += ms;
      k_alg[k] += timing.rec[i].alg;
      k_pipe[k] += timing.rec[i].pipe;
      ++k_launches[k];
    }
    timing.used = 0;
  }

  Tensor alloc(std::vector<int64_t> d) {
    Tensor t;
    t.dims = std::move(d);
    t.p = (double *)arena.alloc(std::max<int64_t>(t.size(), 1) * sizeof(double));
    return t;
  }
  double *scratch() { return dscal + 8; }
};

// the library-global context of trg_init_* / trg_step
Ctx &ctx();

inline Tensor view(double *p, std::vector<int64_t> d) {
  Tensor t;
  t.p = p;
  t.dims = std::move(d);
  return t;
}

// product of d[a .. min(b, size)) (1 for an empty range)
inline int64_t prod(const std::vector<int64_t> &d, size_t a = 0, size_t b = SIZE_MAX) {
  int64_t n = 1;
  const size_t e = std::min(b, d.size());
  for (auto it = d.begin() + (ptrdiff_t)std::min(a, e); it != d.begin() + (ptrdiff_t)e; ++it)
    n *= *it;
  return n;
}


// Where a product runs: the bulk digit GEMM (digits > 0 with on_tc), the split GEMM
// (on_tc, digits 0), the seven-digit FP64-equivalent digit GEMM (on_x7) or FP64 cores.
struct Route {
  bool on_tc = false, on_x7 = false;
  int digits = 0;   // digit count of a digit-GEMM route, 0 otherwise
};

int slices_of(int precision);

bool is_digit_form(int precision);

int digits_of(int precision);

Route route_of(const Ctx &c, int64_t M, int64_t N, int64_t K);

const OzOperand *cached_planes(const Ctx &c, const double *X, int64_t rows, int64_t K,
                                      int64_t ld, int64_t stride, int64_t batch, bool trans,
                                      int ns);

void gemm(Ctx &c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                 const double *A, int64_t lda, int64_t sA, const double *B, int64_t ldb,
                 int64_t sB, double beta, double *C, int64_t ldc, int64_t sC, int64_t batch);

// ------------------------------------------------------------------ GEMM dispatch
struct Cheap {  // marks products that feed only the impurity
  Ctx &c;
  explicit Cheap(Ctx &cc) : c(cc) { if (c.cheap_policy) ++c.bulk_cheap; }
  ~Cheap() { if (c.cheap_policy) --c.bulk_cheap; }
};


struct Crit {  // marks a decomposition: its GEMMs may be routed to FP64
  Ctx &c;
  explicit Crit(Ctx &cc) : c(cc) { ++c.crit_depth; }
  ~Crit() { --c.crit_depth; }
};


struct ArenaScratch : TcScratch {
  Arena &a;
  explicit ArenaScratch(Arena &ar) : a(ar) {}
  void *alloc(size_t bytes) override { return a.alloc(bytes); }
};


// Operands that several products of a scope share are split into digit planes once:
// share() prepares the planes when a product of the given shape would run on a digit
// GEMM, from the arena at the current level (so they live until the enclosing arena mark
// is released), and gemm() finds them by pointer and layout.  The destructor forgets the
// scope's entries.
struct PlaneScope {
  Ctx &c;
  size_t n0;
  explicit PlaneScope(Ctx &cc) : c(cc), n0(cc.plane_cache.size()) {}
  ~PlaneScope() { c.plane_cache.resize(n0); }
  // X as op(A) (as_a) or op(B) of the product op(A) op(B) with sizes M, N, K; t is that
  // side's transpose flag (ta or tb) and ld its leading dimension
  // (a batch of products: `batch` matrices `stride` doubles apart)
  void share(const double *X, bool as_a, bool t, int64_t M, int64_t N, int64_t K, int64_t ld,
             int64_t stride = 0, int64_t batch = 1) {
    const Route rt = route_of(c, M, N, K);
    if (rt.digits == 0) return;
    const int64_t rows = as_a ? M : N;
    const bool trans = as_a ? t : !t;
    if (cached_planes(c, X, rows, K, ld, stride, batch, trans, rt.digits)) return;
    ArenaScratch scr(c.arena);
    OzOperand op = oz_prepare(X, rows, K, ld, stride, trans, batch, rt.digits, scr, c.stream);
    c.plane_cache.push_back({X, rows, K, ld, stride, batch, trans, rt.digits, op});
  }
};


// Grams that feed a Cholesky factor, and the products with its inverse, do not run on the
// bulk digit GEMM: a Gram squares the spectrum, and a digit error of 2^-35 of the largest
// entry would swamp the eigenvalues near the truncation cut (the digit forms run them as
// the seven-digit FP64-equivalent GEMM, the other forms in FP64)
struct Ortho {
  Ctx &c;
  explicit Ortho(Ctx &cc) : c(cc) { ++c.ortho; }
  ~Ortho() { --c.ortho; }
};


// The same shifted CholeskyQR3 with its last pass kept as factors: Y = Q2 R, with Q2 the
// basis after two passes, Ri3 the inverse of the third pass's Cholesky factor and
// R = R3 R2 R1 (each pass Q_{i+1} = Q_i R_i^-1, so Y = Q2 R2 R1 = Q R3 R2 R1).  The
// orthonormal factor is Q = Q2 Ri3; a caller that needs Q W forms Q2 (Ri3 W), which
// saves the third tall product and the product Q^T Y that R would otherwise cost.
struct FoldedQR {
  Tensor Q2, Ri3, R;
};


struct Svd {
  Tensor U, S, V;
};

Tensor copy(Ctx &c, const Tensor &a);

Tensor permuted(Ctx &c, const Tensor &a, const std::vector<int> &perm);

Tensor mm(Ctx &c, const Tensor &A, const Tensor &B, bool ta, bool tb);

Tensor mm_cols(Ctx &c, const Tensor &Q, const Tensor &U, int64_t ncols);

Tensor contract(Ctx &c, const std::string &spec, const Tensor &A, const Tensor &B,
                       Tensor *into = nullptr, double beta_into = 0.0);

void scale_last(Ctx &c, Tensor &t, const double *v, int mode = 0,
                       const double *vmax = nullptr, double tol = 0.0);

Tensor orth_sc(Ctx &c, const Tensor &Y);

std::pair<Tensor, Tensor> orth_qr(Ctx &c, const Tensor &Y);

FoldedQR orth_qr_folded(Ctx &c, const Tensor &Y);

Svd svd_small(Ctx &c, const Tensor &A);

Tensor transpose2(Ctx &c, const Tensor &a);

Tensor identity(Ctx &c, int64_t n);

Tensor range_from(Ctx &c, const Tensor &rho, const Tensor &Om, int q);

Tensor rsvd_sym(Ctx &c, const Tensor &rho, int64_t chi, int q, uint64_t key);

Tensor orth_sc_batched(Ctx &c, const Tensor &Y);

Tensor rsvd_sym_batched(Ctx &c, const Tensor &rho, int64_t chi, int q,
                               const std::vector<uint64_t> &keys);

Tensor range_from_factor(Ctx &c, const Tensor &F, const Tensor &Om, int q);

void share_factor(PlaneScope &ps, const Tensor &F, int64_t chi);

Tensor rsvd_factor(Ctx &c, const Tensor &F, int64_t chi, int q, uint64_t key);

Tensor rsvd_factor_batched(Ctx &c, const Tensor &Fs, int64_t chi, int q,
                                  const std::vector<uint64_t> &keys);

void probe_residual2(Ctx &c, const Tensor &Q, const Tensor &P, double *out);

Tensor range_factor_full(Ctx &c, const Tensor &F, int64_t da, int64_t db, int64_t chi,
                                int q, uint64_t key, uint64_t key_probe);

Tensor gram_root(Ctx &c, const Tensor &rho, int64_t chi, int q, uint64_t key);

std::pair<Tensor, Tensor> squeezer_from_roots(Ctx &c, const Tensor &R1, const Tensor &R2,
                                                     int64_t D, double *gap_out);

std::pair<Tensor, Tensor> squeezer(Ctx &c, const Tensor &rf, const Tensor &rb, int64_t D,
                                          int64_t chi, int q, uint64_t kf, uint64_t kb,
                                          double *gap_out);

Tensor gram_root_batched(Ctx &c, const Tensor &rho, int64_t chi, int q,
                                const std::vector<uint64_t> &keys);

int64_t t_slice(int64_t kt, int64_t per_t_elems);

Tensor contract_upper(Ctx &c, const Tensor &E, const Tensor &F, const Tensor &I_,
                             const Tensor &J_, const Tensor &M2, const Tensor &M3,
                             const Tensor &M4);

Tensor theta_lower(Ctx &c, const Tensor &K_, const Tensor &L_, const Tensor &N2,
                          const Tensor &N3);

Tensor contract_lower(Ctx &c, const Tensor &G, const Tensor &H, const Tensor &K_,
                             const Tensor &L_, const Tensor &N2, const Tensor &N3,
                             const Tensor &N4);

Tensor contract_lower_sum(Ctx &c, const Tensor &G1, const Tensor &H1, const Tensor &G2,
                                 const Tensor &H2, const Tensor &K_, const Tensor &L_,
                                 const Tensor &N2, const Tensor &N3, const Tensor &N4,
                                 double w);

void replace_state(double *&dst, int64_t old_size, const Tensor &src, cudaStream_t s);

void rotate(Ctx &c, int axis);


// run f() in an arena scope and keep only its result (copied into a buffer allocated
// before the scope)
template <class F>
Tensor keep(Ctx &c, const std::vector<int64_t> &dims, F &&f) {
  Tensor out = c.alloc(dims);
  Arena::Mark mk = c.arena.mark();
  Tensor r = f();
  if (r.size() != out.size()) throw Error(TRG_ERR_ARG, "keep: size mismatch");
  TRG_CUDA(cudaMemcpyAsync(out.p, r.p, r.size() * 8, cudaMemcpyDeviceToDevice, c.stream));
  c.arena.release(mk);
  out.dims = r.dims;
  return out;
}


// ------------------------------------------------------------ steps (triad_step.cu)
// one step of the current state along physical `axis` (the 4D or 3D triad step), with
// the error context of the phase that failed
void step_ctx(Ctx &c, int axis, int D, int p);

// ------------------------------------------------------------ contexts (context.cu)
void ensure_ctx(Ctx &c);
void free_state(Ctx &c);
void init_ising_ctx(Ctx &c, double beta, double h, int d = 4);
void init_clock_ctx(Ctx &c, int q, double beta, double h, int d = 4);
void free_energy_ctx(Ctx &c, double *f_per_site, double *lnZ_per_site);
double magnetisation_ctx(Ctx &c);
double gu_wen_ctx(Ctx &c);
void batch_free_all();      // batch.cu
void atrg_free_all();       // atrg.cu

// every C entry point runs its body here: errors become status codes and the message of
// trg_last_error(); success clears it
template <class F>
trg_status guarded(F &&f) {
  try {
    f();
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

}  // namespace trg
