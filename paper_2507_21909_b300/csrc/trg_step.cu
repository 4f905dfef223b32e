// Step orchestration of libtrg and the C ABI (include/trg.h).
//
// One triad-ATRG coarse-graining step (arXiv 2507.21909, Sec. II B and Appendix A) as a
// sequence of device kernels on one stream, with its ILO width (Sec. II C), the one-site
// and pair impurities (Sec. III D), the batched lanes of a coupling sweep, and the plain
// ATRG step of the paper's comparison (eqs. makeG / makeH).  Every tensor contraction is
// planned as (permute) + batched GEMM; the small dense decompositions run in the kernels
// of linalg_small.cu.  Shapes are structural (fixed by D, p and the step history), so
// the host reads back only small diagnostics inside a step (the singular values at the
// cuts, for the gap report) and the final norm and status.
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

static Ctx &ctx() {
  static Ctx c;
  return c;
}
static thread_local std::string g_err = "ok";  // per host thread (batched lanes)
void set_last_error(const std::string &msg) { g_err = msg; }

static Tensor view(double *p, std::vector<int64_t> d) {
  Tensor t;
  t.p = p;
  t.dims = std::move(d);
  return t;
}

static int64_t prod(const std::vector<int64_t> &d, size_t a = 0, size_t b = SIZE_MAX) {
  int64_t n = 1;
  for (size_t i = a; i < std::min(b, d.size()); ++i) n *= d[i];
  return n;
}

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

static int slices_of(int precision) {
  return precision == TRG_PREC_BF16X3 || precision == TRG_PREC_TF32X3 ? 2
         : precision == TRG_PREC_BF16X6                              ? 3
                                                                     : 4;
}
static bool is_digit_form(int precision) {
  return (precision >= TRG_PREC_OZ4 && precision <= TRG_PREC_OZ6) || precision == TRG_PREC_OZ7;
}
static int digits_of(int precision) { return precision == TRG_PREC_OZ7 ? 7 : precision; }

// Where a product runs: the bulk digit GEMM (digits > 0 with on_tc), the split GEMM
// (on_tc, digits 0), the seven-digit FP64-equivalent digit GEMM (on_x7) or FP64 cores.
struct Route {
  bool on_tc = false, on_x7 = false;
  int digits = 0;   // digit count of a digit-GEMM route, 0 otherwise
};
static Route route_of(const Ctx &c, int64_t M, int64_t N, int64_t K) {
  // per-matrix work decides the route, so that batching independent problems does not
  // change how each one is computed
  const double work = (double)M * N * K;
  Route r;
  const bool tc_allowed = c.mixed_now && ((c.phase_mask >> c.phase) & 1u) &&
                          !(c.crit_fp64 && c.crit_depth > 0) && work >= (double)(1 << 22) &&
                          K >= 16;
  r.on_tc = tc_allowed && c.ortho == 0 && std::min(M, N) >= c.tc_min_mn &&
            std::max(M, N) >= c.tc_min_max && !(c.b_upper && N < c.tc_min_max);
  // digit forms: the products the rule above keeps off the bulk digit GEMM (Grams and
  // R^-1 products of orthonormalisations, squeezer Gram roots, thin products) run as the
  // seven-digit FP64-equivalent digit GEMM instead of on the FP64 CUDA cores
  r.on_x7 = !r.on_tc && tc_allowed && c.x7_policy && is_digit_form(c.precision) &&
            std::min(M, N) >= 8;
  // exact-digit forms: products that feed only the impurity (not the free energy) run as
  // 6-term BF16 splits (the bond-swap range finder stays exact: with q_swap = 4 rounds its
  // range depends on the iterates at first order)
  const bool cheap = is_digit_form(c.precision) && c.bulk_cheap > 0 && c.crit_depth == 0;
  if (r.on_x7)
    r.digits = 7;
  else if (r.on_tc && is_digit_form(c.precision) && !cheap)
    r.digits = c.digits_override > 0 ? c.digits_override : digits_of(c.precision);
  return r;
}

static const OzOperand *cached_planes(const Ctx &c, const double *X, int64_t rows, int64_t K,
                                      int64_t ld, int64_t stride, int64_t batch, bool trans,
                                      int ns) {
  for (const auto &e : c.plane_cache)
    if (e.ptr == X && e.rows == rows && e.K == K && e.ld == ld && e.batch == batch &&
        e.trans == trans && e.ns == ns && (batch == 1 || e.stride == stride))
      return &e.op;
  return nullptr;
}

// every GEMM of the step goes through here: in the mixed forms bulk products run on the
// tensor cores (digit or split GEMMs), in the digit forms the decomposition products as
// the seven-digit GEMM; everything else (and every GEMM of the FP64 form) on the FP64
// CUDA cores
static void gemm(Ctx &c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
                 const double *A, int64_t lda, int64_t sA, const double *B, int64_t ldb,
                 int64_t sB, double beta, double *C, int64_t ldc, int64_t sC, int64_t batch) {
  const Route rt = route_of(c, M, N, K);
  static const bool dbg = debug_opt("gemm");
  if (dbg)
    fprintf(stderr,
            "gemm phase %d M %lld N %lld K %lld batch %lld ta %d tb %d crit %d cheap %d ortho %d "
            "route %s digits %d\n",
            c.phase, (long long)M, (long long)N, (long long)K, (long long)batch, (int)ta, (int)tb,
            c.crit_depth, c.bulk_cheap, c.ortho, rt.on_tc ? "tc" : rt.on_x7 ? "x7" : "f64",
            rt.digits);
  if (rt.digits > 0) {
    Arena::Mark mk = c.arena.mark();
    ArenaScratch scr(c.arena);
    const OzOperand *pa = cached_planes(c, A, M, K, lda, sA, batch, ta, rt.digits);
    const OzOperand *pb = cached_planes(c, B, N, K, ldb, sB, batch, !tb, rt.digits);
    gemm_oz(ta, tb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, rt.digits,
            scr, c.stream, &c.timing, pa, pb);
    c.arena.release(mk);
  } else if (rt.on_tc) {
    Arena::Mark mk = c.arena.mark();
    ArenaScratch scr(c.arena);
    const bool cheap = is_digit_form(c.precision);   // an impurity-only product of a digit form
    gemm_tc(ta, tb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch,
            cheap ? 3 : slices_of(c.precision), scr, c.stream, &c.timing,
            !cheap && c.precision == TRG_PREC_TF32X3);
    c.arena.release(mk);
  } else {
    gemm_f64(ta, tb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, c.stream,
             c.b_upper && !tb);
  }
}

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

// ------------------------------------------------------------------ tensor helpers
static Tensor copy(Ctx &c, const Tensor &a) {
  Tensor t = c.alloc(a.dims);
  TRG_CUDA(cudaMemcpyAsync(t.p, a.p, a.size() * sizeof(double), cudaMemcpyDeviceToDevice,
                           c.stream));
  return t;
}

static Tensor permuted(Ctx &c, const Tensor &a, const std::vector<int> &perm) {
  std::vector<int64_t> d(perm.size());
  for (size_t i = 0; i < perm.size(); ++i) d[i] = a.dims[perm[i]];
  Tensor t = c.alloc(d);
  permute(a.p, t.p, a.dims, perm, c.stream);
  return t;
}

// C = op(A) op(B) for 2-D views
static Tensor mm(Ctx &c, const Tensor &A, const Tensor &B, bool ta, bool tb) {
  int64_t M = ta ? A.dims[1] : A.dims[0], K = ta ? A.dims[0] : A.dims[1];
  int64_t Kb = tb ? B.dims[1] : B.dims[0], N = tb ? B.dims[0] : B.dims[1];
  if (K != Kb) throw Error(TRG_ERR_ARG, "mm: inner dimensions differ");
  Tensor C = c.alloc({M, N});
  gemm(c, ta, tb, M, N, K, 1.0, A.p, A.dims[1], 0, B.p, B.dims[1], 0, 0.0, C.p, N, 0, 1);
  return C;
}

// first `ncols` columns of U (rows x ucols) applied from the right: C = Q U[:, :ncols]
static Tensor mm_cols(Ctx &c, const Tensor &Q, const Tensor &U, int64_t ncols) {
  int64_t M = Q.dims[0], K = Q.dims[1];
  Tensor C = c.alloc({M, ncols});
  gemm(c, false, false, M, ncols, K, 1.0, Q.p, K, 0, U.p, U.dims[1], 0, 0.0, C.p, ncols, 0, 1);
  return C;
}

// einsum-style contraction of two tensors (every index appears in exactly two of the
// three index strings): batch = in all three, M = A and out, N = B and out, K = A and B.
// With `into`, the result goes to that buffer: written (beta_into = 0, any output order)
// or accumulated as *into = result + beta_into * *into (then the output order must be
// the GEMM's natural one, batch + M + N indices).
static Tensor contract(Ctx &c, const std::string &spec, const Tensor &A, const Tensor &B,
                       Tensor *into = nullptr, double beta_into = 0.0) {
  size_t comma = spec.find(','), arrow = spec.find("->");
  std::string sa = spec.substr(0, comma), sb = spec.substr(comma + 1, arrow - comma - 1),
              so = spec.substr(arrow + 2);
  if ((int)sa.size() != (int)A.dims.size() || (int)sb.size() != (int)B.dims.size())
    throw Error(TRG_ERR_ARG, "contract: rank mismatch in " + spec);
  std::map<char, int64_t> dim;
  for (size_t i = 0; i < sa.size(); ++i) dim[sa[i]] = A.dims[i];
  for (size_t i = 0; i < sb.size(); ++i) {
    auto it = dim.find(sb[i]);
    if (it != dim.end() && it->second != B.dims[i])
      throw Error(TRG_ERR_ARG, "contract: dimension mismatch in " + spec);
    dim[sb[i]] = B.dims[i];
  }
  auto has = [](const std::string &s, char ch) { return s.find(ch) != std::string::npos; };
  std::string bt, Mi, Ni, Ki;
  for (char ch : so) {
    if (has(sa, ch) && has(sb, ch)) bt += ch;
    else if (has(sa, ch)) Mi += ch;
    else if (has(sb, ch)) Ni += ch;
    else throw Error(TRG_ERR_ARG, "contract: free output index in " + spec);
  }
  for (char ch : sa) {
    if (has(sb, ch) && !has(so, ch)) Ki += ch;
    if (!has(sb, ch) && !has(so, ch)) throw Error(TRG_ERR_ARG, "contract: lone index " + spec);
  }
  for (char ch : sb)
    if (!has(sa, ch) && !has(so, ch)) throw Error(TRG_ERR_ARG, "contract: lone index " + spec);
  auto pd = [&](const std::string &s) {
    int64_t n = 1;
    for (char ch : s) n *= dim[ch];
    return n;
  };
  auto arrange = [&](const Tensor &T, const std::string &s, const std::string &want) {
    std::vector<int> perm;
    for (char ch : want) perm.push_back((int)s.find(ch));
    return permuted(c, T, perm);
  };
  std::vector<int64_t> odims;
  for (char ch : so) odims.push_back(dim[ch]);
  if (into && (into->dims != odims || (beta_into != 0.0 && so != bt + Mi + Ni)))
    throw Error(TRG_ERR_ARG, "contract: accumulation needs the natural output order in " + spec);
  Tensor out = into ? *into : c.alloc(odims);
  Arena::Mark mk = c.arena.mark();
  bool ta = false, tb = false;
  const double *pa, *pb;
  Tensor tA, tB;
  if (sa == bt + Mi + Ki) pa = A.p;
  else if (sa == bt + Ki + Mi) { pa = A.p; ta = true; }
  else { tA = arrange(A, sa, bt + Mi + Ki); pa = tA.p; }
  if (sb == bt + Ki + Ni) pb = B.p;
  else if (sb == bt + Ni + Ki) { pb = B.p; tb = true; }
  else { tB = arrange(B, sb, bt + Ki + Ni); pb = tB.p; }
  int64_t nb = pd(bt), M = pd(Mi), N = pd(Ni), K = pd(Ki);
  std::string nat = bt + Mi + Ni;
  std::vector<int64_t> ndims;
  for (char ch : nat) ndims.push_back(dim[ch]);
  Tensor C = (so == nat) ? out : c.alloc(ndims);
  gemm(c, ta, tb, M, N, K, 1.0, pa, ta ? M : K, M * K, pb, tb ? K : N, K * N,
       into ? beta_into : 0.0, C.p, N, M * N, nb);
  if (so != nat) {
    std::vector<int> perm;
    for (char ch : so) perm.push_back((int)nat.find(ch));
    permute(C.p, out.p, C.dims, perm, c.stream);
  }
  c.arena.release(mk);
  return out;
}

// run f() in an arena scope and keep only its result (copied into a buffer allocated
// before the scope)
template <class F>
static Tensor keep(Ctx &c, const std::vector<int64_t> &dims, F &&f) {
  Tensor out = c.alloc(dims);
  Arena::Mark mk = c.arena.mark();
  Tensor r = f();
  if (r.size() != out.size()) throw Error(TRG_ERR_ARG, "keep: size mismatch");
  TRG_CUDA(cudaMemcpyAsync(out.p, r.p, r.size() * 8, cudaMemcpyDeviceToDevice, c.stream));
  c.arena.release(mk);
  out.dims = r.dims;
  return out;
}

static void scale_last(Ctx &c, Tensor &t, const double *v, int mode = 0,
                       const double *vmax = nullptr, double tol = 0.0) {
  int64_t n = t.dims.back();
  scale_axis(t.p, t.size(), 1, n, v, mode, vmax, tol, c.stream);
}

// ------------------------------------------------------------- decompositions
// Orthonormal basis of range(Y) (n x w) by shifted CholeskyQR3 (Fukaya et al. 2020):
// each pass Q <- Q R^{-1} keeps the span, so the span error stays O(eps * cond(Y)) like
// Householder QR; directions at the rounding level come out as zero columns.
static Tensor orth_sc(Ctx &c, const Tensor &Y) {
  Ortho og(c);
  int64_t w = Y.dims[1];
  Tensor out = c.alloc(Y.dims);
  Arena::Mark mk = c.arena.mark();
  Tensor Q = Y;
  for (int pass = 0; pass < 3; ++pass) {
    Tensor G = mm(c, Q, Q, true, false);
    Tensor R = c.alloc({w, w}), Ri = c.alloc({w, w});
    chol_rinv(G.p, R.p, Ri.p, (int)w, 1, pass == 0 ? 0.0 : kPivotTol,
              pass == 0 ? kShiftRel : 0.0, c.stream);
    c.b_upper = true;
    if (pass == 2) {
      gemm(c, false, false, Q.dims[0], w, w, 1.0, Q.p, w, 0, Ri.p, w, 0, 0.0, out.p, w, 0, 1);
    } else {
      Q = mm(c, Q, Ri, false, false);
    }
    c.b_upper = false;
  }
  c.arena.release(mk);
  return out;
}

static std::pair<Tensor, Tensor> orth_qr(Ctx &c, const Tensor &Y) {
  Crit cr(c);
  Tensor Q = orth_sc(c, Y);
  Tensor R = mm(c, Q, Y, true, false);
  return {Q, R};
}

// The same shifted CholeskyQR3 with its last pass kept as factors: Y = Q2 R, with Q2 the
// basis after two passes, Ri3 the inverse of the third pass's Cholesky factor and
// R = R3 R2 R1 (each pass Q_{i+1} = Q_i R_i^-1, so Y = Q2 R2 R1 = Q R3 R2 R1).  The
// orthonormal factor is Q = Q2 Ri3; a caller that needs Q W forms Q2 (Ri3 W), which
// saves the third tall product and the product Q^T Y that R would otherwise cost.
struct FoldedQR {
  Tensor Q2, Ri3, R;
};
static FoldedQR orth_qr_folded(Ctx &c, const Tensor &Y) {
  Crit cr(c);
  Ortho og(c);
  const int64_t n = Y.dims[0], w = Y.dims[1];
  FoldedQR f;
  f.Q2 = c.alloc(Y.dims);
  f.Ri3 = c.alloc({w, w});
  f.R = c.alloc({w, w});
  Arena::Mark mk = c.arena.mark();
  Tensor Q = Y;
  Tensor Rp[3];
  for (int pass = 0; pass < 3; ++pass) {
    Tensor G = mm(c, Q, Q, true, false);
    Rp[pass] = c.alloc({w, w});
    Tensor Ri = pass == 2 ? f.Ri3 : c.alloc({w, w});
    chol_rinv(G.p, Rp[pass].p, Ri.p, (int)w, 1, pass == 0 ? 0.0 : kPivotTol,
              pass == 0 ? kShiftRel : 0.0, c.stream);
    if (pass < 2) {
      Tensor Qn = pass == 1 ? f.Q2 : c.alloc(Y.dims);
      c.b_upper = true;
      gemm(c, false, false, n, w, w, 1.0, Q.p, w, 0, Ri.p, w, 0, 0.0, Qn.p, w, 0, 1);
      c.b_upper = false;
      Q = Qn;
    }
  }
  Tensor R32 = mm(c, Rp[2], Rp[1], false, false);
  gemm(c, false, false, w, w, w, 1.0, R32.p, w, 0, Rp[0].p, w, 0, 0.0, f.R.p, w, 0, 1);
  c.arena.release(mk);
  return f;
}

struct Svd {
  Tensor U, S, V;
};
static Svd svd_small(Ctx &c, const Tensor &A) {
  int64_t m = A.dims[0], n = A.dims[1];
  Svd r;
  r.U = c.alloc({m, n});
  r.S = c.alloc({n});
  r.V = c.alloc({n, n});
  Tensor work = c.alloc({(int64_t)svd_jacobi_work((int)m, (int)n, 1) + 1});
  static const bool dbg = debug_opt("svd");
  int *info = dbg ? reinterpret_cast<int *>(work.p + work.size() - 1) : nullptr;
  svd_jacobi(A.p, (int)m, (int)n, r.U.p, r.S.p, r.V.p, 1, work.p, info, c.stream);
  if (dbg) {
    int sweeps = 0;
    TRG_CUDA(cudaMemcpyAsync(&sweeps, info, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    TRG_CUDA(cudaStreamSynchronize(c.stream));
    fprintf(stderr, "svd_jacobi %lld x %lld: %d sweeps\n", (long long)m, (long long)n, sweeps);
  }
  return r;
}

static Tensor transpose2(Ctx &c, const Tensor &a) { return permuted(c, a, {1, 0}); }

static Tensor identity(Ctx &c, int64_t n) {
  Tensor t = c.alloc({n, n});
  fill_identity(t.p, n, n, c.stream);
  return t;
}

// orthonormal basis of range(rho^(q+1) Omega)
static Tensor range_from(Ctx &c, const Tensor &rho, const Tensor &Om, int q) {
  Tensor Q = orth_sc(c, mm(c, rho, Om, false, false));
  for (int i = 0; i < q; ++i) Q = orth_sc(c, mm(c, rho, Q, false, false));
  return Q;
}

// orthonormal basis (n x chi) of range(rho^(q+1) Omega), or the identity if chi >= n
static Tensor rsvd_sym(Ctx &c, const Tensor &rho, int64_t chi, int q, uint64_t key) {
  int64_t n = rho.dims[0];
  if (chi >= n) return identity(c, n);
  Tensor Om = c.alloc({n, chi});
  fill_gaussian(Om.p, n, chi, key, c.stream);
  return range_from(c, rho, Om, q);
}

// nb independent shifted CholeskyQR3 (as orth_sc) on stacked Y [nb][rows][w]: every
// Gram, Cholesky and product of a pass is one batched launch
static Tensor orth_sc_batched(Ctx &c, const Tensor &Y) {
  Ortho og(c);
  const int64_t nb = Y.dims[0], rows = Y.dims[1], w = Y.dims[2];
  Tensor out = c.alloc(Y.dims);
  Arena::Mark mk = c.arena.mark();
  Tensor Q = Y;
  for (int pass = 0; pass < 3; ++pass) {
    Tensor G = c.alloc({nb, w, w}), R = c.alloc({nb, w, w}), Ri = c.alloc({nb, w, w});
    gemm(c, true, false, w, w, rows, 1.0, Q.p, w, rows * w, Q.p, w, rows * w, 0.0, G.p, w, w * w,
         nb);
    chol_rinv(G.p, R.p, Ri.p, (int)w, (int)nb, pass == 0 ? 0.0 : kPivotTol,
              pass == 0 ? kShiftRel : 0.0, c.stream);
    Tensor Qn = pass == 2 ? out : c.alloc({nb, rows, w});
    c.b_upper = true;
    gemm(c, false, false, rows, w, w, 1.0, Q.p, w, rows * w, Ri.p, w, w * w, 0.0, Qn.p, w,
         rows * w, nb);
    c.b_upper = false;
    Q = Qn;
  }
  c.arena.release(mk);
  return out;
}

// nb range finders (as rsvd_sym, chi < n) on stacked symmetric rho [nb][n][n]
static Tensor rsvd_sym_batched(Ctx &c, const Tensor &rho, int64_t chi, int q,
                               const std::vector<uint64_t> &keys) {
  const int64_t nb = rho.dims[0], n = rho.dims[1];
  Tensor out = c.alloc({nb, n, chi});
  Arena::Mark mk = c.arena.mark();
  Tensor Om = c.alloc({nb, n, chi});
  for (int64_t b = 0; b < nb; ++b) fill_gaussian(Om.p + b * n * chi, n, chi, keys[b], c.stream);
  auto apply = [&](const Tensor &V) {
    Tensor Yb = c.alloc({nb, n, chi});
    gemm(c, false, false, n, chi, n, 1.0, rho.p, n, n * n, V.p, chi, n * chi, 0.0, Yb.p, chi,
         n * chi, nb);
    return Yb;
  };
  Tensor Q = orth_sc_batched(c, apply(Om));
  for (int i = 0; i < q; ++i) Q = orth_sc_batched(c, apply(Q));
  TRG_CUDA(cudaMemcpyAsync(out.p, Q.p, out.size() * 8, cudaMemcpyDeviceToDevice, c.stream));
  c.arena.release(mk);
  return out;
}

// Range finder of rho = F F^T from the factor F (n x m) alone: range((F F^T)^(q+1) Omega)
// = range(F (F^T F)^q F^T Omega), the same sketch and the same subspace as on rho, but
// every product is with F, whose spectrum is the square root of rho's, so the digit
// forms keep the eigenvalues near the cut (forming rho would square the spectrum).
static Tensor range_from_factor(Ctx &c, const Tensor &F, const Tensor &Om, int q) {
  auto apply = [&](const Tensor &V) {
    Tensor Z = mm(c, F, V, true, false);          // F^T V   (m x chi)
    return mm(c, F, Z, false, false);             // F F^T V (n x chi)
  };
  Tensor Q = orth_sc(c, apply(Om));
  for (int i = 0; i < q; ++i) Q = orth_sc(c, apply(Q));
  return Q;
}

// F's digit planes for both products of the range finder (F^T V and F Z), split once
static void share_factor(PlaneScope &ps, const Tensor &F, int64_t chi) {
  const int64_t n = F.dims[0], m = F.dims[1];
  ps.share(F.p, true, true, m, chi, n, m);    // F^T V: op(A) = F^T (m x n)
  ps.share(F.p, true, false, n, chi, m, m);   // F Z:   op(A) = F   (n x m)
}

static Tensor rsvd_factor(Ctx &c, const Tensor &F, int64_t chi, int q, uint64_t key) {
  const int64_t n = F.dims[0];
  Tensor out = c.alloc({n, chi});
  Arena::Mark mk = c.arena.mark();
  PlaneScope ps(c);
  share_factor(ps, F, chi);
  Tensor Om = c.alloc({n, chi});
  fill_gaussian(Om.p, n, chi, key, c.stream);
  Tensor Q = range_from_factor(c, F, Om, q);
  TRG_CUDA(cudaMemcpyAsync(out.p, Q.p, out.size() * 8, cudaMemcpyDeviceToDevice, c.stream));
  c.arena.release(mk);
  return out;
}

// nb range finders of rho_i = F_i F_i^T at once (every F_i n x m, stacked [nb][n][m]):
// the sketches and subspaces of rsvd_factor on each, with every product, Gram and
// Cholesky of a power round one batched launch and the F_i split into digit planes once
static Tensor rsvd_factor_batched(Ctx &c, const Tensor &Fs, int64_t chi, int q,
                                  const std::vector<uint64_t> &keys) {
  const int64_t nb = Fs.dims[0], n = Fs.dims[1], m = Fs.dims[2];
  Tensor out = c.alloc({nb, n, chi});
  Arena::Mark mk = c.arena.mark();
  PlaneScope ps(c);
  ps.share(Fs.p, true, true, m, chi, n, m, n * m, nb);    // F^T V: op(A) = F^T (m x n)
  ps.share(Fs.p, true, false, n, chi, m, m, n * m, nb);   // F Z:   op(A) = F   (n x m)
  Tensor Om = c.alloc({nb, n, chi});
  for (int64_t b = 0; b < nb; ++b) fill_gaussian(Om.p + b * n * chi, n, chi, keys[b], c.stream);
  auto apply = [&](const Tensor &V) {
    Tensor Z = c.alloc({nb, m, chi}), Y = c.alloc({nb, n, chi});
    gemm(c, true, false, m, chi, n, 1.0, Fs.p, m, n * m, V.p, chi, n * chi, 0.0, Z.p, chi,
         m * chi, nb);
    gemm(c, false, false, n, chi, m, 1.0, Fs.p, m, n * m, Z.p, chi, m * chi, 0.0, Y.p, chi,
         n * chi, nb);
    return Y;
  };
  Tensor Q = orth_sc_batched(c, apply(Om));
  for (int i = 0; i < q; ++i) Q = orth_sc_batched(c, apply(Q));
  TRG_CUDA(cudaMemcpyAsync(out.p, Q.p, out.size() * 8, cudaMemcpyDeviceToDevice, c.stream));
  c.arena.release(mk);
  return out;
}

// squared probe residual ||P - Q Q^T P||_F^2 into *out (device)
static void probe_residual2(Ctx &c, const Tensor &Q, const Tensor &P, double *out) {
  Arena::Mark mk = c.arena.mark();
  Tensor T = mm(c, Q, P, true, false);
  Tensor E = copy(c, P);
  gemm(c, false, false, Q.dims[0], P.dims[1], Q.dims[1], -1.0, Q.p, Q.dims[1], 0, T.p,
       P.dims[1], 0, 1.0, E.p, P.dims[1], 0, 1);
  Tensor scratch = c.alloc({1024});
  dot(E.p, E.p, E.size(), out, scratch.p, c.stream);
  c.arena.release(mk);
}

// Range of a triad Gram rho = F F^T over legs (da, db), from its factor F (n x m).
// Plain form: the Gaussian sketch.  Learned form: the same Gaussian with rows rescaled by
// the sketch network, kept unless its probe residual exceeds 1.5x the plain range's
// (then the plain range).  With collection on, the (features, leverage target) rows of
// both legs are appended from the plain range.  diag(rho) = row norms^2 of F, and the
// probes rho P = F (F^T P).
static Tensor range_factor_full(Ctx &c, const Tensor &F, int64_t da, int64_t db, int64_t chi,
                                int q, uint64_t key, uint64_t key_probe) {
  const int64_t n = F.dims[0], m = F.dims[1];
  if (chi >= n) return identity(c, n);
  const bool learned = c.sketch_mode == 1 && c.net.loaded;
  const bool collect = c.col_cap > 0;
  if (!learned && !collect) return rsvd_factor(c, F, chi, q, key);
  cudaStream_t s = c.stream;
  Tensor out = c.alloc({n, chi});
  Arena::Mark mk = c.arena.mark();
  PlaneScope ps(c);
  share_factor(ps, F, chi);
  Tensor G = c.alloc({n, chi});
  fill_gaussian(G.p, n, chi, key, s);
  Tensor Qp = range_from_factor(c, F, G, q);
  Tensor Fe = c.alloc({(da + db) * kMlpIn / 2 + 1});   // (da + db) x 5 floats
  Tensor dg = c.alloc({n});
  sketch_features_factor(F.p, m, (int)da, (int)db, (int)chi, dg.p,
                         reinterpret_cast<float *>(Fe.p), s);
  if (collect) {
    const long long r = da + db;
    if (c.col_rows + r <= c.col_cap) {
      TRG_CUDA(cudaMemcpyAsync(c.col_x + c.col_rows * kMlpIn, Fe.p, r * kMlpIn * sizeof(float),
                               cudaMemcpyDeviceToDevice, s));
      leverage_targets(Qp.p, (int)da, (int)db, (int)chi, c.col_t + c.col_rows, s);
      c.col_rows += r;
    } else {
      c.col_dropped += r;
    }
  }
  if (!learned) {
    TRG_CUDA(cudaMemcpyAsync(out.p, Qp.p, out.size() * 8, cudaMemcpyDeviceToDevice, s));
    c.arena.release(mk);
    return out;
  }
  Tensor U = c.alloc({(da + db) / 2 + 1});                 // da + db floats
  float *u = reinterpret_cast<float *>(U.p);
  mlp_forward(c.net, reinterpret_cast<const float *>(Fe.p), da + db, u, true, s);
  Tensor w = c.alloc({n});
  sketch_row_weights(u, (int)da, (int)db, w.p, s);
  scale_rows(G.p, n, chi, w.p, s);
  Tensor Ql = range_from_factor(c, F, G, q);
  Tensor P0 = c.alloc({n, 8});
  fill_gaussian(P0.p, n, 8, key_probe, s);
  Tensor P = mm(c, F, mm(c, F, P0, true, false), false, false);
  Tensor r2 = c.alloc({2});
  probe_residual2(c, Ql, P, r2.p);
  probe_residual2(c, Qp, P, r2.p + 1);
  select_range(Ql.p, Qp.p, out.size(), r2.p, r2.p + 1, 1.5 * 1.5, out.p, c.d_sketch_cnt, s);
  c.arena.release(mk);
  return out;
}

// R (c' x n) with R^T R = Q Q^T rho Q Q^T, Q the rank-chi range of rho.  R = L Q^T with
// L the upper Cholesky factor of Q^T rho Q (dead pivots give zero rows); any square root
// serves, since the squeezer only uses the singular triplets of R1 R2^T, which are
// invariant under R -> O R.
static Tensor gram_root(Ctx &c, const Tensor &rho, int64_t chi, int q, uint64_t key) {
  Crit cr(c);
  Ortho og(c);   // all FP64: rho's range near the cut is what the squeezer keeps
  Tensor Q = rsvd_sym(c, rho, chi, q, key);
  Tensor Bm = mm(c, Q, mm(c, rho, Q, false, false), true, false);
  const int64_t cc = Bm.dims[0];
  Tensor L = c.alloc({cc, cc}), Li = c.alloc({cc, cc});
  chol_rinv(Bm.p, L.p, Li.p, (int)cc, 1, kPivotTol, 0.0, c.stream);
  return mm(c, L, Q, false, true);                  // c' x n
}

// oblique squeezer pair from the Gram roots R1 (forward) and R2 (backward), chi x n each
static std::pair<Tensor, Tensor> squeezer_from_roots(Ctx &c, const Tensor &R1, const Tensor &R2,
                                                     int64_t D, double *gap_out) {
  const int64_t n = R1.dims[1];
  Crit cr(c);
  Ortho og(c);
  Tensor K = mm(c, R1, R2, false, true);
  Svd sv = svd_small(c, K);
  int64_t k = std::min<int64_t>(D, K.dims[1]);
  Tensor M = mm_cols(c, transpose2(c, R2), sv.V, k);
  Tensor N = mm_cols(c, transpose2(c, R1), sv.U, k);
  scale_axis(M.p, M.size(), 1, k, sv.S.p, 2, sv.S.p, kRankTol, c.stream);
  scale_axis(N.p, N.size(), 1, k, sv.S.p, 2, sv.S.p, kRankTol, c.stream);
  sign_gauge(M.p, n, N.p, n, k, c.stream);
  // relative gap at the cut, for diagnostics
  std::vector<double> hs(K.dims[1]);
  TRG_CUDA(cudaMemcpyAsync(hs.data(), sv.S.p, hs.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, c.stream));
  TRG_CUDA(cudaStreamSynchronize(c.stream));
  *gap_out = ((int64_t)hs.size() > k && hs[k - 1] > 0) ? (hs[k - 1] - hs[k]) / hs[k - 1]
                                                        : INFINITY;
  return {M, N};
}

// oblique squeezer pair on one pair bond: M (n x k) on the forward side, N on the backward
static std::pair<Tensor, Tensor> squeezer(Ctx &c, const Tensor &rf, const Tensor &rb, int64_t D,
                                          int64_t chi, int q, uint64_t kf, uint64_t kb,
                                          double *gap_out) {
  int64_t n = rf.dims[0];
  if (n <= D) {
    *gap_out = INFINITY;
    return {identity(c, n), identity(c, n)};
  }
  Crit cr(c);
  Tensor R1 = gram_root(c, rf, chi, q, kf), R2 = gram_root(c, rb, chi, q, kb);
  return squeezer_from_roots(c, R1, R2, D, gap_out);
}

// gram_root of nb Grams of one shape (stacked [nb][n][n], chi < n) as one batch:
// R[b] = L_b Q_b^T, stacked [nb][chi][n]
static Tensor gram_root_batched(Ctx &c, const Tensor &rho, int64_t chi, int q,
                                const std::vector<uint64_t> &keys) {
  Crit cr(c);
  Ortho og(c);   // all FP64, as gram_root
  const int64_t nb = rho.dims[0], n = rho.dims[1];
  Tensor R = c.alloc({nb, chi, n});
  Arena::Mark mk = c.arena.mark();
  Tensor Q = rsvd_sym_batched(c, rho, chi, q, keys);
  Tensor T = c.alloc({nb, n, chi}), Bm = c.alloc({nb, chi, chi});
  gemm(c, false, false, n, chi, n, 1.0, rho.p, n, n * n, Q.p, chi, n * chi, 0.0, T.p, chi,
       n * chi, nb);
  gemm(c, true, false, chi, chi, n, 1.0, Q.p, chi, n * chi, T.p, chi, n * chi, 0.0, Bm.p, chi,
       chi * chi, nb);
  Tensor L = c.alloc({nb, chi, chi}), Li = c.alloc({nb, chi, chi});
  chol_rinv(Bm.p, L.p, Li.p, (int)chi, (int)nb, kPivotTol, 0.0, c.stream);
  gemm(c, false, true, chi, n, chi, 1.0, L.p, chi, chi * chi, Q.p, chi, n * chi, 0.0, R.p, n,
       chi * n, nb);
  c.arena.release(mk);
  return R;
}

// Rows of t (the first leg, i1 of the paper's Table I) per slice of the coarse
// contraction, so that the intermediate Phi1 (t kA k4 kX g) of one slice stays below
// `budget` bytes (default 1 GiB; the study switch slice_mb overrides it, for tests).  The slices
// are independent GEMM chains; their outputs are disjoint rows of Phi / Psi.
static int64_t t_slice(int64_t kt, int64_t per_t_elems) {
  int64_t budget = int64_t(1) << 30;
  const std::string e = study_opt("slice_mb");
  if (!e.empty()) budget = std::max<int64_t>(1, atoll(e.c_str())) << 20;
  const int64_t per_t = std::max<int64_t>(per_t_elems * (int64_t)sizeof(double), 1);
  return std::max<int64_t>(1, std::min<int64_t>(kt, budget / per_t));
}

// Phi[t,k2,k3,k4,g] = sum (E F M4)(I J M2 M3)   (eq. makeMG), sliced over t.  Operands
// that every slice reuses are put in GEMM order once (F as (al q4 | kX g)); each slice's
// EM comes out in GEMM order, and its result is permuted straight into Phi's rows.
static Tensor contract_upper(Ctx &c, const Tensor &E, const Tensor &F, const Tensor &I_,
                             const Tensor &J_, const Tensor &M2, const Tensor &M3,
                             const Tensor &M4) {
  const int64_t kt = E.dims[0], kr = F.dims[3];
  Tensor out = c.alloc({kt, M2.dims[2], M3.dims[2], M4.dims[2], kr});
  const int64_t out_t = out.size() / kt, e_t = E.size() / kt;
  Arena::Mark mk = c.arena.mark();
  // Theta = (I M2)(J M3) over the inner legs (b, B) pairs: intermediates stay D^3 chi
  // (the order (I M2 J) M3 would hold D^3 chi^2)
  Tensor IM2 = contract(c, "bck,bBm->ckBm", I_, M2);              // (c kA B k2)
  Tensor JM3 = contract(c, "BCl,cCn->Blcn", J_, M3);              // (B kX c k3)
  Tensor Theta = contract(c, "ckBm,Blcn->klmn", IM2, JM3);        // (kA kX k2 k3)
  Tensor Fg = permuted(c, F, {0, 2, 1, 3});                       // (al q4 kX g)
  const int64_t ts = t_slice(kt, E.dims[1] * M4.dims[2] * F.dims[1] * kr);
  // every slice reuses F and Theta as B operands: their digit planes are split once
  PlaneScope ps(c);
  {
    const int64_t kA = E.dims[1], k4 = M4.dims[2], kX = F.dims[1];
    const int64_t alq = F.dims[0] * F.dims[2];
    ps.share(Fg.p, false, false, ts * kA * k4, kX * kr, alq, kX * kr);
    ps.share(Theta.p, false, false, ts * k4 * kr, Theta.dims[2] * Theta.dims[3], kA * kX,
             Theta.dims[2] * Theta.dims[3]);
  }
  for (int64_t t0 = 0; t0 < kt; t0 += ts) {
    const int64_t tn = std::min(ts, kt - t0);
    Arena::Mark ms = c.arena.mark();
    Tensor Es = view(E.p + t0 * e_t, {tn, E.dims[1], E.dims[2], E.dims[3]});
    Tensor EM = contract(c, "tkda,dDm->tkmaD", Es, M4);           // (t kA k4 al q4)
    Tensor Phi1 = contract(c, "tkmaD,aDlg->tkmlg", EM, Fg);       // (t kA k4 kX g)
    Tensor dst = view(out.p + t0 * out_t, {tn, out.dims[1], out.dims[2], out.dims[3], kr});
    contract(c, "tkmlg,klKL->tKLmg", Phi1, Theta, &dst);          // (t k2 k3 k4 g)
    c.arena.release(ms);
  }
  c.arena.release(mk);
  return out;
}

// Theta of the lower block in the order (kD kY k2' k3') that the slices' GEMMs read
static Tensor theta_lower(Ctx &c, const Tensor &K_, const Tensor &L_, const Tensor &N2,
                          const Tensor &N3) {
  Tensor KN2 = contract(c, "bck,bBm->ckBm", K_, N2);              // (c kY B k2)
  Tensor LN3 = contract(c, "BCl,cCn->Blcn", L_, N3);              // (B kD c k3)
  return contract(c, "ckBm,Blcn->lkmn", KN2, LN3);                // (kD kY k2 k3)
}

// Psi (eq. makeMH), sliced over its first leg w
static Tensor contract_lower(Ctx &c, const Tensor &G, const Tensor &H, const Tensor &K_,
                             const Tensor &L_, const Tensor &N2, const Tensor &N3,
                             const Tensor &N4) {
  const int64_t kt = H.dims[0], kr = G.dims[3];
  Tensor out = c.alloc({kt, N2.dims[2], N3.dims[2], N4.dims[2], kr});
  const int64_t out_t = out.size() / kt, h_t = H.size() / kt;
  Arena::Mark mk = c.arena.mark();
  Tensor ThetaT = theta_lower(c, K_, L_, N2, N3);                 // (kD kY k2 k3)
  Tensor Gg = permuted(c, G, {0, 2, 1, 3});                       // (be P4 kY g)
  const int64_t ts = t_slice(kt, H.dims[1] * N4.dims[2] * G.dims[1] * kr);
  PlaneScope ps(c);
  {
    const int64_t kD = H.dims[1], k4 = N4.dims[2], kY = G.dims[1];
    const int64_t beq = G.dims[0] * G.dims[2];
    ps.share(Gg.p, false, false, ts * kD * k4, kY * kr, beq, kY * kr);
    ps.share(ThetaT.p, false, false, ts * k4 * kr, ThetaT.dims[2] * ThetaT.dims[3], kD * kY,
             ThetaT.dims[2] * ThetaT.dims[3]);
  }
  for (int64_t t0 = 0; t0 < kt; t0 += ts) {
    const int64_t tn = std::min(ts, kt - t0);
    Arena::Mark ms = c.arena.mark();
    Tensor Hs = view(H.p + t0 * h_t, {tn, H.dims[1], H.dims[2], H.dims[3]});
    Tensor HN = contract(c, "wkdb,Ddm->wkmbD", Hs, N4);           // (w kD k4 be P4)
    Tensor Psi1 = contract(c, "wkmbD,bDjg->wkmjg", HN, Gg);       // (w kD k4 kY g)
    Tensor dst = view(out.p + t0 * out_t, {tn, out.dims[1], out.dims[2], out.dims[3], kr});
    contract(c, "wkmjg,kjKL->wKLmg", Psi1, ThetaT, &dst);         // (w k2 k3 k4 g)
    c.arena.release(ms);
  }
  c.arena.release(mk);
  return out;
}

// w (Psi(G1, H1) + Psi(G2, H2)) in one pass (eq. makeMH is linear in each of G and H):
// per slice the two first contractions accumulate into one Psi1, so the second
// contraction with Theta (the larger GEMM of the chain) runs once
static Tensor contract_lower_sum(Ctx &c, const Tensor &G1, const Tensor &H1, const Tensor &G2,
                                 const Tensor &H2, const Tensor &K_, const Tensor &L_,
                                 const Tensor &N2, const Tensor &N3, const Tensor &N4,
                                 double w) {
  const int64_t kt = H1.dims[0], kr = G1.dims[3];
  Tensor out = c.alloc({kt, N2.dims[2], N3.dims[2], N4.dims[2], kr});
  const int64_t out_t = out.size() / kt, h_t = H1.size() / kt;
  Arena::Mark mk = c.arena.mark();
  Tensor ThetaT = theta_lower(c, K_, L_, N2, N3);                 // (kD kY k2 k3)
  axpby(ThetaT.p, ThetaT.p, w, 0.0, ThetaT.size(), c.stream);     // w folded into Theta
  Tensor G1g = permuted(c, G1, {0, 2, 1, 3}), G2g = permuted(c, G2, {0, 2, 1, 3});
  const int64_t ts = t_slice(kt, H1.dims[1] * N4.dims[2] * G1.dims[1] * kr);
  for (int64_t t0 = 0; t0 < kt; t0 += ts) {
    const int64_t tn = std::min(ts, kt - t0);
    Arena::Mark ms = c.arena.mark();
    Tensor H1s = view(H1.p + t0 * h_t, {tn, H1.dims[1], H1.dims[2], H1.dims[3]});
    Tensor H2s = view(H2.p + t0 * h_t, {tn, H2.dims[1], H2.dims[2], H2.dims[3]});
    Tensor Psi1 = contract(c, "wkmbD,bDjg->wkmjg", contract(c, "wkdb,Ddm->wkmbD", H1s, N4), G1g);
    {
      Arena::Mark m2 = c.arena.mark();
      contract(c, "wkmbD,bDjg->wkmjg", contract(c, "wkdb,Ddm->wkmbD", H2s, N4), G2g, &Psi1,
               1.0);
      c.arena.release(m2);
    }
    Tensor dst = view(out.p + t0 * out_t, {tn, out.dims[1], out.dims[2], out.dims[3], kr});
    contract(c, "wkmjg,kjKL->wKLmg", Psi1, ThetaT, &dst);         // (w k2 k3 k4 g)
    c.arena.release(ms);
  }
  c.arena.release(mk);
  return out;
}

// state buffer <- src; the buffer is reused when the size is unchanged (the steady state),
// because cudaFree synchronises the whole device (and so every lane of a batch)
static void replace_state(double *&dst, int64_t old_size, const Tensor &src, cudaStream_t s) {
  if (dst && old_size == src.size()) {
    TRG_CUDA(cudaMemcpyAsync(dst, src.p, src.size() * sizeof(double), cudaMemcpyDeviceToDevice,
                             s));
    return;
  }
  if (dst) TRG_CUDA(cudaFree(dst));
  dst = nullptr;
  if (cudaMalloc(&dst, std::max<int64_t>(src.size(), 1) * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    dst = nullptr;
    throw Error(TRG_ERR_OOM, "state allocation failed");
  }
  TRG_CUDA(cudaMemcpyAsync(dst, src.p, src.size() * sizeof(double), cudaMemcpyDeviceToDevice, s));
}

// bring the slot of physical `axis` to the front, keeping the cyclic leg order
static void rotate(Ctx &c, int axis) {
  const int d = c.d;
  int slot = -1;
  for (int i = 0; i < d; ++i)
    if (c.axes[i] == axis) slot = i;
  if (slot < 0) throw Error(TRG_ERR_ARG, "axis out of range");
  if (slot == 0) return;
  std::vector<int> perm(d + 1);
  for (int i = 0; i < d; ++i) perm[i] = (slot + i) % d;
  perm[d] = d;
  for (double **buf : {&c.phi, &c.psi, &c.psi_imp}) {
    if (!*buf) continue;
    Tensor t = permuted(c, view(*buf, c.dims), perm);
    TRG_CUDA(cudaMemcpyAsync(*buf, t.p, t.size() * sizeof(double), cudaMemcpyDeviceToDevice,
                             c.stream));
  }
  std::vector<int64_t> nd(d + 1);
  int na[4] = {-1, -1, -1, -1};
  for (int i = 0; i <= d; ++i) nd[i] = c.dims[perm[i]];
  for (int i = 0; i < d; ++i) na[i] = c.axes[perm[i]];
  c.dims = nd;
  std::memcpy(c.axes, na, sizeof(na));
}

// (a) of the step, shared by the 3D and 4D triad steps: re-split T = Phi Psi^T =
// A s D^T (eq. ABCD; SVD of T) of the current state, A and Dm as (legs, k)
struct Resplit {
  Tensor A, Dm, sv;
  int64_t k = 0, Db = 0;
};
static Resplit resplit(Ctx &c, int64_t D) {
  cudaStream_t s = c.stream;
  const int64_t r = c.dims.back(), Nf = prod(c.dims) / r;
  Tensor P2 = view(c.phi, {Nf, r}), S2 = view(c.psi, {Nf, r});
  Crit crit_resplit(c);
  Resplit out;
  // the bond lines (re-split alpha/beta, swapped gamma) keep Db = r_bond D values; the
  // ILO form (Sec. II C, Appendix A) has r_bond > 1, the pair legs stay at D
  const int64_t Db = D * c.r_bond;
  const int64_t k = std::min<int64_t>(Db, r);
  out.Db = Db;
  out.k = k;
  // only A, D and s outlive the re-split (its orthonormal factors are released)
  Tensor A = c.alloc({Nf, k}), Dm = c.alloc({Nf, k}), svT = c.alloc({r});
  {
    Arena::Mark mk = c.arena.mark();
    FoldedQR fp = orth_qr_folded(c, P2), fs = orth_qr_folded(c, S2);
    Svd rs = svd_small(c, mm(c, fp.R, fs.R, false, true));
    // A = Q_Phi U[:, :k] = Q2_Phi (Ri3_Phi U[:, :k]), D likewise with V
    Tensor Wp = c.alloc({r, k}), Ws = c.alloc({r, k});
    gemm(c, false, false, r, k, r, 1.0, fp.Ri3.p, r, 0, rs.U.p, r, 0, 0.0, Wp.p, k, 0, 1);
    gemm(c, false, false, r, k, r, 1.0, fs.Ri3.p, r, 0, rs.V.p, r, 0, 0.0, Ws.p, k, 0, 1);
    gemm(c, false, false, Nf, k, r, 1.0, fp.Q2.p, r, 0, Wp.p, k, 0, 0.0, A.p, k, 0, 1);
    gemm(c, false, false, Nf, k, r, 1.0, fs.Q2.p, r, 0, Ws.p, k, 0, 0.0, Dm.p, k, 0, 1);
    TRG_CUDA(cudaMemcpyAsync(svT.p, rs.S.p, r * sizeof(double), cudaMemcpyDeviceToDevice, s));
    c.arena.release(mk);
  }
  sign_gauge(A.p, Nf, Dm.p, Nf, k, s);
  kill_dead(svT.p, k, kRankTol, A.p, Nf, Dm.p, Nf, s);
  out.A = A;
  out.Dm = Dm;
  out.sv = svT;
  return out;
}

// (c) of the step, shared by the 3D and 4D triad steps: the four triad isometries U^A,
// U^X, U^Y, U^D (eq. HOSVD), ranges of width chi of rho = F F^T over the leg pair
// (d2, d3).  src[i] holds the tensor whose permutation `perm` (pair legs first) is the
// factor F_i, or, with W[i] given, the tensor T with F_i = perm(T R^T), R^T R = W[i].
// With the plain Gaussian sketch and no row collection, factors of one shape run their
// range finders as one batch; otherwise each runs range_factor_full (learned sketch,
// collection).  chi >= pair dimension: the identity.
static std::vector<Tensor> triad_isometries(Ctx &c, const Tensor *src[4], const Tensor *W[4],
                                            const std::vector<int> &perm, int64_t d2,
                                            int64_t d3, int64_t chi, int n) {
  const int64_t npair = d2 * d3;
  const int tags[4] = {TAG_RHO_A, TAG_RHO_X, TAG_RHO_Y, TAG_RHO_D};
  auto key = [&](int tag) { return sketch_key(c.seed, n, tag); };
  std::vector<Tensor> U(4);
  for (int i = 0; i < 4; ++i) {
    U[i] = c.alloc({npair, std::min(chi, npair)});
    if (chi >= npair) fill_identity(U[i].p, npair, npair, c.stream);
  }
  if (chi < npair) {
    Arena::Mark mk = c.arena.mark();
    // the factor of isometry i, written to dst (npair x m_i)
    auto write_factor = [&](int i, double *dst) {
      const Tensor &T = *src[i];
      Arena::Mark m2 = c.arena.mark();
      Tensor TT = T;
      if (W[i]) {
        const int64_t k = T.dims.back(), rows = T.size() / k;
        Tensor R = c.alloc({k, k}), Ri = c.alloc({k, k});
        chol_rinv(W[i]->p, R.p, Ri.p, (int)k, 1, kPivotTol, 0.0, c.stream);
        TT = mm(c, view(T.p, {rows, k}), R, false, true);
        TT.dims = T.dims;
      }
      permute(TT.p, dst, TT.dims, perm, c.stream);
      c.arena.release(m2);
    };
    const bool batchable = c.sketch_mode == 0 && c.col_cap == 0;
    std::vector<bool> done(4, false);
    for (int i = 0; i < 4 && batchable; ++i) {
      if (done[i]) continue;
      const int64_t mi = src[i]->size() / npair;
      // a batch member holds its factor (8 B per value) and digit planes of both
      // orientations (up to 2 x 5 x 2 B per value): at most 24 GB of them at once
      const int64_t per = npair * mi * 28;
      const int64_t max_grp = std::max<int64_t>(1, (int64_t(24) << 30) / per);
      std::vector<int> grp;
      for (int j = i; j < 4 && (int64_t)grp.size() < max_grp; ++j)
        if (!done[j] && src[j]->size() / npair == mi) grp.push_back(j);
      Arena::Mark mg = c.arena.mark();
      const int64_t nb = (int64_t)grp.size();
      Tensor Fs = c.alloc({nb, npair, mi});
      std::vector<uint64_t> keys;
      for (int64_t b = 0; b < nb; ++b) {
        write_factor(grp[b], Fs.p + b * npair * mi);
        keys.push_back(key(tags[grp[b]]));
      }
      Tensor Q = rsvd_factor_batched(c, Fs, chi, c.q_rho, keys);
      for (int64_t b = 0; b < nb; ++b) {
        TRG_CUDA(cudaMemcpyAsync(U[grp[b]].p, Q.p + b * npair * chi, npair * chi * 8,
                                 cudaMemcpyDeviceToDevice, c.stream));
        done[grp[b]] = true;
      }
      c.arena.release(mg);
    }
    for (int i = 0; i < 4; ++i) {
      if (done[i]) continue;
      Arena::Mark m2 = c.arena.mark();
      const int64_t mi = src[i]->size() / npair;
      Tensor F = c.alloc({npair, mi});
      write_factor(i, F.p);
      Tensor Q = range_factor_full(c, F, d2, d3, chi, c.q_rho, key(tags[i]),
                                   key(TAG_PROBE_A + tags[i] - TAG_RHO_A));
      TRG_CUDA(cudaMemcpyAsync(U[i].p, Q.p, npair * chi * 8, cudaMemcpyDeviceToDevice,
                               c.stream));
      c.arena.release(m2);
    }
    c.arena.release(mk);
  }
  for (auto &u : U) u.dims = {d2, d3, u.dims[1]};
  return U;
}

// (b) of the step, shared by the 3D and 4D triad steps: the bond swap
//     sum_x C[x I be] B[x J al] ~ X sigma Y of the re-split factors A (x, I, k) and
//     Dm (x, J, k) with singular values sv; returns X (k, I, Dg), Y (k, J, Dg), sigma
//     (w values, the first Dg kept) and the relative gap at the cut.
struct SwapOut {
  Tensor X, Y, sig;
  int64_t Dg = 0;
  double gap = INFINITY;
};
static SwapOut bond_swap(Ctx &c, const Tensor &A, const Tensor &Dm, const double *sv, int64_t k,
                         int64_t x, int64_t I, int64_t Db, int64_t p, int n) {
  // (b) bond swap: M[(I al),(J be)] = sum_x C[x I be] B[x J al] ~ X sigma Y (Appendix A).
  //     The randomized SVD of M runs in the compressed space of Appendix A, written in
  //     Gram coordinates: a left vector is Y = (C (x) 1) Y' and a right vector
  //     V = (B (x) 1) W, so that with G^C = C^T C and G^B = B^T B (D^2 x D^2, the QR
  //     compression's R^T R)
  //         M V  = (C (x) 1) P (G^B W),        M^T Q = (B (x) 1) P (G^C Q'),
  //         Y^T Y = Y'^T (G^C (x) 1) Y',        V^T V = W^T (G^B (x) 1) W,
  //     with P the swap of the two bond legs.  Only the two Grams and the final
  //     X = (C (x) 1) X', Y = (B (x) 1) Y' cost D^7; the power rounds cost D^6.
  cudaStream_t s = c.stream;
  auto key = [&](int tag) { return sketch_key(c.seed, n, tag); };
  const int64_t J = I;
  const int64_t w = std::min<int64_t>(Db + p, k * I);
  const int64_t xk = x * k, rows = x * k * k;     // coordinate rows (x, leg, leg)
  const int64_t Dg = std::min<int64_t>(Db, w);
  SwapOut out;
  out.Dg = Dg;
  out.X = c.alloc({k, I, Dg});
  out.Y = c.alloc({k, I, Dg});
  out.sig = c.alloc({w});
  Tensor &X = out.X, &Y = out.Y;
  double *sig = out.sig.p;
  Arena::Mark mk_swap = c.arena.mark();
  Tensor C = copy(c, A), B = copy(c, Dm);         // C = A s, B = D s (released after)
  scale_last(c, C, sv);
  scale_last(c, B, sv);
  Tensor Cq = permuted(c, view(C.p, {x, I, k}), {0, 2, 1});   // (x, be, I)
  Tensor Bq = permuted(c, view(B.p, {x, J, k}), {0, 2, 1});   // (x, al, J)
  Tensor GC = c.alloc({xk, xk}), GB = c.alloc({xk, xk});
  {
    // the compression Grams square the spectra of C and B: more digits (or FP64)
    const int gd = c.swap_gram_digits;
    if (gd >= 64) ++c.ortho;
    else if (is_digit_form(c.precision)) c.digits_override = std::max(gd, digits_of(c.precision));
    gemm(c, false, true, xk, xk, I, 1.0, Cq.p, I, 0, Cq.p, I, 0, 0.0, GC.p, xk, 0, 1);
    gemm(c, false, true, xk, xk, J, 1.0, Bq.p, J, 0, Bq.p, J, 0, 0.0, GB.p, xk, 0, 1);
    if (gd >= 64) --c.ortho;
    c.digits_override = 0;
  }
  // G (x) 1 applied to coordinates [(x leg) rows][(leg m)], then the two bond legs swapped
  auto apply_g = [&](const Tensor &G, const Tensor &Yc) {
    Tensor Z = c.alloc({x, k, k, w});
    gemm(c, false, false, xk, k * w, xk, 1.0, G.p, xk, 0, Yc.p, k * w, 0, 0.0, Z.p, k * w, 0,
         1);
    return Z;
  };
  auto apply_gp = [&](const Tensor &G, const Tensor &Yc) {
    Tensor out = c.alloc({x, k, k, w});
    Arena::Mark mk = c.arena.mark();
    Tensor Z = apply_g(G, Yc);
    permute(Z.p, out.p, Z.dims, {0, 2, 1, 3}, c.stream);
    c.arena.release(mk);
    return out;
  };
  // shifted CholeskyQR3 in the metric G (x) 1: Q'^T (G (x) 1) Q' = 1 (cf. orth_sc)
  auto orth_g = [&](const Tensor &G, const Tensor &Yc) {
    Tensor out = c.alloc({x, k, k, w});
    Arena::Mark mk = c.arena.mark();
    Tensor Qc = Yc;
    for (int pass = 0; pass < 3; ++pass) {
      Tensor Z = apply_g(G, Qc);
      Tensor S = c.alloc({w, w}), R = c.alloc({w, w}), Ri = c.alloc({w, w});
      Ortho og(c);   // the metric Gram and its R^-1 product in FP64
      gemm(c, true, false, w, w, rows, 1.0, Qc.p, w, 0, Z.p, w, 0, 0.0, S.p, w, 0, 1);
      chol_rinv(S.p, R.p, Ri.p, (int)w, 1, pass == 0 ? 0.0 : kPivotTol,
                pass == 0 ? kShiftRel : 0.0, c.stream);
      Tensor Qn = pass == 2 ? out : c.alloc({x, k, k, w});
      gemm(c, false, false, rows, w, w, 1.0, Qc.p, w, 0, Ri.p, w, 0, 0.0, Qn.p, w, 0, 1);
      Qc = Qn;
    }
    c.arena.release(mk);
    return out;
  };
  // first left block M Omega for the Khatri-Rao sketch Omega[(J be), m] = g2[J,m] g1[be,m]:
  // Y'[(x be), al, m] = (B^T g2)[(x al), m] g1[be, m]
  Tensor Yc = c.alloc({x, k, k, w});
  {
    Arena::Mark mk = c.arena.mark();
    Tensor g1 = c.alloc({k, w}), g2 = c.alloc({J, w}), h = c.alloc({x, k, w});
    fill_gaussian(g1.p, k, w, key(TAG_SWAP_G1), s);
    fill_gaussian(g2.p, J, w, key(TAG_SWAP_G2), s);
    gemm(c, false, false, xk, w, J, 1.0, Bq.p, J, 0, g2.p, w, 0, 0.0, h.p, w, 0, 1);
    for (int64_t ix = 0; ix < x; ++ix)
      khatri_rao(g1.p, h.p + ix * k * w, Yc.p + ix * k * k * w, k, k, w, s);
    c.arena.release(mk);
  }
  Tensor Qc = c.alloc({x, k, k, w}), Ytc = c.alloc({x, k, k, w});
  const int qs = std::max(c.q_swap, 1);
  for (int rnd = 0; rnd < qs; ++rnd) {
    Arena::Mark mk = c.arena.mark();
    if (rnd > 0) {
      Tensor Wc = orth_g(GB, Ytc);
      Tensor Yn = apply_gp(GB, Wc);
      TRG_CUDA(cudaMemcpyAsync(Yc.p, Yn.p, Yc.size() * 8, cudaMemcpyDeviceToDevice, s));
      c.arena.release(mk);
    }
    {
      Tensor Qn = orth_g(GC, Yc);
      TRG_CUDA(cudaMemcpyAsync(Qc.p, Qn.p, Qc.size() * 8, cudaMemcpyDeviceToDevice, s));
      c.arena.release(mk);
    }
    std::unique_ptr<Crit> cr(rnd + 1 == qs ? new Crit(c) : nullptr);  // feeds the core SVD
    Tensor Yt = apply_gp(GC, Qc);
    TRG_CUDA(cudaMemcpyAsync(Ytc.p, Yt.p, Ytc.size() * 8, cudaMemcpyDeviceToDevice, s));
    c.arena.release(mk);
  }
  // core: M^T Q = (B (x) 1) Ytc = Qt Rt with Qt orthonormal  ->  Q^T M = Rt^T Qt^T
  std::unique_ptr<Crit> crit_core(new Crit(c));
  Tensor Qtc = orth_g(GB, Ytc);
  Tensor Rt = c.alloc({w, w});
  {
    Arena::Mark mk = c.arena.mark();
    Tensor Z = apply_g(GB, Ytc);
    gemm(c, true, false, w, w, rows, 1.0, Qtc.p, w, 0, Z.p, w, 0, 0.0, Rt.p, w, 0, 1);
    c.arena.release(mk);
  }
  Svd cs = svd_small(c, transpose2(c, Rt));
  Tensor Xc = mm_cols(c, view(Qc.p, {rows, w}), cs.U, Dg);    // [(x be) al, g]
  Tensor Yd = mm_cols(c, view(Qtc.p, {rows, w}), cs.V, Dg);   // [(x al) be, g]
  TRG_CUDA(cudaMemcpyAsync(sig, cs.S.p, w * 8, cudaMemcpyDeviceToDevice, s));
  kill_dead(sig, Dg, kRankTol, Xc.p, rows, Yd.p, rows, s);
  {
    // X[al, I, g] = sum_{x be} C[x I be] Xc[(x be), (al g)]; same for Y with B
    Arena::Mark mk = c.arena.mark();
    Tensor Xf = c.alloc({I, k, Dg});
    gemm(c, true, false, I, k * Dg, xk, 1.0, Cq.p, I, 0, Xc.p, k * Dg, 0, 0.0, Xf.p, k * Dg, 0,
         1);
    permute(Xf.p, X.p, {I, k, Dg}, {1, 0, 2}, s);
    Tensor Yf = c.alloc({J, k, Dg});
    gemm(c, true, false, J, k * Dg, xk, 1.0, Bq.p, J, 0, Yd.p, k * Dg, 0, 0.0, Yf.p, k * Dg, 0,
         1);
    permute(Yf.p, Y.p, {J, k, Dg}, {1, 0, 2}, s);
    c.arena.release(mk);
  }
  crit_core.reset();
  double &gap_swap = out.gap;
  {
    std::vector<double> hs(w);
    TRG_CUDA(cudaMemcpyAsync(hs.data(), cs.S.p, w * sizeof(double), cudaMemcpyDeviceToHost, s));
    TRG_CUDA(cudaStreamSynchronize(s));
    if (w > Dg && hs[Dg - 1] > 0) gap_swap = (hs[Dg - 1] - hs[Dg]) / hs[Dg - 1];
  }
  c.arena.release(mk_swap);
  return out;
}

// (g) of the step, shared by the 3D and 4D triad steps: normalisation c_n = ||T||_F,
// Psi /= c_n, ln Z bookkeeping, the new state, and the step's status read back
static void finish_step(Ctx &c, Tensor &PhiN, Tensor &PsiN, Tensor &PsiImpN, int n, double gap) {
  c.mark(7);
  // normalisation c_n = ||T||_F and ln Z bookkeeping
  Crit crit_norm(c);
  cudaStream_t s = c.stream;
  const int64_t rn = PhiN.dims.back(), Nn = PhiN.size() / rn;
  Tensor Gp = mm(c, view(PhiN.p, {Nn, rn}), view(PhiN.p, {Nn, rn}), true, false);
  Tensor Gs = mm(c, view(PsiN.p, {Nn, rn}), view(PsiN.p, {Nn, rn}), true, false);
  dot(Gp.p, Gs.p, rn * rn, c.dscal + 2, c.scratch(), s);
  norm_update(c.dscal + 2, c.dscal + 1, c.dscal + 0, std::ldexp(1.0, -(n + 1)), c.dflag, s);
  scale_by_scalar(PsiN.p, PsiN.size(), c.dscal + 1, 1, s);
  if (c.have_imp) scale_by_scalar(PsiImpN.p, PsiImpN.size(), c.dscal + 1, 1, s);

  const int64_t old_size = prod(c.dims);
  replace_state(c.phi, old_size, PhiN, s);
  replace_state(c.psi, old_size, PsiN, s);
  if (c.have_imp) replace_state(c.psi_imp, old_size, PsiImpN, s);
  c.dims = PhiN.dims;
  c.nsteps = n + 1;
  if (c.imp_pair == 1) c.imp_pair = 2;
  double hc = 1.0;
  int flag = 0;
  TRG_CUDA(cudaMemcpyAsync(&hc, c.dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  TRG_CUDA(cudaMemcpyAsync(&flag, c.dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  c.mark(8);
  TRG_CUDA(cudaStreamSynchronize(s));
  c.collect_tc();
  for (int i = 0; i < Ctx::kPhases; ++i) {
    float ms = 0.f;
    TRG_CUDA(cudaEventElapsedTime(&ms, c.ev[i], c.ev[i + 1]));
    c.phase_ms[i] = ms;
  }
  c.last_logc = std::log(hc);
  c.last_gap = gap;
  c.arena.reset();
  if (flag) throw Error(flag, "non-finite norm in the coarse-graining step");
  if (linalg_error_flag(true))
    throw Error(TRG_ERR_TIMEOUT, "grid barrier of the cooperative Jacobi SVD timed out");
  if (c.mixed_now && (tc_error_flag(true) | oz_error_flag(true)))
    throw Error(TRG_ERR_TIMEOUT, "tensor-core GEMM pipeline wait timed out");
}

// ----------------------------------------------------------------------- the step
static void step_impl(Ctx &c, int axis, int64_t D, int64_t p) {
  cudaStream_t s = c.stream;
  c.mark(0);
  rotate(c, axis);
  const int64_t d1 = c.dims[0], d2 = c.dims[1], d3 = c.dims[2], d4 = c.dims[3], r = c.dims[4];
  const int64_t Nf = d1 * d2 * d3 * d4;
  const int n = c.nsteps;
  // mixed forms: tensor cores from the fourth step on; the first three steps carry
  // weights 1, 1/2, 1/4 of the free energy and have small legs, so they stay in FP64
  c.mixed_now = c.precision != TRG_PREC_FP64 && n >= 3;
  auto key = [&](int tag) { return sketch_key(c.seed, n, tag); };

  // (a) re-split T = Phi Psi^T = A s D^T (eq. ABCD; SVD of T)
  Resplit rsp = resplit(c, D);
  const int64_t Db = rsp.Db, k = rsp.k;
  Tensor A = rsp.A, Dm = rsp.Dm;
  double *sv = rsp.sv.p;  // first k entries used
  A.dims = {d1, d2, d3, d4, k};
  Dm.dims = {d1, d2, d3, d4, k};

  c.mark(1);
  SwapOut sw = bond_swap(c, A, Dm, sv, k, d1, d2 * d3 * d4, Db, p, n);
  const int64_t x = d1, I = d2 * d3 * d4, J = I, Dg = sw.Dg;
  Tensor X = sw.X, Y = sw.Y;
  X.dims = {k, d2, d3, d4, Dg};
  Y.dims = {k, d2, d3, d4, Dg};
  double *sig = sw.sig.p;
  const double gap_swap = sw.gap;

  c.mark(2);
  // (c) triad isometries from the canonical-form Grams (eq. HOSVD)
  Tensor Xs = copy(c, X), Ys = copy(c, Y);
  scale_last(c, Xs, sig);
  scale_last(c, Ys, sig);
  Tensor Wal = mm(c, view(Xs.p, {k, I * Dg}), view(Xs.p, {k, I * Dg}), false, true);
  Tensor Wbe = mm(c, view(Ys.p, {k, J * Dg}), view(Ys.p, {k, J * Dg}), false, true);
  const int64_t npair = d2 * d3;
  const int64_t chi = std::min<int64_t>(D + p, npair);
  // rho = F F^T for each of the four; the range finders run on the factors F
  // (rho^X: Xs over (al, q4, g); rho^Y: Ys; rho^A = A W_al A^T: F = A R^T with
  // R^T R = W_al; rho^D likewise with W_be)
  Tensor UA, UX, UY, UD;
  {
    const Tensor *src[4] = {&A, &Xs, &Ys, &Dm};
    const Tensor *Ws[4] = {&Wal, nullptr, nullptr, &Wbe};
    std::vector<Tensor> U = triad_isometries(c, src, Ws, {1, 2, 0, 3, 4}, d2, d3, chi, n);
    UA = U[0];
    UX = U[1];
    UY = U[2];
    UD = U[3];
  }

  c.mark(3);
  // (d) triads, eqs. E-L
  Tensor E = contract(c, "tbcda,bck->tkda", A, UA);
  Tensor F = contract(c, "abcdg,bck->akdg", X, UX);
  scale_last(c, F, sig);
  Tensor G = contract(c, "bPQRg,PQk->bkRg", Y, UY);
  Tensor H = contract(c, "wPQRb,PQk->wkRb", Dm, UD);
  const Tensor &I_ = UA, &J_ = UX, &K_ = UY, &L_ = UD;

  // (e) Gram matrices O (upper block) and P (lower block), environments, squeezers
  Tensor Ig = contract(c, "bck,bcl->kl", I_, I_), Jg = contract(c, "bck,bcl->kl", J_, J_);
  Tensor Kg = contract(c, "bck,bcl->kl", K_, K_), Lg = contract(c, "bck,bcl->kl", L_, L_);
  Tensor EI = contract(c, "tkda,kl->tlda", E, Ig);
  Tensor EEI = contract(c, "tlda,tlde->ae", EI, E);
  Tensor FJ = contract(c, "eldh,kl->ekdh", F, Jg);
  Tensor O = contract(c, "akdg,akdh->gh", F, contract(c, "ae,ekdh->akdh", EEI, FJ));
  Tensor HL = contract(c, "wkdb,kl->wldb", H, Lg);
  Tensor HHL = contract(c, "wldb,wlde->be", HL, H);
  Tensor GK = contract(c, "eldh,kl->ekdh", G, Kg);
  Tensor Pm = contract(c, "bkdg,bkdh->gh", G, contract(c, "be,ekdh->bkdh", HHL, GK));

  std::map<int, Tensor> rf, rb;
  Tensor EE4 = contract(c, "tlda,tlDe->daDe", EI, E);                       // (p4 al p4' al')
  Tensor FP = contract(c, "akdg,gh->akdh", F, Pm);
  Tensor FPJ = contract(c, "akdh,kl->aldh", FP, Jg);
  Tensor FPF4 = contract(c, "aldh,elDh->adeD", FPJ, F);                     // (al q4 al' q4')
  rf[4] = contract(c, "paPe,aqeQ->pqPQ", EE4, FPF4);
  Tensor GO = contract(c, "bkPg,gh->bkPh", G, O);
  Tensor GOK = contract(c, "bkPh,kl->blPh", GO, Kg);
  Tensor GOG4 = contract(c, "blPh,elQh->bPeQ", GOK, G);                     // (be P4 be' P4')
  Tensor HH4 = contract(c, "wldb,wlDe->bdeD", HL, H);                       // (be Q4 be' Q4')
  rb[4] = contract(c, "bPeR,bQeS->PQRS", GOG4, HH4);
  Tensor EE2 = contract(c, "tkda,tlde->kale", E, E);
  Tensor FPF2 = contract(c, "akdh,eldh->akel", FP, F);
  Tensor GOG2 = contract(c, "bkdh,eldh->kble", GO, G);
  Tensor HH2 = contract(c, "wkdb,wlde->kble", H, H);
  for (int mu : {2, 3}) {
    const char *sub = mu == 2 ? "bck,Bcl->bkBl" : "cbk,cBl->bkBl";
    Tensor II = contract(c, sub, I_, I_), JJ = contract(c, sub, J_, J_);
    Tensor KK = contract(c, sub, K_, K_), LL = contract(c, sub, L_, L_);
    Tensor G1 = contract(c, "pkPl,kale->paPe", II, EE2);
    Tensor G2 = contract(c, "qkQl,akel->aqeQ", JJ, FPF2);
    rf[mu] = contract(c, "paPe,aqeQ->pqPQ", G1, G2);
    Tensor G1b = contract(c, "PkRl,kble->PbRe", KK, GOG2);
    Tensor G2b = contract(c, "QkSl,kble->bQeS", LL, HH2);
    rb[mu] = contract(c, "PbRe,bQeS->PQRS", G1b, G2b);
  }
  c.mark(4);
  const int64_t dmu[5] = {0, 0, d2, d3, d4};
  std::map<int, Tensor> Msq, Nsq;
  double gap_sq = INFINITY;
  // the six Gram roots (forward and backward of mu = 2, 3, 4) are independent: when the
  // three pair bonds have one size, they run as one batch
  const int64_t nn0 = d2 * d2;
  const bool same = d3 * d3 == nn0 && d4 * d4 == nn0 && nn0 > D;
  const int64_t chi_s = std::min<int64_t>(D + p, nn0);
  Tensor R6;
  if (same && chi_s < nn0) {
    Tensor rho6 = c.alloc({6, nn0, nn0});
    std::vector<uint64_t> keys6;
    for (int mu : {2, 3, 4}) {
      const int b = 2 * (mu - 2);
      TRG_CUDA(cudaMemcpyAsync(rho6.p + b * nn0 * nn0, rf[mu].p, nn0 * nn0 * 8,
                               cudaMemcpyDeviceToDevice, s));
      TRG_CUDA(cudaMemcpyAsync(rho6.p + (b + 1) * nn0 * nn0, rb[mu].p, nn0 * nn0 * 8,
                               cudaMemcpyDeviceToDevice, s));
      keys6.push_back(key(TAG_SQ_F2 + mu - 2));
      keys6.push_back(key(TAG_SQ_B2 + mu - 2));
    }
    R6 = gram_root_batched(c, rho6, chi_s, c.q_rho, keys6);
  }
  for (int mu : {2, 3, 4}) {
    int64_t nn = dmu[mu] * dmu[mu];
    double g;
    auto [M, N] = R6.p
        ? squeezer_from_roots(c, view(R6.p + 2 * (mu - 2) * chi_s * nn0, {chi_s, nn0}),
                              view(R6.p + (2 * (mu - 2) + 1) * chi_s * nn0, {chi_s, nn0}), D,
                              &g)
        : squeezer(c, view(rf[mu].p, {nn, nn}), view(rb[mu].p, {nn, nn}), D,
                   std::min<int64_t>(D + p, nn), c.q_rho, key(TAG_SQ_F2 + mu - 2),
                   key(TAG_SQ_B2 + mu - 2), &g);
    gap_sq = std::min(gap_sq, g);
    M.dims = {dmu[mu], dmu[mu], M.dims[1]};
    N.dims = {dmu[mu], dmu[mu], N.dims[1]};
    Msq[mu] = M;
    Nsq[mu] = N;
  }

  c.mark(5);
  // (f) coarse contraction, eqs. makeMG / makeMH
  Tensor PhiN = contract_upper(c, E, F, I_, J_, Msq[2], Msq[3], Msq[4]);
  Tensor PsiN = contract_lower(c, G, H, K_, L_, Nsq[2], Nsq[3], Nsq[4]);
  c.mark(6);
  Tensor PsiImpN;
  if (c.have_imp) {
    Cheap ch(c);
    // impurity at slot n+1: B_imp = T_imp^T A; frozen X projector -> Y_imp = M_imp^T X / sigma
    Tensor PA = mm(c, view(c.phi, {Nf, r}), view(A.p, {Nf, k}), true, false);
    Tensor Bimp = mm(c, view(c.psi_imp, {Nf, r}), PA, false, false);
    Bimp.dims = {x, d2, d3, d4, k};
    // C = A s: contract A with X, then scale the b leg by s
    Tensor CX = contract(c, "xIJKb,aIJKg->xbag", A, X);
    scale_axis(CX.p, CX.size(), (int64_t)CX.dims[2] * CX.dims[3], k, sv, 0, nullptr, 0.0, s);
    Tensor Ytil = contract(c, "xPQRa,xbag->bPQRg", Bimp, CX);
    scale_last(c, Ytil, sig, 1, sig, 0.0);
    Tensor Gimp = contract(c, "bPQRg,PQk->bkRg", Ytil, UY);
    // impurity at slot n: D_imp = T_imp^T A s^+, frozen U^D
    Tensor Dimp = copy(c, Bimp);
    scale_last(c, Dimp, sv, 1, sv, 0.0);
    Tensor Himp = contract(c, "wPQRb,PQk->wkRb", Dimp, UD);
    if (c.imp_pair == 1) {
      // both sites of the unit cell carry the impurity: one coarse impurity tensor
      PsiImpN = contract_lower(c, Gimp, Himp, K_, L_, Nsq[2], Nsq[3], Nsq[4]);
    } else {
      // one impurity, at slot n+1 or at slot n with equal weight
      PsiImpN = contract_lower_sum(c, Gimp, H, G, Himp, K_, L_, Nsq[2], Nsq[3], Nsq[4], 0.5);
    }
  }

  finish_step(c, PhiN, PsiN, PsiImpN, n, std::min(gap_swap, gap_sq));
}

// ------------------------------------------------------------- the step in three dimensions
// The triad step for d = 3 (the case the paper costs at O(r^2 D^6), end of Sec. II B): the
// state is Phi (i1, i2, i3, g) and Psi (j1, j2, j3, g).  Re-split, bond swap and
// normalisation are the 4D step's; the pair (i2, i3) of each of A, X, Y, D is compressed
// by a triad isometry (ranges of the canonical-form Grams of eq. HOSVD); the triads are
// E (t, kA, al), F (al, kX, g), G (be, kY, g), H (w, kD, be); two squeezers (mu = 2, 3)
// come from the block environments; Phi = (E F)(I J M2 M3), Psi = (H G)(K L N2 N3).
static void step3_impl(Ctx &c, int axis, int64_t D, int64_t p) {
  cudaStream_t s = c.stream;
  c.mark(0);
  rotate(c, axis);
  const int64_t d1 = c.dims[0], d2 = c.dims[1], d3 = c.dims[2], r = c.dims[3];
  const int64_t Nf = d1 * d2 * d3;
  const int n = c.nsteps;
  c.mixed_now = c.precision != TRG_PREC_FP64 && n >= 3;
  auto key = [&](int tag) { return sketch_key(c.seed, n, tag); };

  Resplit rsp = resplit(c, D);
  const int64_t Db = rsp.Db, k = rsp.k;
  Tensor A = rsp.A, Dm = rsp.Dm;
  double *sv = rsp.sv.p;
  A.dims = {d1, d2, d3, k};
  Dm.dims = {d1, d2, d3, k};

  c.mark(1);
  SwapOut sw = bond_swap(c, A, Dm, sv, k, d1, d2 * d3, Db, p, n);
  const int64_t x = d1, I = d2 * d3, Dg = sw.Dg;
  Tensor X = sw.X, Y = sw.Y;
  X.dims = {k, d2, d3, Dg};
  Y.dims = {k, d2, d3, Dg};
  double *sig = sw.sig.p;

  c.mark(2);
  // (c) triad isometries from the canonical-form Grams (eq. HOSVD), range finders on the
  // factors F with rho = F F^T, as in 4D
  Tensor Xs = copy(c, X), Ys = copy(c, Y);
  scale_last(c, Xs, sig);
  scale_last(c, Ys, sig);
  Tensor Wal = mm(c, view(Xs.p, {k, I * Dg}), view(Xs.p, {k, I * Dg}), false, true);
  Tensor Wbe = mm(c, view(Ys.p, {k, I * Dg}), view(Ys.p, {k, I * Dg}), false, true);
  const int64_t npair = d2 * d3;
  const int64_t chi = std::min<int64_t>(D + p, npair);
  Tensor UA, UX, UY, UD;
  {
    const Tensor *src[4] = {&A, &Xs, &Ys, &Dm};
    const Tensor *Ws[4] = {&Wal, nullptr, nullptr, &Wbe};
    std::vector<Tensor> U = triad_isometries(c, src, Ws, {1, 2, 0, 3}, d2, d3, chi, n);
    UA = U[0];
    UX = U[1];
    UY = U[2];
    UD = U[3];
  }

  c.mark(3);
  // (d) triads
  Tensor E = contract(c, "tbca,bck->tka", A, UA);
  Tensor F = contract(c, "abcg,bck->akg", X, UX);
  scale_last(c, F, sig);
  Tensor G = contract(c, "bPQg,PQk->bkg", Y, UY);
  Tensor H = contract(c, "wPQb,PQk->wkb", Dm, UD);
  const Tensor &I_ = UA, &J_ = UX, &K_ = UY, &L_ = UD;

  // (e) Grams O (upper block E F I J) and P (lower block G H K L) on the bond gamma, the
  // environments of the two pairs, squeezers
  Tensor Ig = contract(c, "bck,bcl->kl", I_, I_), Jg = contract(c, "bck,bcl->kl", J_, J_);
  Tensor Kg = contract(c, "bck,bcl->kl", K_, K_), Lg = contract(c, "bck,bcl->kl", L_, L_);
  Tensor EEI = contract(c, "tla,tle->ae", contract(c, "tka,kl->tla", E, Ig), E);
  Tensor O = contract(c, "akg,akh->gh", F,
                      contract(c, "ae,ekh->akh", EEI, contract(c, "elh,kl->ekh", F, Jg)));
  Tensor HHL = contract(c, "wlb,wle->be", contract(c, "wkb,kl->wlb", H, Lg), H);
  Tensor Pm = contract(c, "bkg,bkh->gh", G,
                       contract(c, "be,ekh->bkh", HHL, contract(c, "elh,kl->ekh", G, Kg)));
  Tensor EE2 = contract(c, "tka,tle->kale", E, E);                          // (kA al kA' al')
  Tensor FPF2 = contract(c, "akh,elh->akel", contract(c, "akg,gh->akh", F, Pm), F);
  Tensor GOG2 = contract(c, "bkh,elh->kble", contract(c, "bkg,gh->bkh", G, O), G);
  Tensor HH2 = contract(c, "wkb,wle->kble", H, H);                          // (kD be kD' be')
  std::map<int, Tensor> rf, rb;
  for (int mu : {2, 3}) {
    const char *sub = mu == 2 ? "bck,Bcl->bkBl" : "cbk,cBl->bkBl";
    Tensor II = contract(c, sub, I_, I_), JJ = contract(c, sub, J_, J_);
    Tensor KK = contract(c, sub, K_, K_), LL = contract(c, sub, L_, L_);
    rf[mu] = contract(c, "paPe,aqeQ->pqPQ", contract(c, "pkPl,kale->paPe", II, EE2),
                      contract(c, "qkQl,akel->aqeQ", JJ, FPF2));
    rb[mu] = contract(c, "PbRe,bQeS->PQRS", contract(c, "PkRl,kble->PbRe", KK, GOG2),
                      contract(c, "QkSl,kble->bQeS", LL, HH2));
  }
  c.mark(4);
  const int64_t dmu[4] = {0, 0, d2, d3};
  std::map<int, Tensor> Msq, Nsq;
  double gap_sq = INFINITY;
  for (int mu : {2, 3}) {
    const int64_t nn = dmu[mu] * dmu[mu];
    double g;
    auto [M, N] = squeezer(c, view(rf[mu].p, {nn, nn}), view(rb[mu].p, {nn, nn}), D,
                           std::min<int64_t>(D + p, nn), c.q_rho, key(TAG_SQ_F2 + mu - 2),
                           key(TAG_SQ_B2 + mu - 2), &g);
    gap_sq = std::min(gap_sq, g);
    M.dims = {dmu[mu], dmu[mu], M.dims[1]};
    N.dims = {dmu[mu], dmu[mu], N.dims[1]};
    Msq[mu] = M;
    Nsq[mu] = N;
  }

  c.mark(5);
  // (f) coarse contraction: Phi[t, k2, k3, g] = (E F)[t kA kX g] Theta_U[kA kX k2 k3]
  auto theta = [&](const Tensor &P, const Tensor &Q, const Tensor &S2, const Tensor &S3) {
    Tensor PS = contract(c, "bck,bBm->ckBm", P, S2);
    Tensor QS = contract(c, "BCl,cCn->Blcn", Q, S3);
    return contract(c, "ckBm,Blcn->klmn", PS, QS);
  };
  Tensor ThU = theta(I_, J_, Msq[2], Msq[3]);                                // (kA kX k2 k3)
  Tensor ThL = theta(K_, L_, Nsq[2], Nsq[3]);                                // (kY kD k2 k3)
  Tensor PhiN = contract(c, "tklg,klmn->tmng", contract(c, "tka,alg->tklg", E, F), ThU);
  // Psi[w, k2', k3', g] = (H G)[w kD kY g] Theta_L[kY kD k2' k3']
  auto lower = [&](const Tensor &Gx, const Tensor &Hx) {
    return contract(c, "wlkg,klmn->wmng", contract(c, "wlb,bkg->wlkg", Hx, Gx), ThL);
  };
  Tensor PsiN = lower(G, H);

  c.mark(6);
  Tensor PsiImpN;
  if (c.have_imp) {
    Cheap ch(c);
    // frozen pure projectors, as in 4D: slot n+1 gives B_imp = T_imp^T A and
    // Y_imp = M_imp^T X / sigma; slot n gives D_imp = T_imp^T A s^+
    Tensor PA = mm(c, view(c.phi, {Nf, r}), view(A.p, {Nf, k}), true, false);
    Tensor Bimp = mm(c, view(c.psi_imp, {Nf, r}), PA, false, false);
    Bimp.dims = {x, d2, d3, k};
    Tensor CX = contract(c, "xIJb,aIJg->xbag", A, X);
    scale_axis(CX.p, CX.size(), (int64_t)CX.dims[2] * CX.dims[3], k, sv, 0, nullptr, 0.0, s);
    Tensor Ytil = contract(c, "xPQa,xbag->bPQg", Bimp, CX);
    scale_last(c, Ytil, sig, 1, sig, 0.0);
    Tensor Gimp = contract(c, "bPQg,PQk->bkg", Ytil, UY);
    Tensor Dimp = copy(c, Bimp);
    scale_last(c, Dimp, sv, 1, sv, 0.0);
    Tensor Himp = contract(c, "wPQb,PQk->wkb", Dimp, UD);
    if (c.imp_pair == 1) {
      PsiImpN = lower(Gimp, Himp);
    } else {
      // (H G_imp + H_imp G) Theta_L / 2: the two slots share the Theta_L product
      Tensor HG = contract(c, "wlb,bkg->wlkg", H, Gimp);
      contract(c, "wlb,bkg->wlkg", Himp, G, &HG, 1.0);
      axpby(HG.p, HG.p, 0.5, 0.0, HG.size(), s);
      PsiImpN = contract(c, "wlkg,klmn->wmng", HG, ThL);
    }
  }
  finish_step(c, PhiN, PsiN, PsiImpN, n, std::min(sw.gap, gap_sq));
}

// -------------------------------------------------------------------- init helpers
static void ensure_ctx(Ctx &c) {
  std::string e;
  if (!(e = study_opt("decomp_fp64")).empty()) c.crit_fp64 = e[0] == '1';
  if (!(e = study_opt("tc_phases")).empty()) c.phase_mask = (unsigned)strtoul(e.c_str(), nullptr, 0);
  if (!(e = study_opt("exact_everywhere")).empty()) c.cheap_policy = e[0] != '1';
  if (!(e = study_opt("tc_min_max")).empty()) c.tc_min_max = atoll(e.c_str());
  if (!(e = study_opt("swap_gram_digits")).empty()) c.swap_gram_digits = atoi(e.c_str());
  if (!(e = study_opt("decomp_cuda_fp64")).empty()) c.x7_policy = e[0] != '1';
  if (!c.dscal) {
    TRG_CUDA(cudaMalloc(&c.dscal, 512 * sizeof(double)));
    TRG_CUDA(cudaMalloc(&c.dflag, sizeof(int)));
    TRG_CUDA(cudaMalloc(&c.d_sketch_cnt, 2 * sizeof(unsigned long long)));
    TRG_CUDA(cudaMemset(c.d_sketch_cnt, 0, 2 * sizeof(unsigned long long)));
  }
  if (!c.stream && !c.own_stream) {
    TRG_CUDA(cudaStreamCreateWithFlags(&c.own_stream, cudaStreamNonBlocking));
    c.stream = c.own_stream;
  }
}

static void free_state(Ctx &c) {
  for (double **b : {&c.phi, &c.psi, &c.psi_imp}) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  c.init = false;
}

// T0 from a CP factor W (rows: site states, columns: bond index), weights and observable
static void init_cp(Ctx &c, double beta, const std::vector<double> &W, int nstate, int nb,
                    const std::vector<double> &weight, const std::vector<double> &obs,
                    int d = 4) {
  ensure_ctx(c);
  TRG_CUDA(cudaStreamSynchronize(c.stream));
  free_state(c);
  int64_t nf = 1;
  for (int mu = 0; mu < d; ++mu) nf *= nb;
  std::vector<double> phi(nf * nstate), psi(nf * nstate), imp(nf * nstate);
  for (int64_t i = 0; i < nf; ++i) {
    for (int a = 0; a < nstate; ++a) {
      double v = 1.0;
      int64_t rem = i;
      for (int mu = d - 1; mu >= 0; --mu, rem /= nb) v *= W[a * nb + rem % nb];
      phi[i * nstate + a] = v;
      psi[i * nstate + a] = v * weight[a];
      imp[i * nstate + a] = v * weight[a] * obs[a];
    }
  }
  c.d = d;
  c.dims.assign(d, nb);
  c.dims.push_back(nstate);
  for (int i = 0; i < 4; ++i) c.axes[i] = i < d ? i : -1;
  for (auto pr : {std::make_pair(&c.phi, &phi), std::make_pair(&c.psi, &psi),
                  std::make_pair(&c.psi_imp, &imp)}) {
    TRG_CUDA(cudaMalloc(pr.first, pr.second->size() * sizeof(double)));
    TRG_CUDA(cudaMemcpyAsync(*pr.first, pr.second->data(), pr.second->size() * sizeof(double),
                             cudaMemcpyHostToDevice, c.stream));
  }
  TRG_CUDA(cudaMemsetAsync(c.dscal, 0, 8 * sizeof(double), c.stream));
  TRG_CUDA(cudaMemsetAsync(c.dflag, 0, sizeof(int), c.stream));
  Tensor Gp = mm(c, view(c.phi, {nf, nstate}), view(c.phi, {nf, nstate}), true, false);
  Tensor Gs = mm(c, view(c.psi, {nf, nstate}), view(c.psi, {nf, nstate}), true, false);
  dot(Gp.p, Gs.p, (int64_t)nstate * nstate, c.dscal + 2, c.scratch(), c.stream);
  norm_update(c.dscal + 2, c.dscal + 1, c.dscal + 0, 1.0, c.dflag, c.stream);
  scale_by_scalar(c.psi, nf * nstate, c.dscal + 1, 1, c.stream);
  scale_by_scalar(c.psi_imp, nf * nstate, c.dscal + 1, 1, c.stream);
  TRG_CUDA(cudaStreamSynchronize(c.stream));
  c.arena.reset();
  c.beta = beta;
  c.nsteps = 0;
  c.have_imp = true;
  c.imp_pair = 0;
  c.ising = false;
  c.init = true;
}

static void init_ising_ctx(Ctx &c, double beta, double h, int d = 4) {
  double cb = std::sqrt(std::cosh(beta)), sb = std::sqrt(std::sinh(beta));
  init_cp(c, beta, {cb, sb, cb, -sb}, 2, 2, {std::exp(h), std::exp(-h)}, {1.0, -1.0}, d);
  c.ising = true;
}

static void init_clock_ctx(Ctx &c, int q, double beta, double h, int d = 4) {
  // real Fourier basis diagonalises the circulant bond matrix exp(beta cos(th - th'))
  std::vector<std::vector<double>> F;
  std::vector<double> th(q);
  for (int k = 0; k < q; ++k) th[k] = 2.0 * M_PI * k / q;
  F.push_back(std::vector<double>(q, 1.0 / std::sqrt((double)q)));
  for (int m = 1; m <= (q - 1) / 2; ++m) {
    std::vector<double> cc(q), ss(q);
    for (int k = 0; k < q; ++k) {
      cc[k] = std::cos(m * th[k]) * std::sqrt(2.0 / q);
      ss[k] = std::sin(m * th[k]) * std::sqrt(2.0 / q);
    }
    F.push_back(cc);
    F.push_back(ss);
  }
  if (q % 2 == 0) {
    std::vector<double> alt(q);
    for (int k = 0; k < q; ++k) alt[k] = std::cos(M_PI * k) / std::sqrt((double)q);
    F.push_back(alt);
  }
  std::vector<double> W(q * q), wt(q), obs(q);
  for (int m = 0; m < q; ++m) {
    double lam = 0.0;
    for (int a = 0; a < q; ++a)
      for (int b = 0; b < q; ++b)
        lam += F[m][a] * std::exp(beta * std::cos(th[a] - th[b])) * F[m][b];
    if (lam < 0.0) lam = 0.0;
    for (int a = 0; a < q; ++a) W[a * q + m] = F[m][a] * std::sqrt(lam);
  }
  for (int a = 0; a < q; ++a) {
    obs[a] = std::cos(th[a]);
    wt[a] = std::exp(h * obs[a]);
  }
  init_cp(c, beta, W, q, q, wt, obs, d);
}

// ln Z/V and f of the current state (synchronises the stream)
static void free_energy_ctx(Ctx &c, double *f_per_site, double *lnZ_per_site) {
  if (!c.init) throw Error(TRG_ERR_NOINIT, "no model initialised");
  int64_t n = prod(c.dims);
  dot(c.phi, c.psi, n, c.dscal + 3, c.scratch(), c.stream);
  double h[4];
  TRG_CUDA(cudaMemcpyAsync(h, c.dscal, 4 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  TRG_CUDA(cudaStreamSynchronize(c.stream));
  double lz = h[0] + std::log(std::fabs(h[3])) * std::ldexp(1.0, -c.nsteps);
  if (lnZ_per_site) *lnZ_per_site = lz;
  if (f_per_site) *f_per_site = c.beta > 0.0 ? -lz / c.beta : NAN;
}

static double magnetisation_ctx(Ctx &c) {
  if (!c.init || !c.have_imp) throw Error(TRG_ERR_NOINIT, "no impurity state");
  int64_t n = prod(c.dims);
  dot(c.phi, c.psi, n, c.dscal + 3, c.scratch(), c.stream);
  dot(c.phi, c.psi_imp, n, c.dscal + 4, c.scratch(), c.stream);
  double h[2];
  TRG_CUDA(cudaMemcpyAsync(h, c.dscal + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  TRG_CUDA(cudaStreamSynchronize(c.stream));
  return h[1] / h[0];
}

// Gu-Wen ratio X = (Tr A)^2 / Tr(A^2), A_kl = sum T[i1 i2 i3 k, i1 i2 i3 l] (Sec. III D,
// eq. X): the open leg is the slot of the last physical axis, the others are traced
// pairwise.  A = Phi' Psi'^T over the three traced legs and the bond (one GEMM).
static double gu_wen_ctx(Ctx &c) {
  if (!c.init) throw Error(TRG_ERR_NOINIT, "no model initialised");
  int slot = 0;
  for (int i = 0; i < c.d; ++i)
    if (c.axes[i] == c.d - 1) slot = i;
  std::string fa = std::string("abcd").substr(0, c.d) + "g", fb = fa;
  fa[slot] = 'k';
  fb[slot] = 'l';
  Arena::Mark mk = c.arena.mark();
  Tensor A = contract(c, fa + "," + fb + "->kl", view(c.phi, c.dims), view(c.psi, c.dims));
  const int64_t n = A.dims[0];
  std::vector<double> h(n * n);
  TRG_CUDA(cudaMemcpyAsync(h.data(), A.p, n * n * sizeof(double), cudaMemcpyDeviceToHost,
                           c.stream));
  TRG_CUDA(cudaStreamSynchronize(c.stream));
  c.arena.release(mk);
  double tr = 0.0, tr2 = 0.0;
  for (int64_t k = 0; k < n; ++k) {
    tr += h[k * n + k];
    for (int64_t l = 0; l < n; ++l) tr2 += h[k * n + l] * h[l * n + k];
  }
  return tr * tr / tr2;
}

// one step with the error context of the phase that failed
static void step_ctx(Ctx &c, int axis, int D, int p) {
  try {
    if (c.d == 3)
      step3_impl(c, axis, D, p);
    else
      step_impl(c, axis, D, p);
  } catch (const Error &e) {
    cudaStreamSynchronize(c.stream);
    c.arena.reset();
    throw Error(e.code, std::string(e.what()) + " [step phase " + std::to_string(c.phase) + "]");
  }
}

// ------------------------------------------------------------ batched instances (S14)
// A coupling sweep: many independent instances (model, beta, h, D, seed), each with its
// own persistent state.  `lanes` engine contexts, each with its own CUDA stream and
// scratch arena, run concurrently (one host thread per lane); every instance is bound to
// one lane, which swaps its state in, runs its steps and swaps it out.  Instances do not
// interact, so the results do not depend on the lane count or schedule.
struct InstState {
  int model = 0;  // 0: Ising, q >= 2: Z_q clock
  double beta = 0.0, h = 0.0;
  int D = 0, p = 0;
  uint64_t seed = 0;
  bool init = false, have_imp = false;
  double *phi = nullptr, *psi = nullptr, *psi_imp = nullptr;
  std::vector<int64_t> dims;
  int axes[4] = {0, 1, 2, 3};
  int d = 4;                   // lattice dimension (3 or 4)
  int nsteps = 0;
  double *dscal = nullptr;
  int *dflag = nullptr;
  double last_logc = 0.0, last_gap = INFINITY;
};

struct Lane {
  std::unique_ptr<Ctx> c;
  double *own_dscal = nullptr;
  int *own_dflag = nullptr;
  std::vector<int> members;
  double cost = 0.0;
};

static void swap_in(Lane &L, InstState &s) {
  Ctx &c = *L.c;
  c.init = s.init;
  c.have_imp = s.have_imp;
  c.beta = s.beta;
  c.phi = s.phi;
  c.psi = s.psi;
  c.psi_imp = s.psi_imp;
  c.dims = s.dims;
  std::memcpy(c.axes, s.axes, sizeof(c.axes));
  c.nsteps = s.nsteps;
  c.dscal = s.dscal;
  c.dflag = s.dflag;
  c.seed = s.seed;
  c.last_logc = s.last_logc;
  c.last_gap = s.last_gap;
}

static void swap_out(Lane &L, InstState &s) {
  Ctx &c = *L.c;
  s.init = c.init;
  s.have_imp = c.have_imp;
  s.beta = c.beta;
  s.phi = c.phi;
  s.psi = c.psi;
  s.psi_imp = c.psi_imp;
  s.dims = c.dims;
  std::memcpy(s.axes, c.axes, sizeof(s.axes));
  s.nsteps = c.nsteps;
  s.last_logc = c.last_logc;
  s.last_gap = c.last_gap;
  c.phi = c.psi = c.psi_imp = nullptr;
  c.init = false;
  c.dscal = L.own_dscal;
  c.dflag = L.own_dflag;
}

struct Batch {
  std::vector<InstState> inst;
  std::vector<Lane> lanes;
  int device = 0;
};
static std::unique_ptr<Batch> g_batch;

// run f(lane, instance) for every instance, lanes in parallel host threads
template <class F>
static void for_each_lane(Batch &B, F &&f) {
  std::vector<std::string> errs(B.lanes.size());
  std::vector<int> codes(B.lanes.size(), TRG_OK);
  std::vector<std::thread> th;
  for (size_t l = 0; l < B.lanes.size(); ++l) {
    th.emplace_back([&, l] {
      Lane &L = B.lanes[l];
      try {
        TRG_CUDA(cudaSetDevice(B.device));
        for (int id : L.members) {
          swap_in(L, B.inst[id]);
          try {
            f(L, B.inst[id]);
          } catch (...) {
            swap_out(L, B.inst[id]);
            throw;
          }
          swap_out(L, B.inst[id]);
        }
      } catch (const Error &e) {
        errs[l] = e.what();
        codes[l] = e.code;
      } catch (const std::exception &e) {
        errs[l] = e.what();
        codes[l] = TRG_ERR_CUDA;
      }
    });
  }
  for (auto &t : th) t.join();
  for (size_t l = 0; l < errs.size(); ++l)
    if (codes[l] != TRG_OK) throw Error(codes[l], "lane " + std::to_string(l) + ": " + errs[l]);
}

static void batch_free_all() {
  if (!g_batch) return;
  for (Lane &L : g_batch->lanes)
    if (L.c && L.c->stream) cudaStreamSynchronize(L.c->stream);
  for (InstState &s : g_batch->inst) {
    for (double *b : {s.phi, s.psi, s.psi_imp, s.dscal})
      if (b) cudaFree(b);
    if (s.dflag) cudaFree(s.dflag);
  }
  for (Lane &L : g_batch->lanes) {
    if (!L.c) continue;
    L.c->arena.release();
    if (L.own_dscal) cudaFree(L.own_dscal);
    if (L.own_dflag) cudaFree(L.own_dflag);
    if (L.c->d_sketch_cnt) cudaFree(L.c->d_sketch_cnt);
    if (L.c->own_stream) cudaStreamDestroy(L.c->own_stream);
  }
  g_batch.reset();
}

}  // namespace trg

// ================================================================== C ABI
using namespace trg;

template <class F>
static trg_status guarded(F &&f) {
  try {
    f();
    g_err = "ok";
    return TRG_OK;
  } catch (const Error &e) {
    g_err = e.what();
    return e.code;
  } catch (const std::exception &e) {
    g_err = e.what();
    return TRG_ERR_CUDA;
  }
}

// ------------------------------------------------------------------------------------
// Plain ATRG in d = 2, 3, 4 dimensions (eqs. makeG / makeH), the paper's comparison
// method.  Same re-split, sketches, squeezer rule and normalisation as the triad step;
// the bond swap forms M[(al I), (J be)] = sum_x C[x I be] B[x J al] explicitly and runs
// the randomized SVD of Appendix A on it (the compressed form of the appendix gives the
// same subspaces); the blocks Up = A X sigma and Lo = Y D and every environment are
// formed as tensors.  M, Up and Lo hold D^(2d) values, so d = 4 is limited to small D;
// d = 2 compares with Onsager's solution (for d = 2 the triad form is this method).
// The state is separate from the triad state.
// ------------------------------------------------------------------------------------
struct AtrgState {
  bool init = false;
  int d = 0;
  double beta = 0.0;
  double *phi = nullptr, *psi = nullptr;
  std::vector<int64_t> dims;     // d legs, then the bond
  int axes[4] = {0, 1, 2, 3};
  int nsteps = 0;
  double logsum = 0.0;           // sum_n ln(c_n) / 2^n
  double last_logc = 0.0, last_gap = INFINITY;
};
static AtrgState &atrg_state() {
  static AtrgState a;
  return a;
}

static void atrg_free(AtrgState &a) {
  for (double **b : {&a.phi, &a.psi}) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  a.init = false;
}

// Tr((Phi^T Phi)(Psi^T Psi)) = ||Phi Psi^T||_F^2, read back to the host
static double atrg_norm2(Ctx &c, const Tensor &Phi, const Tensor &Psi) {
  const int64_t r = Phi.dims.back(), n = Phi.size() / r;
  Arena::Mark mk = c.arena.mark();
  Tensor Gp = mm(c, view(Phi.p, {n, r}), view(Phi.p, {n, r}), true, false);
  Tensor Gs = mm(c, view(Psi.p, {n, r}), view(Psi.p, {n, r}), true, false);
  Tensor out = c.alloc({1});
  dot(Gp.p, Gs.p, r * r, out.p, c.scratch(), c.stream);
  double h = 0.0;
  TRG_CUDA(cudaMemcpyAsync(&h, out.p, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  TRG_CUDA(cudaStreamSynchronize(c.stream));
  c.arena.release(mk);
  return h;
}

static void atrg_init_ising(Ctx &c, int d, double beta, double h) {
  ensure_ctx(c);
  TRG_CUDA(cudaStreamSynchronize(c.stream));
  AtrgState &a = atrg_state();
  atrg_free(a);
  // Phi0[i1..id, s] = prod_mu W[s, i_mu], Psi0 = e^{h s} Phi0 (Sec. III CP form)
  const double cb = std::sqrt(std::cosh(beta)), sb = std::sqrt(std::sinh(beta));
  const double W[2][2] = {{cb, sb}, {cb, -sb}}, wt[2] = {std::exp(h), std::exp(-h)};
  const int64_t nf = int64_t(1) << d;
  std::vector<double> phi(nf * 2), psi(nf * 2);
  for (int64_t i = 0; i < nf; ++i)
    for (int s = 0; s < 2; ++s) {
      double v = 1.0;
      for (int mu = 0; mu < d; ++mu) v *= W[s][(i >> (d - 1 - mu)) & 1];
      phi[i * 2 + s] = v;
      psi[i * 2 + s] = v * wt[s];
    }
  a.dims.assign(d, 2);
  a.dims.push_back(2);
  for (int i = 0; i < 4; ++i) a.axes[i] = i;
  for (auto pr : {std::make_pair(&a.phi, &phi), std::make_pair(&a.psi, &psi)}) {
    TRG_CUDA(cudaMalloc(pr.first, pr.second->size() * sizeof(double)));
    TRG_CUDA(cudaMemcpyAsync(*pr.first, pr.second->data(), pr.second->size() * sizeof(double),
                             cudaMemcpyHostToDevice, c.stream));
  }
  const double n2 = atrg_norm2(c, view(a.phi, a.dims), view(a.psi, a.dims));
  const double c0 = std::sqrt(std::max(n2, 0.0));
  if (!(c0 > 0.0) || !std::isfinite(c0)) throw Error(TRG_ERR_NONFINITE, "initial norm");
  axpby(a.psi, a.psi, 1.0 / c0, 0.0, prod(a.dims), c.stream);
  TRG_CUDA(cudaStreamSynchronize(c.stream));
  c.arena.reset();
  a.d = d;
  a.beta = beta;
  a.nsteps = 0;
  a.logsum = std::log(c0);
  a.init = true;
}

static void atrg_step_impl(Ctx &c, int axis, int64_t D, int64_t p) {
  AtrgState &a = atrg_state();
  cudaStream_t s = c.stream;
  const int d = a.d, n = a.nsteps;
  c.mixed_now = c.precision != TRG_PREC_FP64 && n >= 3;
  auto key = [&](int tag) { return sketch_key(c.seed, n, tag); };
  // rotate the slot of `axis` to the front, keeping the cyclic order
  int slot = -1;
  for (int i = 0; i < d; ++i)
    if (a.axes[i] == axis) slot = i;
  if (slot < 0) throw Error(TRG_ERR_ARG, "axis out of range");
  if (slot > 0) {
    std::vector<int> perm;
    for (int i = 0; i < d; ++i) perm.push_back((slot + i) % d);
    perm.push_back(d);
    for (double *buf : {a.phi, a.psi}) {
      Tensor t = permuted(c, view(buf, a.dims), perm);
      TRG_CUDA(cudaMemcpyAsync(buf, t.p, t.size() * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    std::vector<int64_t> nd;
    int na[4];
    for (int i = 0; i <= d; ++i) nd.push_back(a.dims[perm[i]]);
    for (int i = 0; i < d; ++i) na[i] = a.axes[perm[i]];
    a.dims = nd;
    std::memcpy(a.axes, na, sizeof(int) * d);
  }
  const int64_t x = a.dims[0], r = a.dims[d];
  const int64_t I = prod(a.dims, 1, d), Nf = x * I;

  // (a) re-split T = Phi Psi^T = A s D^T.  c.phase labels each part with the triad
  // step's phase numbers, so the precision policy's phase mask applies alike (no
  // timing events are recorded for these steps)
  c.phase = 0;
  const int64_t k = std::min<int64_t>(D, std::min<int64_t>(r, Nf));
  Tensor A = c.alloc({Nf, k}), Dm = c.alloc({Nf, k}), sv = c.alloc({std::max<int64_t>(r, 1)});
  {
    Crit cr(c);
    Arena::Mark mk = c.arena.mark();
    auto [Qp, Rp] = orth_qr(c, view(a.phi, {Nf, r}));
    auto [Qs, Rs] = orth_qr(c, view(a.psi, {Nf, r}));
    Svd rs = svd_small(c, mm(c, Rp, Rs, false, true));
    gemm(c, false, false, Nf, k, r, 1.0, Qp.p, r, 0, rs.U.p, r, 0, 0.0, A.p, k, 0, 1);
    gemm(c, false, false, Nf, k, r, 1.0, Qs.p, r, 0, rs.V.p, r, 0, 0.0, Dm.p, k, 0, 1);
    TRG_CUDA(cudaMemcpyAsync(sv.p, rs.S.p, r * sizeof(double), cudaMemcpyDeviceToDevice, s));
    c.arena.release(mk);
  }
  sign_gauge(A.p, Nf, Dm.p, Nf, k, s);
  kill_dead(sv.p, k, kRankTol, A.p, Nf, Dm.p, Nf, s);

  // (b) bond swap on the explicit M[(al I), (J be)] (Appendix A, q_swap rounds)
  c.phase = 1;
  const int64_t w = std::min<int64_t>(D + p, k * I), Dg = std::min<int64_t>(D, w);
  Tensor C = copy(c, A), B = copy(c, Dm);                    // C = A s, B = D s
  scale_last(c, C, sv.p);
  scale_last(c, B, sv.p);
  Tensor M = contract(c, "xib,xja->aijb", view(C.p, {x, I, k}), view(B.p, {x, I, k}));
  const int64_t mr = k * I;                                  // rows (al I) = cols (J be)
  Tensor Mv = view(M.p, {mr, mr});
  Tensor Q, Z;
  {
    Tensor Om = c.alloc({mr, w});
    Arena::Mark mk = c.arena.mark();
    Tensor g1 = c.alloc({k, w}), g2 = c.alloc({I, w});
    fill_gaussian(g1.p, k, w, key(TAG_SWAP_G1), s);
    fill_gaussian(g2.p, I, w, key(TAG_SWAP_G2), s);
    khatri_rao(g2.p, g1.p, Om.p, I, k, w, s);                // Om[(J be), m] = g2[J,m] g1[be,m]
    c.arena.release(mk);
    const int qs = std::max(c.q_swap, 1);
    for (int rnd = 0; rnd < qs; ++rnd) {
      Q = orth_sc(c, mm(c, Mv, Om, false, false));
      if (rnd + 1 < qs) Om = orth_sc(c, mm(c, Mv, Q, true, false));
    }
    Z = mm(c, Mv, Q, true, false);                           // M^T Q = (Q^T M)^T, mr x w
  }
  Svd cs;
  {
    Crit cr(c);
    cs = svd_small(c, Z);                                    // Z = U S V^T: Q^T M = V S U^T
  }
  Tensor X = mm_cols(c, Q, cs.V, Dg);                        // [(al I), g]
  Tensor Yc = c.alloc({mr, Dg});                             // [(J be), g]
  TRG_CUDA(cudaMemcpy2DAsync(Yc.p, Dg * sizeof(double), cs.U.p, w * sizeof(double),
                             Dg * sizeof(double), mr, cudaMemcpyDeviceToDevice, s));
  Tensor sig = c.alloc({w});
  TRG_CUDA(cudaMemcpyAsync(sig.p, cs.S.p, w * sizeof(double), cudaMemcpyDeviceToDevice, s));
  kill_dead(sig.p, Dg, kRankTol, X.p, mr, Yc.p, mr, s);
  double gap_swap = INFINITY;
  {
    std::vector<double> hs(w);
    TRG_CUDA(cudaMemcpyAsync(hs.data(), cs.S.p, w * sizeof(double), cudaMemcpyDeviceToHost, s));
    TRG_CUDA(cudaStreamSynchronize(s));
    if (w > Dg && hs[Dg - 1] > 0) gap_swap = (hs[Dg - 1] - hs[Dg]) / hs[Dg - 1];
  }
  Tensor Y = permuted(c, view(Yc.p, {I, k, Dg}), {1, 0, 2});  // [be, J, g]
  scale_last(c, X, sig.p);                                   // X sigma

  c.phase = 3;
  // blocks Up[t, P, Q, g] = sum_al A[t P al] (X sigma)[al Q g],
  //        Lo[w, P, Q, g] = sum_be Y[be P g] D[w Q be]   (P, Q: the d-1 legs of each site)
  Tensor Up = contract(c, "tPa,aQg->tPQg", view(A.p, {x, I, k}), view(X.p, {k, I, Dg}));
  Tensor Lo = contract(c, "bPg,wQb->wPQg", view(Y.p, {k, I, Dg}), view(Dm.p, {x, I, k}));
  const int64_t R = Up.size() / Dg;
  Tensor O = mm(c, view(Up.p, {R, Dg}), view(Up.p, {R, Dg}), true, false);
  Tensor Pm = mm(c, view(Lo.p, {R, Dg}), view(Lo.p, {R, Dg}), true, false);
  Tensor UpP = mm(c, view(Up.p, {R, Dg}), Pm, false, false);
  Tensor LoO = mm(c, view(Lo.p, {R, Dg}), O, false, false);
  // full leg lists: t, p_2..p_d, q_2..q_d, g
  std::vector<int64_t> ldims = {x};
  for (int i = 1; i < d; ++i) ldims.push_back(a.dims[i]);
  for (int i = 1; i < d; ++i) ldims.push_back(a.dims[i]);
  ldims.push_back(Dg);
  const std::string pl = std::string("abc").substr(0, d - 1), ql = std::string("def").substr(0, d - 1);
  const std::string full = "t" + pl + ql + "g";
  double gap_sq = INFINITY;
  std::vector<Tensor> Msq(d + 1), Nsq(d + 1);
  for (int mu = 2; mu <= d; ++mu) {
    const char pc = pl[mu - 2], qc = ql[mu - 2];
    std::string sa = full, sb = full;
    for (auto &ch : sa) ch = ch == pc ? 'P' : ch == qc ? 'Q' : ch;
    for (auto &ch : sb) ch = ch == pc ? 'R' : ch == qc ? 'S' : ch;
    const int64_t dm = a.dims[mu - 1], nn = dm * dm;
    c.phase = 3;
    Tensor rf = contract(c, sa + "," + sb + "->PQRS", view(UpP.p, ldims), view(Up.p, ldims));
    Tensor rb = contract(c, sa + "," + sb + "->PQRS", view(LoO.p, ldims), view(Lo.p, ldims));
    double g = INFINITY;
    c.phase = 4;
    auto [Mq, Nq] = squeezer(c, view(rf.p, {nn, nn}), view(rb.p, {nn, nn}), D,
                             std::min<int64_t>(D + p, nn), c.q_rho, key(TAG_SQ_F2 + mu - 2),
                             key(TAG_SQ_B2 + mu - 2), &g);
    gap_sq = std::min(gap_sq, g);
    Msq[mu] = Mq;
    Nsq[mu] = Nq;
  }
  // coarse tensors Phi[t, k2..kd, g] = Up . M_2 ... M_d, Psi likewise with N
  auto coarse = [&](const Tensor &blk, std::vector<Tensor> &S) {
    Tensor cur = view(blk.p, ldims);
    std::string legs = full;
    for (int mu = 2; mu <= d; ++mu) {
      const char pc = pl[mu - 2], qc = ql[mu - 2], kc = char('K' + (mu - 2));
      std::string out;
      for (char ch : legs)
        if (ch != pc && ch != qc) out += ch;
      out += kc;
      const int64_t dm = a.dims[mu - 1];
      Tensor Sv = view(S[mu].p, {dm, dm, S[mu].dims[1]});
      cur = contract(c, legs + "," + std::string{pc, qc, kc} + "->" + out, cur, Sv);
      legs = out;
    }
    // legs = t g K L M ... -> t K L M ... g
    std::string want = "t";
    for (int mu = 2; mu <= d; ++mu) want += char('K' + (mu - 2));
    want += "g";
    std::vector<int> perm;
    for (char ch : want) perm.push_back((int)legs.find(ch));
    return permuted(c, cur, perm);
  };
  c.phase = 5;
  Tensor PhiN = coarse(Up, Msq);
  Tensor PsiN = coarse(Lo, Nsq);

  // normalisation c_n = ||T||_F, ln Z bookkeeping
  const double c2 = atrg_norm2(c, PhiN, PsiN);
  const double cn = std::sqrt(std::max(c2, 0.0));
  if (!(cn > 0.0) || !std::isfinite(cn))
    throw Error(TRG_ERR_NONFINITE, "non-finite norm in the ATRG step");
  axpby(PsiN.p, PsiN.p, 1.0 / cn, 0.0, PsiN.size(), s);
  const int64_t old_size = prod(a.dims);
  replace_state(a.phi, old_size, PhiN, s);
  replace_state(a.psi, old_size, PsiN, s);
  TRG_CUDA(cudaStreamSynchronize(s));
  a.dims = PhiN.dims;
  a.nsteps = n + 1;
  a.logsum += std::log(cn) * std::ldexp(1.0, -(n + 1));
  a.last_logc = std::log(cn);
  a.last_gap = std::min(gap_swap, gap_sq);
  c.arena.reset();
}

static void atrg_free_energy(Ctx &c, double *f, double *lz_out) {
  AtrgState &a = atrg_state();
  if (!a.init) throw Error(TRG_ERR_NOINIT, "no ATRG model initialised");
  Tensor out = c.alloc({1});
  dot(a.phi, a.psi, prod(a.dims), out.p, c.scratch(), c.stream);
  double tr = 0.0;
  TRG_CUDA(cudaMemcpyAsync(&tr, out.p, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  TRG_CUDA(cudaStreamSynchronize(c.stream));
  c.arena.reset();
  const double lz = a.logsum + std::log(std::fabs(tr)) * std::ldexp(1.0, -a.nsteps);
  if (lz_out) *lz_out = lz;
  if (f) *f = a.beta > 0.0 ? -lz / a.beta : NAN;
}

extern "C" {

trg_status trg_init_ising(int d, double beta, double h) {
  return guarded([&] {
    if (d != 3 && d != 4) throw Error(TRG_ERR_ARG, "the triad step is implemented for d = 3, 4");
    if (!(beta >= 0.0) || !std::isfinite(beta) || !std::isfinite(h))
      throw Error(TRG_ERR_ARG, "need finite beta >= 0 and finite h");
    init_ising_ctx(ctx(), beta, h, d);
  });
}

trg_status trg_init_clock(int d, int q, double beta, double h) {
  return guarded([&] {
    if (d != 3 && d != 4) throw Error(TRG_ERR_ARG, "the triad step is implemented for d = 3, 4");
    if (q < 2 || q > 8 || !(beta >= 0.0) || !std::isfinite(beta) || !std::isfinite(h))
      throw Error(TRG_ERR_ARG, "need 2 <= q <= 8, finite beta >= 0 and finite h");
    init_clock_ctx(ctx(), q, beta, h, d);
  });
}

trg_status trg_step(int axis, int D, int sketch_oversample) {
  return guarded([&] {
    Ctx &c = ctx();
    if (!c.init) throw Error(TRG_ERR_NOINIT, "no model initialised");
    if (axis < 0 || axis >= c.d || D < 1 || sketch_oversample < 0)
      throw Error(TRG_ERR_ARG, "need 0 <= axis < d, D >= 1, p >= 0");
    step_ctx(c, axis, D, sketch_oversample);
  });
}

trg_status trg_free_energy(double *f_per_site, double *lnZ_per_site) {
  return guarded([&] { free_energy_ctx(ctx(), f_per_site, lnZ_per_site); });
}

trg_status trg_magnetisation_impurity(double *m) {
  return guarded([&] {
    if (!m) throw Error(TRG_ERR_ARG, "m is NULL");
    *m = magnetisation_ctx(ctx());
  });
}

trg_status trg_set_params(int q_swap, int q_rho, unsigned long long seed, int precision) {
  return guarded([&] {
    if (q_swap < 1 || q_rho < 0 || precision < 0 || precision > TRG_PREC_OZ7)
      throw Error(TRG_ERR_ARG, "need q_swap >= 1, q_rho >= 0, precision in 0..8");
    Ctx &c = ctx();
    c.q_swap = q_swap;
    c.q_rho = q_rho;
    c.seed = seed;
    c.precision = precision;
  });
}

trg_status trg_atrg_init_ising(int d, double beta, double h) {
  return guarded([&] {
    if (d < 2 || d > 4) throw Error(TRG_ERR_ARG, "the ATRG comparator supports d = 2, 3, 4");
    if (!(beta >= 0.0) || !std::isfinite(beta) || !std::isfinite(h))
      throw Error(TRG_ERR_ARG, "need finite beta >= 0 and finite h");
    atrg_init_ising(ctx(), d, beta, h);
  });
}

trg_status trg_atrg_step(int axis, int D, int sketch_oversample) {
  return guarded([&] {
    AtrgState &a = atrg_state();
    if (!a.init) throw Error(TRG_ERR_NOINIT, "no ATRG model initialised");
    if (axis < 0 || axis >= a.d || D < 1 || sketch_oversample < 0)
      throw Error(TRG_ERR_ARG, "need 0 <= axis < d, D >= 1, p >= 0");
    Ctx &c = ctx();
    try {
      atrg_step_impl(c, axis, D, sketch_oversample);
    } catch (...) {
      cudaStreamSynchronize(c.stream);
      c.arena.reset();
      throw;
    }
  });
}

trg_status trg_atrg_free_energy(double *f_per_site, double *lnZ_per_site) {
  return guarded([&] { atrg_free_energy(ctx(), f_per_site, lnZ_per_site); });
}

trg_status trg_atrg_diag(double *log_c, double *min_gap, int *nsteps) {
  return guarded([&] {
    AtrgState &a = atrg_state();
    if (log_c) *log_c = a.last_logc;
    if (min_gap) *min_gap = a.last_gap;
    if (nsteps) *nsteps = a.nsteps;
  });
}

trg_status trg_set_impurity_pair(void) {
  return guarded([&] {
    Ctx &c = ctx();
    if (!c.init || !c.have_imp) throw Error(TRG_ERR_NOINIT, "no model initialised");
    if (c.nsteps != 0) throw Error(TRG_ERR_ARG, "the pair is placed before the first step");
    c.imp_pair = 1;
  });
}

trg_status trg_internal_energy(double *u) {
  return guarded([&] {
    Ctx &c = ctx();
    if (!u) throw Error(TRG_ERR_ARG, "u is NULL");
    if (c.imp_pair != 2)
      throw Error(TRG_ERR_NOINIT, "no merged impurity pair (trg_set_impurity_pair, then a step)");
    if (!c.ising) throw Error(TRG_ERR_ARG, "the pair gives the internal energy of the Ising model");
    *u = -(double)c.d * magnetisation_ctx(c);
  });
}

trg_status trg_set_bond_overspan(int r_bond) {
  return guarded([&] {
    if (r_bond < 1 || r_bond > 8) throw Error(TRG_ERR_ARG, "need 1 <= r_bond <= 8");
    ctx().r_bond = r_bond;
  });
}

trg_status trg_set_stream(void *cuda_stream) {
  return guarded([&] {
    Ctx &c = ctx();
    if (c.stream) TRG_CUDA(cudaStreamSynchronize(c.stream));
    c.stream = cuda_stream ? (cudaStream_t)cuda_stream : c.own_stream;
  });
}

trg_status trg_diag(double *log_c, double *min_gap, int *nsteps) {
  return guarded([&] {
    Ctx &c = ctx();
    if (log_c) *log_c = c.last_logc;
    if (min_gap) *min_gap = c.last_gap;
    if (nsteps) *nsteps = c.nsteps;
  });
}

trg_status trg_get_state(int which, int *dims_out, int *axes_out, double *host,
                         long long capacity) {
  return guarded([&] {
    Ctx &c = ctx();
    if (!c.init) throw Error(TRG_ERR_NOINIT, "no model initialised");
    if (which < 0 || which > 2 || !dims_out) throw Error(TRG_ERR_ARG, "bad which / dims_out");
    double *src = which == 0 ? c.phi : which == 1 ? c.psi : c.psi_imp;
    if (!src) throw Error(TRG_ERR_ARG, "factor not present");
    // a 3D state (d1, d2, d3, r) is reported as (d1, d2, d3, 1, r): the same memory layout
    for (int i = 0; i < 5; ++i)
      dims_out[i] = c.d == 4 ? (int)c.dims[i] : i < 3 ? (int)c.dims[i] : i == 3 ? 1 : (int)c.dims[3];
    if (axes_out)
      for (int i = 0; i < 4; ++i) axes_out[i] = c.axes[i];
    if (host) {
      int64_t n = prod(c.dims);
      if (capacity < n) throw Error(TRG_ERR_ARG, "host buffer too small");
      TRG_CUDA(cudaMemcpyAsync(host, src, n * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
      TRG_CUDA(cudaStreamSynchronize(c.stream));
    }
  });
}

trg_status trg_get_scalars(double *beta, double *logsum, int *nsteps) {
  return guarded([&] {
    Ctx &c = ctx();
    if (!c.init) throw Error(TRG_ERR_NOINIT, "no model initialised");
    double ls = 0.0;
    TRG_CUDA(cudaMemcpyAsync(&ls, c.dscal, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    TRG_CUDA(cudaStreamSynchronize(c.stream));
    if (beta) *beta = c.beta;
    if (logsum) *logsum = ls;
    if (nsteps) *nsteps = c.nsteps;
  });
}

trg_status trg_set_state(double beta, const int *dims, const double *phi, const double *psi,
                         const double *psi_imp, const int *axes, int nsteps, double logsum) {
  return guarded([&] {
    if (!dims || !phi || !psi || !axes || nsteps < 0) throw Error(TRG_ERR_ARG, "bad state");
    // everything is checked before the current state is released
    for (int i = 0; i < 5; ++i)
      if (dims[i] < 1) throw Error(TRG_ERR_ARG, "dims must be >= 1");
    // axes[3] = -1 with dims[3] = 1 marks a three-dimensional state (d1, d2, d3, r)
    const int dd = (axes[3] == -1 && dims[3] == 1) ? 3 : 4;
    int seen = 0;
    for (int i = 0; i < dd; ++i)
      if (axes[i] >= 0 && axes[i] < dd) seen |= 1 << axes[i];
    if (seen != (1 << dd) - 1)
      throw Error(TRG_ERR_ARG, "axes must be a permutation of 0..3 (or of 0..2 with axes[3] = -1)");
    if (!std::isfinite(beta) || !(beta >= 0.0) || !std::isfinite(logsum))
      throw Error(TRG_ERR_ARG, "need finite beta >= 0 and finite logsum");
    int64_t total = 1;
    for (int i = 0; i < 5; ++i) total *= dims[i];
    for (const double *buf : {phi, psi, psi_imp}) {
      if (!buf) continue;
      for (int64_t i = 0; i < total; ++i)
        if (!std::isfinite(buf[i]))
          throw Error(TRG_ERR_NONFINITE, "state buffer holds NaN or Inf at index " +
                                             std::to_string(i));
    }
    Ctx &c = ctx();
    ensure_ctx(c);
    TRG_CUDA(cudaStreamSynchronize(c.stream));
    free_state(c);
    c.d = dd;
    if (dd == 4) {
      c.dims.assign(dims, dims + 5);
    } else {
      c.dims.assign(dims, dims + 3);
      c.dims.push_back(dims[4]);
    }
    for (int i = 0; i < 4; ++i) c.axes[i] = axes[i];
    int64_t n = prod(c.dims);
    for (auto pr : {std::make_pair(&c.phi, phi), std::make_pair(&c.psi, psi),
                    std::make_pair(&c.psi_imp, psi_imp)}) {
      if (!pr.second) continue;
      TRG_CUDA(cudaMalloc(pr.first, n * sizeof(double)));
      TRG_CUDA(cudaMemcpyAsync(*pr.first, pr.second, n * sizeof(double), cudaMemcpyHostToDevice,
                               c.stream));
    }
    double sc[8] = {logsum, 1.0, 0, 0, 0, 0, 0, 0};
    TRG_CUDA(cudaMemcpyAsync(c.dscal, sc, sizeof(sc), cudaMemcpyHostToDevice, c.stream));
    TRG_CUDA(cudaMemsetAsync(c.dflag, 0, sizeof(int), c.stream));
    TRG_CUDA(cudaStreamSynchronize(c.stream));
    c.beta = beta;
    c.nsteps = nsteps;
    c.have_imp = psi_imp != nullptr;
    c.imp_pair = 0;
    c.ising = false;
    c.init = true;
  });
}

trg_status trg_finalize(void) {
  return guarded([&] {
    batch_free_all();
    Ctx &c = ctx();
    if (c.stream) cudaStreamSynchronize(c.stream);
    free_state(c);
    atrg_free(atrg_state());
    c.arena.release();
    if (c.dscal) cudaFree(c.dscal);
    if (c.dflag) cudaFree(c.dflag);
    if (c.d_sketch_cnt) cudaFree(c.d_sketch_cnt);
    if (c.col_x) cudaFree(c.col_x);
    if (c.col_t) cudaFree(c.col_t);
    for (void *q : {(void *)c.net.w, (void *)c.net.m, (void *)c.net.v, (void *)c.net.wb})
      if (q) cudaFree(q);
    c.net = SketchNet{};
    c.sketch_mode = 0;
    c.col_x = c.col_t = nullptr;
    c.col_cap = c.col_rows = c.col_dropped = 0;
    c.d_sketch_cnt = nullptr;
    c.dscal = nullptr;
    c.dflag = nullptr;
    if (c.own_stream) cudaStreamDestroy(c.own_stream);
    c.own_stream = nullptr;
    c.stream = nullptr;
  });
}

trg_status trg_step_timings(double *ms, int n) {
  return guarded([&] {
    Ctx &c = ctx();
    if (!ms || n < 0) throw Error(TRG_ERR_ARG, "bad timing buffer");
    for (int i = 0; i < n && i < Ctx::kPhases; ++i) ms[i] = c.phase_ms[i];
  });
}

// ------------------------------------------------------------ batched instances (S14)
trg_status trg_batch_create(int n, const int *model, const double *beta, const double *h,
                            const int *D, const int *p, const unsigned long long *seed,
                            int lanes, int q_swap, int q_rho, int precision) {
  return guarded([&] {
    if (n < 1 || !model || !beta || !h || !D || lanes < 1 || q_swap < 1 || q_rho < 0 ||
        precision < 0 || precision > TRG_PREC_OZ7)
      throw Error(TRG_ERR_ARG, "trg_batch_create: bad arguments");
    for (int i = 0; i < n; ++i)
      if (!(model[i] == 0 || (model[i] >= 2 && model[i] <= 8)) || !(beta[i] >= 0.0) ||
          !std::isfinite(beta[i]) || !std::isfinite(h[i]) || D[i] < 1 || (p && p[i] < 0))
        throw Error(TRG_ERR_ARG, "trg_batch_create: bad instance " + std::to_string(i));
    batch_free_all();
    auto B = std::make_unique<Batch>();
    TRG_CUDA(cudaGetDevice(&B->device));
    lanes = std::min(lanes, n);
    B->lanes.resize(lanes);
    for (Lane &L : B->lanes) {
      L.c = std::make_unique<Ctx>();
      L.c->q_swap = q_swap;
      L.c->q_rho = q_rho;
      L.c->precision = precision;
      ensure_ctx(*L.c);
      L.own_dscal = L.c->dscal;
      L.own_dflag = L.c->dflag;
    }
    B->inst.resize(n);
    for (int i = 0; i < n; ++i) {
      InstState &s = B->inst[i];
      s.model = model[i];
      s.beta = beta[i];
      s.h = h[i];
      s.D = D[i];
      s.p = p ? p[i] : 2 * D[i];
      s.seed = seed ? seed[i] : 0x5EED;
      TRG_CUDA(cudaMalloc(&s.dscal, 512 * sizeof(double)));
      TRG_CUDA(cudaMalloc(&s.dflag, sizeof(int)));
    }
    // Lanes hold instances of one bond dimension each (a lane's scratch arena grows to its
    // largest instance, so mixing sizes would give every lane the largest arena).  The
    // largest D, whose steps already fill the GPU, gets a quarter of the lanes; the
    // smaller, latency-bound sizes share the rest in proportion to their cost D^7 + 24^7;
    // within a group, instances go round-robin.  With fewer lanes than sizes: plain
    // longest-processing-time assignment over all instances.
    auto cost = [&](int i) { return std::pow((double)B->inst[i].D, 7.0) + std::pow(24.0, 7.0); };
    std::map<int, std::vector<int>, std::greater<int>> groups;
    for (int i = 0; i < n; ++i) groups[B->inst[i].D].push_back(i);
    const int G = (int)groups.size();
    if (lanes >= G) {
      std::vector<int> nl(G, 1);
      std::vector<double> gc(G, 0.0);
      int gi = 0;
      for (auto &kv : groups) {
        for (int i : kv.second) gc[gi] += cost(i);
        ++gi;
      }
      int spare = lanes - G;
      if (G > 1) {
        const int top = std::min(spare, std::max(0, lanes / 4 - 1));
        nl[0] += top;
        spare -= top;
        double rest = 0.0;
        for (int g = 1; g < G; ++g) rest += gc[g];
        for (int g = 1; g < G && spare > 0; ++g) {
          const int add = (int)std::floor(spare * gc[g] / rest);
          nl[g] += add;
        }
        int used = 0;
        for (int g = 0; g < G; ++g) used += nl[g];
        for (int g = 1; used < lanes; g = g % (G - 1) + 1, ++used) nl[g] += 1;
      } else {
        nl[0] = lanes;
      }
      int base = 0;
      gi = 0;
      for (auto &kv : groups) {
        const int k = std::min<int>(nl[gi], (int)kv.second.size());
        for (size_t j = 0; j < kv.second.size(); ++j)
          B->lanes[base + (int)(j % k)].members.push_back(kv.second[j]);
        base += nl[gi];
        ++gi;
      }
    } else {
      std::vector<int> order(n);
      for (int i = 0; i < n; ++i) order[i] = i;
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
      for (int i : order) {
        Lane *best = &B->lanes[0];
        for (Lane &L : B->lanes)
          if (L.cost < best->cost) best = &L;
        best->members.push_back(i);
        best->cost += cost(i);
      }
    }
    // lanes left without instances are dropped (their stream and buffers released)
    for (Lane &L : B->lanes) {
      if (!L.members.empty()) continue;
      if (L.own_dscal) cudaFree(L.own_dscal);
      if (L.own_dflag) cudaFree(L.own_dflag);
      if (L.c->d_sketch_cnt) cudaFree(L.c->d_sketch_cnt);
      if (L.c->own_stream) cudaStreamDestroy(L.c->own_stream);
    }
    B->lanes.erase(std::remove_if(B->lanes.begin(), B->lanes.end(),
                                  [](const Lane &L) { return L.members.empty(); }),
                   B->lanes.end());
    for (Lane &L : B->lanes) std::sort(L.members.begin(), L.members.end());
    g_batch = std::move(B);
    for_each_lane(*g_batch, [](Lane &L, InstState &s) {
      if (s.model == 0)
        init_ising_ctx(*L.c, s.beta, s.h);
      else
        init_clock_ctx(*L.c, s.model, s.beta, s.h);
    });
  });
}

trg_status trg_batch_step(int nsteps, double *wall_ms) {
  return guarded([&] {
    if (!g_batch) throw Error(TRG_ERR_NOINIT, "no batch");
    if (nsteps < 1) throw Error(TRG_ERR_ARG, "nsteps must be >= 1");
    const auto t0 = std::chrono::steady_clock::now();
    for_each_lane(*g_batch, [&](Lane &L, InstState &s) {
      for (int k = 0; k < nsteps; ++k) step_ctx(*L.c, L.c->nsteps % 4, s.D, s.p);
      TRG_CUDA(cudaStreamSynchronize(L.c->stream));
    });
    if (wall_ms)
      *wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                     .count();
  });
}

trg_status trg_batch_results(double *f, double *lnz, double *m, int *nsteps) {
  return guarded([&] {
    if (!g_batch) throw Error(TRG_ERR_NOINIT, "no batch");
    const int n = (int)g_batch->inst.size();
    std::vector<double> hf(n), hl(n), hm(n);
    std::vector<int> hn(n);
    for_each_lane(*g_batch, [&](Lane &L, InstState &s) {
      const int i = (int)(&s - g_batch->inst.data());
      free_energy_ctx(*L.c, &hf[i], &hl[i]);
      hm[i] = magnetisation_ctx(*L.c);
      hn[i] = L.c->nsteps;
    });
    for (int i = 0; i < n; ++i) {
      if (f) f[i] = hf[i];
      if (lnz) lnz[i] = hl[i];
      if (m) m[i] = hm[i];
      if (nsteps) nsteps[i] = hn[i];
    }
  });
}

trg_status trg_batch_lanes(int *lane_of, long long *scratch_bytes) {
  return guarded([&] {
    if (!g_batch) throw Error(TRG_ERR_NOINIT, "no batch");
    for (size_t l = 0; l < g_batch->lanes.size(); ++l) {
      for (int i : g_batch->lanes[l].members)
        if (lane_of) lane_of[i] = (int)l;
      if (scratch_bytes) scratch_bytes[l] = (long long)g_batch->lanes[l].c->arena.reserved();
    }
  });
}

trg_status trg_gu_wen_ratio(double *X) {
  return guarded([&] {
    if (!X) throw Error(TRG_ERR_ARG, "X is NULL");
    *X = gu_wen_ctx(ctx());
  });
}

trg_status trg_batch_gu_wen(double *X) {
  return guarded([&] {
    if (!g_batch) throw Error(TRG_ERR_NOINIT, "no batch");
    if (!X) throw Error(TRG_ERR_ARG, "X is NULL");
    std::vector<double> hx(g_batch->inst.size());
    for_each_lane(*g_batch, [&](Lane &L, InstState &s) {
      hx[&s - g_batch->inst.data()] = gu_wen_ctx(*L.c);
    });
    for (size_t i = 0; i < hx.size(); ++i) X[i] = hx[i];
  });
}

trg_status trg_batch_free(void) {
  return guarded([&] { batch_free_all(); });
}

// ------------------------------------------------------------ learned sketch (S15)
namespace {
struct DevF {  // device copy of a host float array, freed on scope exit
  float *p = nullptr;
  DevF(const float *h, int64_t n, cudaStream_t s) {
    TRG_CUDA(cudaMalloc(&p, std::max<int64_t>(n, 1) * sizeof(float)));
    if (h) TRG_CUDA(cudaMemcpyAsync(p, h, n * sizeof(float), cudaMemcpyHostToDevice, s));
  }
  ~DevF() {
    if (p) cudaFree(p);
  }
};
}  // namespace

trg_status trg_sketch_set_net(const float *params, long long n) {
  return guarded([&] {
    if (!params || n != kMlpParams) throw Error(TRG_ERR_ARG, "sketch net: need TRG_SKETCH_PARAMS floats");
    Ctx &c = ctx();
    ensure_ctx(c);
    mlp_set(c.net, params, c.stream);
    TRG_CUDA(cudaStreamSynchronize(c.stream));
  });
}

trg_status trg_sketch_get_net(float *params, long long n) {
  return guarded([&] {
    if (!params || n != kMlpParams) throw Error(TRG_ERR_ARG, "sketch net: need TRG_SKETCH_PARAMS floats");
    Ctx &c = ctx();
    ensure_ctx(c);
    mlp_get(c.net, params, c.stream);
  });
}

trg_status trg_sketch_forward(const float *X, long long rows, float *u, int bf16) {
  return guarded([&] {
    if (!X || !u || rows < 1) throw Error(TRG_ERR_ARG, "sketch forward: bad arguments");
    Ctx &c = ctx();
    if (!c.net.loaded) throw Error(TRG_ERR_NOINIT, "no sketch network loaded");
    ensure_ctx(c);
    DevF dX(X, rows * kMlpIn, c.stream), du(nullptr, rows, c.stream);
    mlp_forward(c.net, dX.p, rows, du.p, bf16 != 0, c.stream);
    TRG_CUDA(cudaMemcpyAsync(u, du.p, rows * sizeof(float), cudaMemcpyDeviceToHost, c.stream));
    TRG_CUDA(cudaStreamSynchronize(c.stream));
  });
}

trg_status trg_sketch_grad(const float *X, const float *t, long long rows, double *loss,
                           float *grad) {
  return guarded([&] {
    if (!X || !t || !grad || rows < 1) throw Error(TRG_ERR_ARG, "sketch grad: bad arguments");
    Ctx &c = ctx();
    if (!c.net.loaded) throw Error(TRG_ERR_NOINIT, "no sketch network loaded");
    ensure_ctx(c);
    DevF dX(X, rows * kMlpIn, c.stream), dt(t, rows, c.stream), dg(nullptr, kMlpParams, c.stream);
    const double L = mlp_grad(c.net, dX.p, dt.p, rows, dg.p, c.stream);
    TRG_CUDA(cudaMemcpyAsync(grad, dg.p, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost,
                             c.stream));
    TRG_CUDA(cudaStreamSynchronize(c.stream));
    if (loss) *loss = L;
  });
}

trg_status trg_sketch_train(const float *X, const float *t, long long rows, int epochs,
                            int batch, float lr, unsigned long long seed, double *loss) {
  return guarded([&] {
    if (!X || !t || rows < 1 || epochs < 1 || batch < 1 || !(lr > 0.f))
      throw Error(TRG_ERR_ARG, "sketch train: bad arguments");
    Ctx &c = ctx();
    if (!c.net.loaded) throw Error(TRG_ERR_NOINIT, "no sketch network loaded");
    ensure_ctx(c);
    DevF dX(X, rows * kMlpIn, c.stream), dt(t, rows, c.stream);
    const double L = mlp_train(c.net, dX.p, dt.p, rows, epochs, batch, lr, seed, c.stream);
    if (loss) *loss = L;
  });
}

trg_status trg_set_sketch_mode(int mode) {
  return guarded([&] {
    if (mode != 0 && mode != 1) throw Error(TRG_ERR_ARG, "sketch mode must be 0 or 1");
    Ctx &c = ctx();
    if (mode == 1 && !c.net.loaded) throw Error(TRG_ERR_NOINIT, "no sketch network loaded");
    c.sketch_mode = mode;
  });
}

trg_status trg_sketch_collect(long long capacity) {
  return guarded([&] {
    if (capacity < 0) throw Error(TRG_ERR_ARG, "negative capacity");
    Ctx &c = ctx();
    ensure_ctx(c);
    TRG_CUDA(cudaStreamSynchronize(c.stream));
    if (c.col_x) cudaFree(c.col_x);
    if (c.col_t) cudaFree(c.col_t);
    c.col_x = c.col_t = nullptr;
    c.col_cap = c.col_rows = c.col_dropped = 0;
    if (capacity == 0) return;
    if (cudaMalloc(&c.col_x, capacity * kMlpIn * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&c.col_t, capacity * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      throw Error(TRG_ERR_OOM, "collection buffer allocation failed");
    }
    c.col_cap = capacity;
  });
}

trg_status trg_sketch_fetch(float *X, float *t, long long capacity, long long *rows,
                            long long *dropped) {
  return guarded([&] {
    Ctx &c = ctx();
    if (rows) *rows = c.col_rows;
    if (dropped) *dropped = c.col_dropped;
    if (!X && !t) return;
    if (capacity < c.col_rows) throw Error(TRG_ERR_ARG, "fetch buffer too small");
    TRG_CUDA(cudaStreamSynchronize(c.stream));
    if (X && c.col_rows)
      TRG_CUDA(cudaMemcpy(X, c.col_x, c.col_rows * kMlpIn * sizeof(float), cudaMemcpyDeviceToHost));
    if (t && c.col_rows)
      TRG_CUDA(cudaMemcpy(t, c.col_t, c.col_rows * sizeof(float), cudaMemcpyDeviceToHost));
  });
}

trg_status trg_sketch_stats(long long *learned, long long *fallback, int reset) {
  return guarded([&] {
    Ctx &c = ctx();
    ensure_ctx(c);
    unsigned long long h[2] = {0, 0};
    TRG_CUDA(cudaStreamSynchronize(c.stream));
    TRG_CUDA(cudaMemcpy(h, c.d_sketch_cnt, sizeof(h), cudaMemcpyDeviceToHost));
    if (learned) *learned = (long long)h[0];
    if (fallback) *fallback = (long long)h[1];
    if (reset) TRG_CUDA(cudaMemset(c.d_sketch_cnt, 0, sizeof(h)));
  });
}

trg_status trg_gemm(int precision, int ta, int tb, long long M, long long N, long long K,
                    double alpha, const double *A, long long lda, const double *B,
                    long long ldb, double beta, double *C, long long ldc) {
  return guarded([&] {
    if (!A || !B || !C || M < 0 || N < 0 || K < 0 || precision < 0 ||
        precision > TRG_PREC_OZ7)
      throw Error(TRG_ERR_ARG, "bad gemm arguments");
    Ctx &c = ctx();
    ensure_ctx(c);
    const int64_t rA = ta ? K : M, rB = tb ? N : K;
    // one host matrix passed as both operands (a Gram) is uploaded once, so that the
    // device kernels see A == B
    const bool same = A == B && rA == rB && lda == ldb;
    Tensor dA = c.alloc({rA, lda}), dB = same ? dA : c.alloc({rB, ldb}), dC = c.alloc({M, ldc});
    TRG_CUDA(cudaMemcpyAsync(dA.p, A, rA * lda * 8, cudaMemcpyHostToDevice, c.stream));
    if (!same)
      TRG_CUDA(cudaMemcpyAsync(dB.p, B, rB * ldb * 8, cudaMemcpyHostToDevice, c.stream));
    TRG_CUDA(cudaMemcpyAsync(dC.p, C, M * ldc * 8, cudaMemcpyHostToDevice, c.stream));
    if (precision == TRG_PREC_FP64) {
      gemm_f64(ta, tb, M, N, K, alpha, dA.p, lda, 0, dB.p, ldb, 0, beta, dC.p, ldc, 0, 1, c.stream);
    } else if (is_digit_form(precision)) {
      ArenaScratch scr(c.arena);
      gemm_oz(ta, tb, M, N, K, alpha, dA.p, lda, 0, dB.p, ldb, 0, beta, dC.p, ldc, 0, 1,
              digits_of(precision), scr, c.stream);
    } else {
      ArenaScratch scr(c.arena);
      gemm_tc(ta, tb, M, N, K, alpha, dA.p, lda, 0, dB.p, ldb, 0, beta, dC.p, ldc, 0, 1,
              slices_of(precision), scr, c.stream, nullptr, precision == TRG_PREC_TF32X3);
    }
    TRG_CUDA(cudaMemcpyAsync(C, dC.p, M * ldc * 8, cudaMemcpyDeviceToHost, c.stream));
    TRG_CUDA(cudaStreamSynchronize(c.stream));
    c.arena.reset();
    if (tc_error_flag(true) | oz_error_flag(true))
      throw Error(TRG_ERR_TIMEOUT, "tensor-core GEMM wait timed out");
  });
}

trg_status trg_kernel_stats(double *out, int n, int reset) {
  return guarded([&] {
    if (n < 0 || (n > 0 && !out)) throw Error(TRG_ERR_ARG, "trg_kernel_stats: bad buffer");
    Ctx &c = ctx();
    const double v[13] = {c.k_ms[0], c.k_alg[0], c.k_pipe[0], (double)c.k_launches[0],
                          c.k_ms[1], c.k_alg[1], c.k_pipe[1], (double)c.k_launches[1],
                          c.k_ms[2], c.k_alg[2], c.k_pipe[2], (double)c.k_launches[2],
                          (double)g_kernel_launches.load()};
    for (int i = 0; i < std::min(n, 13); ++i) out[i] = v[i];
    if (reset) {
      for (int k = 0; k < 3; ++k) {
        c.k_ms[k] = c.k_alg[k] = c.k_pipe[k] = 0.0;
        c.k_launches[k] = 0;
      }
      g_kernel_launches.store(0);
    }
  });
}

trg_status trg_mem_stats(long long *in_use, long long *high_water, long long *reserved) {
  return guarded([&] {
    Ctx &c = ctx();
    if (in_use) *in_use = (long long)c.arena.in_use();
    if (high_water) *high_water = (long long)c.arena.high_water();
    if (reserved) *reserved = (long long)c.arena.reserved();
  });
}

const char *trg_last_error(void) { return g_err.c_str(); }

}  // extern "C"
