// Building blocks of the coarse-graining step (declared in engine.h): GEMM routing,
// shared digit planes, tensor helpers, decompositions, the sliced coarse contraction.
#include "engine.h"

namespace trg {

Ctx &ctx() {
  static Ctx c;
  return c;
}

int slices_of(int precision) {
  return precision == TRG_PREC_BF16X3 || precision == TRG_PREC_TF32X3 ? 2
         : precision == TRG_PREC_BF16X6                              ? 3
                                                                     : 4;
}

bool is_digit_form(int precision) {
  return (precision >= TRG_PREC_OZ4 && precision <= TRG_PREC_OZ6) || precision == TRG_PREC_OZ7;
}

int digits_of(int precision) { return precision == TRG_PREC_OZ7 ? 7 : precision; }

Route route_of(const Ctx &c, int64_t M, int64_t N, int64_t K) {
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

const OzOperand *cached_planes(const Ctx &c, const double *X, int64_t rows, int64_t K,
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
void gemm(Ctx &c, bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha,
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
    if (!cheap && c.precision == TRG_PREC_TF32X3)
      gemm_tc(ta, tb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch,
              slices_of(c.precision), scr, c.stream, &c.timing, true);
    else   // BF16 pieces on the persistent tensor-core GEMM (128 x 256 tiles, FP32 sums)
      gemm_oz(ta, tb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch,
              cheap ? 3 : slices_of(c.precision), scr, c.stream, &c.timing, nullptr, nullptr,
              true);
    c.arena.release(mk);
  } else {
    gemm_f64(ta, tb, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, c.stream,
             c.b_upper && !tb);
  }
}


// ------------------------------------------------------------------ tensor helpers
Tensor copy(Ctx &c, const Tensor &a) {
  Tensor t = c.alloc(a.dims);
  TRG_CUDA(cudaMemcpyAsync(t.p, a.p, a.size() * sizeof(double), cudaMemcpyDeviceToDevice,
                           c.stream));
  return t;
}

Tensor permuted(Ctx &c, const Tensor &a, const std::vector<int> &perm) {
  std::vector<int64_t> d(perm.size());
  for (size_t i = 0; i < perm.size(); ++i) d[i] = a.dims[perm[i]];
  Tensor t = c.alloc(d);
  permute(a.p, t.p, a.dims, perm, c.stream);
  return t;
}


// C = op(A) op(B) for 2-D views
Tensor mm(Ctx &c, const Tensor &A, const Tensor &B, bool ta, bool tb) {
  int64_t M = ta ? A.dims[1] : A.dims[0], K = ta ? A.dims[0] : A.dims[1];
  int64_t Kb = tb ? B.dims[1] : B.dims[0], N = tb ? B.dims[0] : B.dims[1];
  if (K != Kb) throw Error(TRG_ERR_ARG, "mm: inner dimensions differ");
  Tensor C = c.alloc({M, N});
  gemm(c, ta, tb, M, N, K, 1.0, A.p, A.dims[1], 0, B.p, B.dims[1], 0, 0.0, C.p, N, 0, 1);
  return C;
}


// first `ncols` columns of U (rows x ucols) applied from the right: C = Q U[:, :ncols]
Tensor mm_cols(Ctx &c, const Tensor &Q, const Tensor &U, int64_t ncols) {
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
Tensor contract(Ctx &c, const std::string &spec, const Tensor &A, const Tensor &B,
                       Tensor *into, double beta_into) {
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

void scale_last(Ctx &c, Tensor &t, const double *v, int mode,
                       const double *vmax, double tol) {
  int64_t n = t.dims.back();
  scale_axis(t.p, t.size(), 1, n, v, mode, vmax, tol, c.stream);
}


// ------------------------------------------------------------- decompositions
// Orthonormal basis of range(Y) (n x w) by shifted CholeskyQR3 (Fukaya et al. 2020):
// each pass Q <- Q R^{-1} keeps the span, so the span error stays O(eps * cond(Y)) like
// Householder QR; directions at the rounding level come out as zero columns.
Tensor orth_sc(Ctx &c, const Tensor &Y) {
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

std::pair<Tensor, Tensor> orth_qr(Ctx &c, const Tensor &Y) {
  Crit cr(c);
  Tensor Q = orth_sc(c, Y);
  Tensor R = mm(c, Q, Y, true, false);
  return {Q, R};
}

FoldedQR orth_qr_folded(Ctx &c, const Tensor &Y) {
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

Svd svd_small(Ctx &c, const Tensor &A) {
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

Tensor transpose2(Ctx &c, const Tensor &a) { return permuted(c, a, {1, 0}); }

Tensor identity(Ctx &c, int64_t n) {
  Tensor t = c.alloc({n, n});
  fill_identity(t.p, n, n, c.stream);
  return t;
}


// orthonormal basis of range(rho^(q+1) Omega)
Tensor range_from(Ctx &c, const Tensor &rho, const Tensor &Om, int q) {
  Tensor Q = orth_sc(c, mm(c, rho, Om, false, false));
  for (int i = 0; i < q; ++i) Q = orth_sc(c, mm(c, rho, Q, false, false));
  return Q;
}


// orthonormal basis (n x chi) of range(rho^(q+1) Omega), or the identity if chi >= n
Tensor rsvd_sym(Ctx &c, const Tensor &rho, int64_t chi, int q, uint64_t key) {
  int64_t n = rho.dims[0];
  if (chi >= n) return identity(c, n);
  Tensor Om = c.alloc({n, chi});
  fill_gaussian(Om.p, n, chi, key, c.stream);
  return range_from(c, rho, Om, q);
}


// nb independent shifted CholeskyQR3 (as orth_sc) on stacked Y [nb][rows][w]: every
// Gram, Cholesky and product of a pass is one batched launch
Tensor orth_sc_batched(Ctx &c, const Tensor &Y) {
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
Tensor rsvd_sym_batched(Ctx &c, const Tensor &rho, int64_t chi, int q,
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
Tensor range_from_factor(Ctx &c, const Tensor &F, const Tensor &Om, int q) {
  auto apply = [&](const Tensor &V) {
    Tensor Z = mm(c, F, V, true, false);          // F^T V   (m x chi)
    return mm(c, F, Z, false, false);             // F F^T V (n x chi)
  };
  Tensor Q = orth_sc(c, apply(Om));
  for (int i = 0; i < q; ++i) Q = orth_sc(c, apply(Q));
  return Q;
}


// F's digit planes for both products of the range finder (F^T V and F Z), split once
void share_factor(PlaneScope &ps, const Tensor &F, int64_t chi) {
  const int64_t n = F.dims[0], m = F.dims[1];
  ps.share(F.p, true, true, m, chi, n, m);    // F^T V: op(A) = F^T (m x n)
  ps.share(F.p, true, false, n, chi, m, m);   // F Z:   op(A) = F   (n x m)
}

Tensor rsvd_factor(Ctx &c, const Tensor &F, int64_t chi, int q, uint64_t key) {
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
Tensor rsvd_factor_batched(Ctx &c, const Tensor &Fs, int64_t chi, int q,
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
void probe_residual2(Ctx &c, const Tensor &Q, const Tensor &P, double *out) {
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
Tensor range_factor_full(Ctx &c, const Tensor &F, int64_t da, int64_t db, int64_t chi,
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
Tensor gram_root(Ctx &c, const Tensor &rho, int64_t chi, int q, uint64_t key) {
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
std::pair<Tensor, Tensor> squeezer_from_roots(Ctx &c, const Tensor &R1, const Tensor &R2,
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
std::pair<Tensor, Tensor> squeezer(Ctx &c, const Tensor &rf, const Tensor &rb, int64_t D,
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
Tensor gram_root_batched(Ctx &c, const Tensor &rho, int64_t chi, int q,
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
int64_t t_slice(int64_t kt, int64_t per_t_elems) {
  int64_t budget = int64_t(1) << 30;
  const std::string e = study_opt("slice_mb");
  if (!e.empty()) budget = std::max<int64_t>(1, atoll(e.c_str())) << 20;
  const int64_t per_t = std::max<int64_t>(per_t_elems * (int64_t)sizeof(double), 1);
  return std::max<int64_t>(1, std::min<int64_t>(kt, budget / per_t));
}


// Phi[t,k2,k3,k4,g] = sum (E F M4)(I J M2 M3)   (eq. makeMG), sliced over t.  Operands
// that every slice reuses are put in GEMM order once (F as (al q4 | kX g)); each slice's
// EM comes out in GEMM order, and its result is permuted straight into Phi's rows.
Tensor contract_upper(Ctx &c, const Tensor &E, const Tensor &F, const Tensor &I_,
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
Tensor theta_lower(Ctx &c, const Tensor &K_, const Tensor &L_, const Tensor &N2,
                          const Tensor &N3) {
  Tensor KN2 = contract(c, "bck,bBm->ckBm", K_, N2);              // (c kY B k2)
  Tensor LN3 = contract(c, "BCl,cCn->Blcn", L_, N3);              // (B kD c k3)
  return contract(c, "ckBm,Blcn->lkmn", KN2, LN3);                // (kD kY k2 k3)
}


// Psi (eq. makeMH), sliced over its first leg w
Tensor contract_lower(Ctx &c, const Tensor &G, const Tensor &H, const Tensor &K_,
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
Tensor contract_lower_sum(Ctx &c, const Tensor &G1, const Tensor &H1, const Tensor &G2,
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
void replace_state(double *&dst, int64_t old_size, const Tensor &src, cudaStream_t s) {
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
void rotate(Ctx &c, int axis) {
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

}  // namespace trg
