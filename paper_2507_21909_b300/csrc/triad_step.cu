// The triad-ATRG coarse-graining step (arXiv 2507.21909, Sec. II B and Appendix A) as a
// sequence of device kernels on one stream, in four dimensions (step_impl) and three
// (step3_impl), with the ILO width (Sec. II C) and the one-site and pair impurities
// (Sec. III D).  Shapes are structural (fixed by D, p and the step history), so the host
// reads back only small diagnostics inside a step (the singular values at the cuts, for
// the gap report) and the final norm and status.
#include "engine.h"

namespace trg {

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

// one step with the error context of the phase that failed
void step_ctx(Ctx &c, int axis, int D, int p) {
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

}  // namespace trg
