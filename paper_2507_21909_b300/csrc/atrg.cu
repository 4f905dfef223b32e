// Plain ATRG, the paper's comparison method (eqs. makeG / makeH), and its C entry points
// (include/trg.h, trg_atrg_*).
#include "engine.h"

namespace trg {

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

void atrg_free_all() { atrg_free(atrg_state()); }

}  // namespace trg

using namespace trg;

extern "C" {


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

}  // extern "C"
