// The single-instance context (initial tensors, free energy, observables) and the C ABI
// of include/trg.h, except the batched sweep (batch.cu) and the plain-ATRG comparator
// (atrg.cu).
#include "engine.h"

namespace trg {

static thread_local std::string g_err = "ok";  // per host thread (batched lanes)
void set_last_error(const std::string &msg) { g_err = msg; }

// -------------------------------------------------------------------- init helpers
void ensure_ctx(Ctx &c) {
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

void free_state(Ctx &c) {
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

void init_ising_ctx(Ctx &c, double beta, double h, int d) {
  double cb = std::sqrt(std::cosh(beta)), sb = std::sqrt(std::sinh(beta));
  init_cp(c, beta, {cb, sb, cb, -sb}, 2, 2, {std::exp(h), std::exp(-h)}, {1.0, -1.0}, d);
  c.ising = true;
}

void init_clock_ctx(Ctx &c, int q, double beta, double h, int d) {
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
void free_energy_ctx(Ctx &c, double *f_per_site, double *lnZ_per_site) {
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

double magnetisation_ctx(Ctx &c) {
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
double gu_wen_ctx(Ctx &c) {
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

}  // namespace trg

// ================================================================== C ABI
using namespace trg;

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
    atrg_free_all();
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


trg_status trg_gu_wen_ratio(double *X) {
  return guarded([&] {
    if (!X) throw Error(TRG_ERR_ARG, "X is NULL");
    *X = gu_wen_ctx(ctx());
  });
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
              digits_of(precision), scr, c.stream, &c.timing);
    } else if (precision == TRG_PREC_TF32X3) {
      ArenaScratch scr(c.arena);
      gemm_tc(ta, tb, M, N, K, alpha, dA.p, lda, 0, dB.p, ldb, 0, beta, dC.p, ldc, 0, 1,
              slices_of(precision), scr, c.stream, &c.timing, true);
    } else {   // BF16x3 / x6 / x10: BF16 pieces on the persistent tensor-core GEMM
      ArenaScratch scr(c.arena);
      gemm_oz(ta, tb, M, N, K, alpha, dA.p, lda, 0, dB.p, ldb, 0, beta, dC.p, ldc, 0, 1,
              slices_of(precision), scr, c.stream, &c.timing, nullptr, nullptr, true);
    }
    TRG_CUDA(cudaMemcpyAsync(C, dC.p, M * ldc * 8, cudaMemcpyDeviceToHost, c.stream));
    TRG_CUDA(cudaStreamSynchronize(c.stream));
    c.collect_tc();   // the product kernel's device time into trg_kernel_stats
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
