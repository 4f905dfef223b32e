// Batched coupling sweep (many independent instances on concurrent lanes) and its C
// entry points (include/trg.h, trg_batch_*).
#include "engine.h"

namespace trg {

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

void batch_free_all() {
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

using namespace trg;

extern "C" {


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

}  // extern "C"
