#!/usr/bin/env python3
"""Benchmark: triad-ATRG RG steps/s at D=48 on the 4D Ising model, one B300.

A "step" is one full coarse-graining step of the triad-ATRG method (re-split, bond
swap, triad isometries, triads, squeezers, coarse contraction, impurity, normalisation)
on a steady-state D=48 tensor (all legs and the bond at D, p = 2D).  The tensor is grown
from the Boltzmann-weight initial tensor by the method itself (untimed), then W warm-up
and K timed steps continue the RG flow.  Inputs (D^5 factors, 2 GB each in FP64) are
far larger than the 126 MB L2, so no flush is needed between steps.

Default: the mixed form "oz5": every bulk GEMM runs on the tcgen05 tensor cores as exact
products of 5 seven-bit digits per row (15 BF16 products, exact FP32 chunks summed in
int64), FP64 for the small decompositions and the log-norm sum; it keeps ΔF/F <= 1e-8.
Prints one JSON line.  Under torchrun every rank runs an independent replica (the method does not
shard; "replicas only") and rank 0 prints the whole-job value.

--impl reference times the FP64 CPU oracle (test infrastructure) on a bounded sample
of the same workload on the host cores.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "triad-ATRG RG steps/s at D=48 4D Ising (mixed vs FP64 form, ΔF/F ≤1e-8)"
PREC = {"fp64": 0, "bf16x3": 1, "bf16x6": 2, "bf16x10": 3, "oz4": 4, "oz5": 5, "oz6": 6,
        "tf32x3": 7, "oz7": 8}


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--D", type=int, default=48)
    ap.add_argument("--precision", default="oz5", choices=list(PREC))
    ap.add_argument("--fp64-form-steps", type=int, default=0,
                    help="also time this many steady-state steps of the FP64 form (slow)")
    ap.add_argument("--precision-steps", type=int, default=6,
                    help="N > 0: also run N steps of the FP64 form and of the mixed form at "
                         "the bench's D from the initial tensor; report dF/F after every "
                         "step and the FP64 form's rate from its last (full-size) step")
    ap.add_argument("--also-forms", default="",
                    help="comma-separated precision forms also compared against the FP64 "
                         "form in the size-level precision check (e.g. oz4,oz7,tf32x3)")
    ap.add_argument("--sensitivity", default="",
                    help="comma-separated D: for each form of --precision and --also-forms, "
                         "the relative change of f after each of --precision-steps steps when "
                         "beta changes by a relative 1e-14 (the run's own conditioning)")
    ap.add_argument("--sensitivity-eps", type=float, default=1e-14,
                    help="relative change of beta in --sensitivity (2e-16: one ulp of 0.1497)")
    ap.add_argument("--beta", type=float, default=0.1497)
    ap.add_argument("--sketch", default="gaussian", choices=["gaussian", "learned"],
                    help="learned: train the sketch network on rows collected from plain "
                         "runs (D = 16..32), then time the learned-sketch form")
    ap.add_argument("--batch", type=int, default=0,
                    help="N > 0: time a coupling sweep of N instances (Ising and Z3 clock "
                         "1:1, beta ~ U[0.14, 0.16], h ~ U[0, 0.01], D ~ U{16,24,32,40}) "
                         "on concurrent lanes instead of the single D=48 step")
    ap.add_argument("--lanes", type=int, default=8)
    ap.add_argument("--compare-atrg", default="",
                    help="comma-separated D list: time the triad step against the plain "
                         "ATRG step (4D Ising, same precision and sketches) at each D "
                         "instead of the single D=48 step; ATRG holds D^8 tensors, so D <= 12")
    ap.add_argument("--triad-d", default="",
                    help="with --compare-atrg: further D (comma-separated) at which only the "
                         "triad step is timed (ATRG holds D^8 tensors beyond D = 12)")
    ap.add_argument("--r-bond", type=int, default=1,
                    help="ILO form: bond lines overspanned to r_bond D (1 = plain method)")
    ap.add_argument("--gemm", default="",
                    help="M,N,K: time one contraction-engine GEMM C = A B of that shape (host "
                         "FP64 buffers through trg_gemm, --precision) instead of the step; "
                         "for kernel profiles")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision-check", action="store_true")
    return ap.parse_args()


def workload(a):
    w = {"workload": f"triad-ATRG coarse-graining step, 4D Ising, beta={a.beta}, h=0, "
                        f"D={a.D}, p=2D (chi=3D), q_swap=4, q_rho=4, steady state",
            "D": a.D, "sketch_oversample": 2 * a.D, "precision": a.precision,
            "l2_flush": "none: inputs (D^5 FP64 factors) far larger than L2"}
    if a.r_bond > 1:
        w["workload"] += f", ILO r_bond={a.r_bond} (bond lines {a.r_bond * a.D})"
        w["r_bond"] = a.r_bond
    return w


# ----------------------------------------------------------------- oracle sample
def sample_sizes(D):
    """Bond dimensions of the oracle sample: the target D itself when a whole oracle step
    there takes seconds, else two smaller D whose whole steps take 3-15 s each."""
    return (D,) if D <= 20 else (16, 20)


class OracleSample:
    """Whole steps of the FP64 CPU oracle (every phase: re-split, bond swap, triad
    isometries, triads, squeezers, coarse contraction, impurity, norm) on 4D Ising states
    grown to the sample bond dimensions (growth untimed).  step() times one more step at
    each sample D; per_step(D_target) is the time of one step at D_target, taken directly
    when D_target is sampled, else extrapolated as c D^e with c, e fitted to the medians of
    the two sample sizes (the method's cost grows as D^7 at large D; the exponent fitted
    at small D is stated with the result)."""

    def __init__(self, D, beta, r_bond=1):
        from oracle import trg_oracle as O
        self.O = O
        self.sizes = sample_sizes(D)
        self.r_bond = r_bond
        self.st, self.n, self.times = {}, {}, {d: [] for d in self.sizes}
        for d in self.sizes:
            st = O.init_ising(4, beta, 0.0)
            n = 0
            while n < 4 or any(x != d for x in st.phi.shape[:4]):
                O.step(st, n % 4, d, 2 * d, 4, 4, 0x5EED, r_bond=r_bond)
                n += 1
            self.st[d], self.n[d] = st, n

    def step(self):
        t_all = 0.0
        for d in self.sizes:
            t0 = time.time()
            self.O.step(self.st[d], self.n[d] % 4, d, 2 * d, 4, 4, 0x5EED, r_bond=self.r_bond)
            dt = time.time() - t0
            self.n[d] += 1
            self.times[d].append(dt)
            t_all += dt
        return t_all

    def per_step(self, D):
        med = {d: statistics.median(v) for d, v in self.times.items() if v}
        if D in med:
            return med[D], None
        (d0, t0), (d1, t1) = sorted(med.items())
        e = math.log(t1 / t0) / math.log(d1 / d0)
        return t1 * (D / d1) ** e, e

    def describe(self, D):
        per, e = self.per_step(D)
        med = {d: round(statistics.median(v), 3) for d, v in self.times.items() if v}
        if e is None:
            return (f"whole oracle steps (all phases) at D={D}, p=2D on a grown 4D Ising state; "
                    f"median {med[D]:.3f} s over {len(self.times[D])} steps")
        return (f"whole oracle steps (all phases) at D={list(med)} (p=2D, grown 4D Ising "
                f"states), median s/step {med}; extrapolated to D={D} as c D^e with the "
                f"fitted e={e:.2f}: {per:.0f} s/step")


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t0 = time.time()
    smp = OracleSample(a.D, a.beta, a.r_bond)       # growth: untimed set-up
    for _ in range(a.warmup):
        smp.step()
    for d in smp.times:
        smp.times[d].clear()
    walls = [smp.step() for _ in range(max(a.steps, 1))]
    per, _ = smp.per_step(a.D)
    v = 1.0 / per
    cores = os.cpu_count()
    sample = smp.describe(a.D)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "RG steps/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        # wall time of one reference step as run (the sample), not of a D=48 step
        "ms_per_step": 1e3 * statistics.mean(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload(a),
        "cpu_baseline": {"value": v, "unit": "RG steps/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "RG steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": time.time() - t0}), flush=True)


# ------------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------- ours
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["bf16_tflops_sustained"], "measured (sustained bf16, MEASURED_PEAKS.json)"
    except Exception:
        return 1400.0, "fallback (sustained bf16 estimate)"


def run_f(trg, prec, D, nsteps):
    trg.trg_set_params(4, 4, 0x5EED, prec)
    trg.trg_init_ising(4, 0.1497, 0.0)
    for n in range(nsteps):
        trg.trg_step(n % 4, D, 2 * D)
    return trg.trg_free_energy()[0]


def net_dict(flat):
    """Flat network parameters (library order) -> the oracle's dictionary."""
    import numpy as np
    shapes = (("W1", (256, 5)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)),
              ("W3", (1, 256)), ("b3", (1,)))
    out, o = {}, 0
    for k, sh in shapes:
        n = int(np.prod(sh))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(sh)
        o += n
    return out


def train_sketch(trg, prec, budget_s=120.0, pairs_goal=2000):
    """Collect (inputs, leverage target) rows from plain runs (the bench's precision form)
    at D = 16, 24, 32 and several couplings, then train the sketch network on the GPU."""
    import numpy as np
    t0 = time.time()
    trg.trg_set_sketch_mode(0)
    trg.trg_sketch_collect(4_000_000)
    pairs, runs = 0, 0
    for D in (16, 24, 32, 16, 24, 32, 16, 24):
        for beta in (0.145, 0.15, 0.155):
            trg.trg_set_params(4, 4, 0x5EED + runs, prec)
            trg.trg_init_ising(4, beta, 0.0)
            for n in range(10):
                trg.trg_step(n % 4, D, 2 * D)
            runs += 1
            rows = trg.trg_sketch_fetch()[0].shape[0]
            pairs = rows // (2 * D)      # rows per range finder = d_a + d_b ~ 2D
            if pairs >= pairs_goal or time.time() - t0 > budget_s:
                break
        if pairs >= pairs_goal or time.time() - t0 > budget_s:
            break
    X, t, _ = trg.trg_sketch_fetch()
    trg.trg_sketch_collect(0)
    t1 = time.time()
    rng = np.random.default_rng(0)
    init = np.concatenate([rng.standard_normal(256 * 5) * np.sqrt(2 / 5), np.zeros(256),
                           rng.standard_normal(256 * 256) * np.sqrt(2 / 256), np.zeros(256),
                           rng.standard_normal(256) * np.sqrt(1 / 256), np.zeros(1)])
    trg.trg_sketch_set_net(init.astype(np.float32))
    loss = trg.trg_sketch_train(X, t, epochs=40, batch=512, lr=1e-3, seed=1)
    t2 = time.time()
    return {"runs": runs, "rows": int(X.shape[0]), "pairs_approx": int(pairs),
            "collect_s": t1 - t0, "train_s": t2 - t1, "train_loss": loss,
            "target_var": float(np.var(t)), "epochs": 40, "batch": 512}


def learned_gain(trg):
    """Oracle-judged effect of the trained network: median over the range finders of a
    D = 10 oracle run (beta 0.1555, not in the training set) of the probe-residual ratio
    learned / Gaussian with one-pass range finders (q_rho = 0)."""
    import numpy as np
    from oracle import trg_oracle as O
    p = net_dict(trg.trg_sketch_get_net())
    st = O.run("ising", 4, 0.1555, 0.0, 10, 20, 6, q_rho=0, mlp=p)
    r = [v["r_learned"] / v["r_plain"] for d in st.diag for v in d.get("sketch", {}).values()
         if v.get("r_plain", 0) > 0]
    return float(np.median(r)) if r else None


def precision_check(trg, prec, mlp=None, r_bond=1):
    """dF/F of the mixed form at small D: against the FP64 CPU oracle at D=14 (16 steps;
    no near-degenerate truncation there) and against this library's FP64 form at D=24
    (12 steps; the FP64 form matches the oracle to 1e-10).  With a sketch network the
    oracle runs the same learned sketch."""
    from oracle import trg_oracle as O
    st = O.run("ising", 4, 0.1497, 0.0, D=14, p=28, nsteps=16, q_swap=4, q_rho=4, mlp=mlp,
               r_bond=r_bond)
    f_or = O.free_energy(st)[0]
    f14 = run_f(trg, prec, 14, 16)
    f24_64 = run_f(trg, 0, 24, 12)
    f24 = run_f(trg, prec, 24, 12)
    return {"vs_oracle_D14_16steps": abs(f14 - f_or) / abs(f_or),
            "vs_fp64_form_D24_12steps": abs(f24 - f24_64) / abs(f24_64)}


def precision_at_size(trg, prec, D, beta, nsteps, stream, others=()):
    """The headline's accuracy gate and its speed-up at the bench's own D: nsteps steps of
    the FP64 form and of the mixed form from the same initial tensor (same sketches), the
    relative free-energy difference after every step, and the FP64 form's rate from its
    last step (full size from the fifth step on; CUDA events on the library stream).
    `others`: further precision forms compared against the same FP64 run."""
    import torch
    out = {}
    for pr in (0, prec) + tuple(others):
        trg.trg_set_params(4, 4, 0x5EED, pr)
        trg.trg_init_ising(4, beta, 0.0)
        fs, ms, gaps = [], [], []
        for k in range(nsteps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            trg.trg_step(k % 4, D, 2 * D)
            e1.record(stream)
            fs.append(trg.trg_free_energy()[0])
            gaps.append(trg.trg_diag()[1])
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        out[pr] = (fs, ms, list(trg.trg_state_dims(0)), gaps)
    f64, ms64, dims64, gaps64 = out[0]
    fmx, msmx, _, _ = out[prec]
    per = [abs(x - y) / abs(y) for x, y in zip(fmx, f64)]
    res = {"steps": nsteps, "per_step": per, "max": max(per),
           "fp64_form_ms_last_step": ms64[-1], "mixed_form_ms_last_step": msmx[-1],
           "last_step_input_dims": dims64, "fp64_form_steps_per_s": 1e3 / ms64[-1],
           # smallest relative singular-value gap at the bond-swap and squeezer cuts of
           # each FP64-form step: a near-degenerate cut amplifies rounding differences
           "fp64_form_min_gap_per_step": gaps64}
    names = {v: k for k, v in PREC.items()}
    for pr in others:
        fo, mso, _, _ = out[pr]
        po = [abs(x - y) / abs(y) for x, y in zip(fo, f64)]
        res.setdefault("other_forms", {})[names[pr]] = {
            "per_step": po, "max": max(po), "ms_last_step": mso[-1]}
    return res


def fp64_form_rate(trg, D, nsteps, beta):
    """Steady-state steps/s of the FP64 form (every GEMM on the FP64 CUDA cores)."""
    import torch
    trg.trg_set_params(4, 4, 0x5EED, 0)
    trg.trg_init_ising(4, beta, 0.0)
    n = 0
    while n < 12:
        trg.trg_step(n % 4, D, 2 * D)
        n += 1
        dims = trg.trg_state_dims(0)
        if all(x == D for x in dims[:4]) and n >= 4:
            break
    torch.cuda.synchronize()
    t = time.time()
    for _ in range(nsteps):
        trg.trg_step(n % 4, D, 2 * D)
        n += 1
    torch.cuda.synchronize()
    return nsteps / (time.time() - t)


def run_batch(a):
    """Coupling sweep (batching variant): instance-steps/s of N instances on lanes."""
    import numpy as np
    import torch
    import paper_2507_21909_b300 as trg
    rng = np.random.default_rng(1)
    n = a.batch
    model = [0 if i % 2 == 0 else 3 for i in range(n)]
    beta = rng.uniform(0.14, 0.16, n)
    h = rng.uniform(0.0, 0.01, n)
    D = rng.choice([16, 24, 32, 40], n)
    prec = PREC[a.precision]
    t0 = time.time()
    trg.trg_batch_create(model, beta, h, D, lanes=a.lanes, q_swap=4, q_rho=4, precision=prec)
    grow_ms = trg.trg_batch_step(5)            # every leg reaches its D within 5 steps
    warm_ms = trg.trg_batch_step(max(a.warmup - 2, 1))
    clk = Clocks(0)
    clk.start()
    torch.cuda.synchronize()
    ms = trg.trg_batch_step(a.steps)
    clocks = clk.stop()
    t_job = time.time() - t0
    res = trg.trg_batch_results(n)
    lane_of, scratch = trg.trg_batch_lanes(n, min(a.lanes, n))
    trg.trg_batch_free()
    value = n * a.steps / (ms / 1e3)
    line = {
        "metric": "batched triad-ATRG instance-steps/s (coupling sweep)", "value": value,
        "unit": "instance-steps/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if prec else "f64", "data": "synthetic",
        "config": {"workload": f"coupling sweep of {n} instances, Ising:Z3 = 1:1, beta ~ "
                               "U[0.14,0.16], h ~ U[0,0.01], D ~ U{16,24,32,40}, p = 2D, "
                               "seed 1", "instances": n, "lanes": int(min(a.lanes, n)),
                   "precision": a.precision,
                   "l2_flush": "none: per-instance state far larger than L2"},
        "e2e": {"value": n * (5 + max(a.warmup - 2, 1) + a.steps) / t_job,
                "unit": "instance-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "region": "whole job from the host: create (H2D of every T0), 5 growth, "
                          "warm-up and timed steps"},
        "clocks": clocks,
        "per_D_instances": {int(d): int((D == d).sum()) for d in (16, 24, 32, 40)},
        "lane_scratch_gb": [round(x / 2 ** 30, 2) for x in scratch],
        "growth_ms": grow_ms, "finite": bool(np.all(np.isfinite(res["lnz"]))),
    }
    print(json.dumps(line), flush=True)


def run_sensitivity(a):
    """Conditioning of the step sequence: f after each step from beta and from
    beta (1 + eps), same sketches, per form and D; with the smallest relative gap at the
    step's cuts.  A perturbation of eps changes f directly by about eps, so a larger
    relative change measures how much the steps amplify differences at the rounding level
    (eps = 2e-16 is one unit in the last place of 0.1497: two FP64 programs that round
    differently disagree by about that much)."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import paper_2507_21909_b300 as trg
    stream = torch.cuda.Stream()
    trg.trg_set_stream(stream.cuda_stream)
    forms = [a.precision] + [x for x in a.also_forms.split(",") if x.strip()]
    nsteps = a.precision_steps if a.precision_steps > 0 else 6
    rows = []
    for D in [int(v) for v in a.sensitivity.split(",") if v.strip()]:
        for name in forms:
            runs = []
            for beta in (a.beta, a.beta * (1 + a.sensitivity_eps)):
                trg.trg_set_params(4, 4, 0x5EED, PREC[name])
                trg.trg_init_ising(4, beta, 0.0)
                fs, gaps = [], []
                for k in range(nsteps):
                    trg.trg_step(k % 4, D, 2 * D)
                    fs.append(trg.trg_free_energy()[0])
                    gaps.append(trg.trg_diag()[1])
                torch.cuda.synchronize()
                runs.append((fs, gaps))
            (f0, g0), (f1, _) = runs
            rows.append({"D": D, "form": name,
                         "df_rel_per_step": [abs(x - y) / abs(x) for x, y in zip(f0, f1)],
                         "min_cut_gap_per_step": [g if math.isfinite(g) else None for g in g0]})
    print(json.dumps({"metric": "relative change of f per step for a relative change of beta",
                      "unit": "1", "steps": nsteps, "beta": a.beta,
                      "beta_rel_change": a.sensitivity_eps,
                      "config": {"workload": "4D Ising, h=0, p=2D, q_swap=4, q_rho=4"},
                      "rows": rows}), flush=True)


def run_compare_atrg(a):
    """Steady-state ms per step of the triad step and of the plain ATRG step (the paper's
    comparison, Sec. III C) at each D, 4D Ising, one GPU.  Each method grows its tensor
    for 8 steps (every leg reaches D), then a.warmup untimed and a.steps timed steps."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import paper_2507_21909_b300 as trg
    stream = torch.cuda.Stream()
    trg.trg_set_stream(stream.cuda_stream)
    prec = PREC[a.precision]
    rows = []
    both = [int(v) for v in a.compare_atrg.split(",") if v.strip()]
    only = [int(v) for v in a.triad_d.split(",") if v.strip()]
    for D in both + only:
        row = {"D": D, "p": 2 * D}
        methods = [("triad", lambda: trg.trg_init_ising(4, a.beta, 0.0), trg.trg_step)]
        if D in both:
            methods.append(("atrg", lambda: trg.trg_atrg_init_ising(4, a.beta, 0.0),
                            trg.trg_atrg_step))
        for name, init, step in methods:
            trg.trg_set_params(4, 4, 0x5EED, prec)
            init()
            n = 0
            for _ in range(8 + a.warmup):
                step(n % 4, D, 2 * D)
                n += 1
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(a.steps):
                step(n % 4, D, 2 * D)
                n += 1
            ev1.record(stream)
            torch.cuda.synchronize()
            row[f"{name}_ms_per_step"] = ev0.elapsed_time(ev1) / a.steps
        row["f_triad"] = trg.trg_free_energy()[0]
        if D in both:
            row["f_atrg"] = trg.trg_atrg_free_energy()[0]
            row["atrg_over_triad"] = row["atrg_ms_per_step"] / row["triad_ms_per_step"]
        rows.append(row)
    # power-law exponents of the step time in D (least squares on log-log), per method
    import numpy as np
    fits = {}
    for name in ("triad", "atrg"):
        pts = [(r["D"], r[name + "_ms_per_step"]) for r in rows if name + "_ms_per_step" in r]
        if len(pts) >= 2:
            x = np.log([d for d, _ in pts])
            y = np.log([t for _, t in pts])
            fits[name] = float(np.polyfit(x, y, 1)[0])
    print(json.dumps({
        "metric": "ms per RG step, triad-ATRG vs plain ATRG, 4D Ising", "unit": "ms",
        "higher_is_better": False, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "dtype": a.precision, "data": "synthetic",
        "config": {"workload": f"4D Ising beta={a.beta}, h=0, p=2D, q_swap=4, q_rho=4",
                   "precision": a.precision, "D": [r["D"] for r in rows]},
        "time_exponent_in_D": fits, "rows": rows}), flush=True)


def run_gemm(a):
    """One GEMM shape through trg_gemm (upload, product, download), warm-up then timed."""
    import numpy as np
    import paper_2507_21909_b300 as trg
    M, N, K = (int(v) for v in a.gemm.split(","))
    rng = np.random.default_rng(7)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    prec = PREC[a.precision]
    for _ in range(a.warmup):
        trg.trg_gemm(A, B, precision=prec)
    t = []
    trg.trg_kernel_stats(reset=True)
    for _ in range(max(a.steps, 1)):
        t0 = time.time()
        C = trg.trg_gemm(A, B, precision=prec)
        t.append(time.time() - t0)
    ks = trg.trg_kernel_stats(reset=True)
    kind = "x7" if a.precision == "oz7" else "oz" if a.precision.startswith("oz") else "tc"
    kms = ks[kind + "_ms"] / max(ks[kind + "_launches"], 1)
    rows = rng.choice(M, 8, replace=False)
    ref = A[rows] @ B
    err = float(np.abs(C[rows] - ref).max() / (np.abs(A[rows]) @ np.abs(B)).max())
    print(json.dumps({"metric": "trg_gemm wall time (upload + product + download)",
                      "unit": "ms", "value": 1e3 * statistics.median(t), "M": M, "N": N, "K": K,
                      "precision": a.precision, "sampled_rel_err": err,
                      "alg_flop": 2.0 * M * N * K,
                      "kernel_ms": kms, "kernel_launches": ks[kind + "_launches"],
                      "kernel_alg_tflops": 2.0 * M * N * K / kms / 1e9 if kms > 0 else None,
                      "kernel_pipe_tflops": (ks[kind + "_pipe_flop"] / max(ks[kind + "_launches"], 1)
                                             / kms / 1e9) if kms > 0 else None}), flush=True)


def reduce_timing(ms, steps, world, dist=None, device="cpu"):
    """Replicas: the slowest rank's timed region counts (max over ranks), and the value is
    the steps all ranks completed in that time."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * steps / (ms_max / 1e3)


# Traffic of the dominant kernel per launch (dram__bytes_read.sum + dram__bytes_write.sum,
# mean over the launches of one timed D = 48 OZ5 step of this script, from a one-pass ncu
# launch list with those two metrics), keyed by GEMM kind; a kind missing here has not
# been captured on the current build of its kernel.
TRAFFIC = {"oz": 2.662e9}


def roofline(stats, step_ms_total, steps, prec, peak, peak_src):
    """Roofline of the dominant kernel: the exact-digit GEMM (digit forms) or the split-BF16
    GEMM.  achieved = algorithmic flop (2 M N K of every product the step asks for, counted
    once) / the kernel's device time (CUDA events around each launch, on its stream);
    pipe_utilisation counts every BF16 digit / slice product as tensor-pipe work."""
    k = "oz" if 4 <= prec <= 6 else "x7" if prec == 8 else "tc"
    name = ("oz_gemm_kernel (exact-digit tcgen05 GEMM, %d digit products per product)"
            % {4: 10, 5: 15, 6: 21, 8: 28}.get(prec, 0) if k in ("oz", "x7") else
            "tc_gemm_kernel (split-BF16 or 3xTF32 tcgen05 GEMM, FP32 accumulation)")
    ms, alg, pipe, n = stats[k + "_ms"], stats[k + "_flop"], stats[k + "_pipe_flop"], stats[
        k + "_launches"]
    ach = alg / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    both_ms = stats["oz_ms"] + stats["tc_ms"] + stats["x7_ms"]
    return {
        "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
        "traffic": TRAFFIC.get(k), "traffic_unit": "DRAM bytes per launch (ncu, mean)",
        "peak_source": peak_src, "kernel": name,
        "flop": "algorithmic: 2 M N K per GEMM the step issues (FP64-equivalent product), "
                "digit/slice products not counted",
        "launches_per_step": n / steps, "alg_flop_per_launch": alg / n if n else 0.0,
        "ms_per_launch": ms / n if n else 0.0, "kernel_ms_per_step": ms / steps,
        "kernel_share_of_step": ms / step_ms_total,
        "pipe_utilisation": (pipe / (ms / 1e3) / 1e12 / peak) if ms > 0 else 0.0,
        "tensor_core_share_of_step": both_ms / step_ms_total,
        "step_alg_tflops": (stats["oz_flop"] + stats["tc_flop"] + stats["x7_flop"])
                           / (step_ms_total / 1e3) / 1e12,
        "by_kind_ms_per_step": {k2: stats[k2 + "_ms"] / steps for k2 in ("oz", "tc", "x7")},
    }


def run_ours(a):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    import paper_2507_21909_b300 as trg
    stream = torch.cuda.Stream()
    trg.trg_set_stream(stream.cuda_stream)
    prec = PREC[a.precision]
    D, p = a.D, 2 * a.D

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    learned = None
    if a.sketch == "learned":
        learned = train_sketch(trg, prec)
        trg.trg_set_sketch_mode(1)
        trg.trg_sketch_stats(reset=True)

    # ---- whole job, end to end from the host: init (H2D of T0), growth, warm-up, timed
    barrier()
    t_job = time.time()
    trg.trg_set_params(4, 4, 0x5EED, prec)
    trg.trg_set_bond_overspan(a.r_bond)
    trg.trg_init_ising(4, a.beta, 0.0)
    n = 0
    while True:  # grow the tensor until every leg reaches D and the bond r_bond D
        trg.trg_step(n % 4, D, p)
        _ = trg.trg_free_energy()
        n += 1
        dims = trg.trg_state_dims(0)
        if all(x == D for x in dims[:4]) and dims[4] == a.r_bond * D and n >= 4:
            break
        if n > 12:
            break
    n_grow = n
    for _ in range(a.warmup):
        trg.trg_step(n % 4, D, p)
        _ = trg.trg_free_energy()
        n += 1
    launches_before = trg.trg_kernel_stats()["launches"]
    trg.trg_kernel_stats(reset=True)
    clk = Clocks(local)
    clk.start()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    phases = {}
    torch.cuda.nvtx.range_push("timed_steps")
    ev0.record(stream)
    for _ in range(a.steps):
        trg.trg_step(n % 4, D, p)
        f_last = trg.trg_free_energy()
        n += 1
        for k, v in trg.trg_step_timings().items():
            phases[k] = phases.get(k, 0.0) + v / a.steps
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    clocks = clk.stop()
    t_job = time.time() - t_job
    ms = ev0.elapsed_time(ev1)
    stats = trg.trg_kernel_stats(reset=True)
    mem = trg.trg_mem_stats()
    ms, value = reduce_timing(ms, a.steps, world, dist, "cuda")
    e2e = world * (n - n_grow) / t_job   # full-size steps per second of the whole job
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak, peak_src = peaks()
    roof = roofline(stats, ms, a.steps, prec, peak, peak_src)
    line = {
        "metric": METRIC, "value": value, "unit": "RG steps/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic", "config": workload(a),
        "roofline": roof,
        "e2e": {"value": e2e, "unit": "RG steps/s", "h2d_bytes_per_step": 3 * 16 * 2 * 8 / n,
                "d2h_bytes_per_step": 16,
                "region": f"whole job from the host: trg_init_ising (H2D of T0), {n_grow} growth "
                          f"steps, {n - n_grow} full-size steps (warm-up + timed), each step "
                          "followed by trg_free_energy (D2H); value counts full-size steps"},
        "gpu_launches": stats["launches"],
        "timed_launch_range": [launches_before, launches_before + stats["launches"]],
        "clocks": clocks,
        "phases_ms": phases,
        "free_energy": f_last[0],
        "device_scratch_gb": {k: round(v / 2 ** 30, 2) for k, v in mem.items()},
    }
    if learned is not None:
        learned.update(trg.trg_sketch_stats())
        learned["oracle_residual_ratio_q0_D10"] = learned_gain(trg)
        line["config"]["sketch"] = "learned (row-weighted Gaussian, plain fallback)"
        line["learned_sketch"] = learned
    if not a.no_precision_check and prec != 0:
        mlp = net_dict(trg.trg_sketch_get_net()) if learned is not None else None
        line["delta_f_rel"] = precision_check(trg, prec, mlp, a.r_bond)
    if a.precision_steps > 0 and prec != 0:
        others = tuple(PREC[x] for x in a.also_forms.split(",") if x.strip())
        chk = precision_at_size(trg, prec, D, a.beta, a.precision_steps, stream, others)
        dfr = line.setdefault("delta_f_rel", {})
        dfr[f"vs_fp64_form_D{D}_per_step"] = chk["per_step"]
        dfr[f"vs_fp64_form_D{D}_max"] = chk["max"]
        dfr[f"fp64_form_D{D}_min_cut_gap_per_step"] = chk["fp64_form_min_gap_per_step"]
        line["fp64_form"] = {
            "value": chk["fp64_form_steps_per_s"], "unit": "RG steps/s",
            "measured": f"step {a.precision_steps - 1} of the FP64-form run above (input legs "
                        f"{chk['last_step_input_dims']}), CUDA events on the library stream",
            "ms_per_step": chk["fp64_form_ms_last_step"],
            "mixed_form_ms_same_step": chk["mixed_form_ms_last_step"],
            "speedup_of_value": value / chk["fp64_form_steps_per_s"]}
        if "other_forms" in chk:
            dfr[f"other_forms_vs_fp64_form_D{D}"] = chk["other_forms"]
    if a.fp64_form_steps > 0:
        r = fp64_form_rate(trg, D, a.fp64_form_steps, a.beta)
        line["fp64_form"] = {"value": r, "unit": "RG steps/s", "steps": a.fp64_form_steps,
                             "speedup_of_value": value / r}
    if not a.no_cpu_baseline:
        smp = OracleSample(D, a.beta, a.r_bond)
        smp.step()
        per, _ = smp.per_step(D)
        line["cpu_baseline"] = {"value": 1.0 / per, "unit": "RG steps/s",
                                "cores": os.cpu_count(), "kind": "oracle",
                                "sample": smp.describe(D)}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    a = args_()
    if a.impl == "reference":
        run_reference(a)
    elif a.gemm:
        run_gemm(a)
    elif a.batch > 0:
        run_batch(a)
    elif a.compare_atrg:
        run_compare_atrg(a)
    elif a.sensitivity:
        run_sensitivity(a)
    else:
        run_ours(a)
