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
PREC = {"fp64": 0, "bf16x3": 1, "bf16x6": 2, "bf16x10": 3, "oz4": 4, "oz5": 5, "oz6": 6}


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
    ap.add_argument("--precision-steps", type=int, default=0,
                    help="N > 0: also run N steps of the FP64 form and of the mixed form at "
                         "the bench's D and report dF/F per step (slow: FP64 form)")
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
    ap.add_argument("--r-bond", type=int, default=1,
                    help="ILO form: bond lines overspanned to r_bond D (1 = plain method)")
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
def oracle_sample(D, budget_s=25.0, r_bond=1):
    """Oracle time per step, from its dominant part: the coarse contraction (eqs.
    makeMG/makeMH) on D-sized triads (bond lines r_bond D) with the i1 leg cut to t = 1
    and 2 of D slices; T(t) = a + b t is extrapolated to t = D.  Other phases are not
    timed, so the result is an upper bound on the oracle's steps/s."""
    import numpy as np
    from oracle import trg_oracle as O
    chi, Db = 3 * D, r_bond * D
    rng = np.random.default_rng(0)
    times = {}
    for t in (1, 2):
        E = rng.standard_normal((t, chi, D, Db))
        F = rng.standard_normal((Db, chi, D, Db))
        G = rng.standard_normal((Db, chi, D, Db))
        H = rng.standard_normal((t, chi, D, Db))
        U = [rng.standard_normal((D, D, chi)) for _ in range(4)]
        Ms = {mu: rng.standard_normal((D, D, D)) for mu in (2, 3, 4)}
        t0 = time.time()
        O.contract_upper(E, F, U[0], U[1], Ms)
        O.contract_lower(G, H, U[2], U[3], Ms)
        times[t] = time.time() - t0
        if times[t] > budget_s:
            break
    b = max(times.get(2, times[1]) - times[1], 0.0)
    a0 = times[1] - b
    per_step = a0 + b * D
    return 1.0 / per_step, times, os.cpu_count()


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t0 = time.time()
    vals = []
    for _ in range(max(a.steps, 1)):
        v, times, cores = oracle_sample(a.D, r_bond=a.r_bond)
        vals.append(v)
    v = statistics.median(vals)
    sample = (f"coarse contraction (eqs. makeMG/makeMH) of one D={a.D} step with the i1 leg "
              f"cut to 1 and 2 of {a.D} slices, extrapolated linearly to {a.D}; other phases "
              f"not timed (upper bound); timings {times}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "RG steps/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 / v,
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
    """ΔF/F of the mixed form: against the FP64 CPU oracle at D=14 (16 steps; no
    near-degenerate truncation there) and against this library's FP64 form at D=24
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
    for D in [int(v) for v in a.compare_atrg.split(",") if v.strip()]:
        row = {"D": D, "p": 2 * D}
        for name, init, step in (
                ("triad", lambda: trg.trg_init_ising(4, a.beta, 0.0), trg.trg_step),
                ("atrg", lambda: trg.trg_atrg_init_ising(4, a.beta, 0.0), trg.trg_atrg_step)):
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
        row["f_atrg"] = trg.trg_atrg_free_energy()[0]
        row["atrg_over_triad"] = row["atrg_ms_per_step"] / row["triad_ms_per_step"]
        rows.append(row)
    print(json.dumps({
        "metric": "ms per RG step, triad-ATRG vs plain ATRG, 4D Ising", "unit": "ms",
        "higher_is_better": False, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "dtype": a.precision, "data": "synthetic",
        "config": {"workload": f"4D Ising beta={a.beta}, h=0, p=2D, q_swap=4, q_rho=4",
                   "precision": a.precision, "D": [r["D"] for r in rows]},
        "rows": rows}), flush=True)


def reduce_timing(ms, steps, world, dist=None, device="cpu"):
    """Replicas: the slowest rank's timed region counts (max over ranks), and the value is
    the steps all ranks completed in that time."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * steps / (ms_max / 1e3)


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
    ev0.record(stream)
    for _ in range(a.steps):
        trg.trg_step(n % 4, D, p)
        f_last = trg.trg_free_energy()
        n += 1
        for k, v in trg.trg_step_timings().items():
            phases[k] = phases.get(k, 0.0) + v / a.steps
    ev1.record(stream)
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
    achieved = stats["tc_flop"] / (stats["tc_ms"] / 1e3) / 1e12 if stats["tc_ms"] > 0 else 0.0
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
            "kernel": "tcgen05 GEMMs (oz_gemm_kernel digit products, tc_gemm_kernel BF16 splits); "
                      "flop = BF16 tensor work of every slice/digit product",
            "tc_launches": stats["tc_launches"], "tc_ms_per_step": stats["tc_ms"] / a.steps,
            "tc_share_of_step": stats["tc_ms"] / ms}
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
    if a.precision_steps > 0:
        per = []
        fs = {}
        for pr in (prec, 0):
            trg.trg_set_params(4, 4, 0x5EED, pr)
            trg.trg_init_ising(4, a.beta, 0.0)
            fs[pr] = []
            for k in range(a.precision_steps):
                trg.trg_step(k % 4, D, p)
                fs[pr].append(trg.trg_free_energy()[0])
        per = [abs(x - y) / abs(y) for x, y in zip(fs[prec], fs[0])]
        dfr = line.setdefault("delta_f_rel", {})
        dfr[f"vs_fp64_form_D{D}_per_step"] = per
        dfr[f"vs_fp64_form_D{D}_max"] = max(per)
    if a.fp64_form_steps > 0:
        r = fp64_form_rate(trg, D, a.fp64_form_steps, a.beta)
        line["fp64_form"] = {"value": r, "unit": "RG steps/s", "steps": a.fp64_form_steps,
                             "speedup_of_value": value / r}
    if not a.no_cpu_baseline:
        v, times, cores = oracle_sample(D, r_bond=a.r_bond)
        line["cpu_baseline"] = {
            "value": v, "unit": "RG steps/s", "cores": cores, "kind": "oracle",
            "sample": f"coarse contraction (eqs. makeMG/makeMH) of one D={D} step with the i1 "
                      f"leg cut to 1 and 2 slices, extrapolated to {D}; other phases not timed"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    a = args_()
    if a.impl == "reference":
        run_reference(a)
    elif a.batch > 0:
        run_batch(a)
    elif a.compare_atrg:
        run_compare_atrg(a)
    else:
        run_ours(a)
